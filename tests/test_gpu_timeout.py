"""The timeout path of the tensor-core products' bounded waits, exercised without faulting the GPU.

mdc_plan_set_wait_probe makes every CTA of the split-BF16 tile kernels wait, before any copy or product is
issued, on an mbarrier that nothing arrives on, for a few thousand cycles.  The wait gives up, and the CTA
must then do what it does after a real timeout: record MDC_ERR_TIMEOUT in the plan's status word, write
no products, free its tensor memory and return.  The checks: the status, the products left unwritten
(the spectral workspaces keep what the previous call left there), and the next calls of the same plan
correct against the FP64 oracle (the context and the tensor memory are usable again).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_04486_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu

PROBE_CYCLES = 20000


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    binding.load_library()


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("recip", [False, True])
def test_bounded_wait_gives_up_cleanly(recip):
    nt, n, ns, nb = 200, 150, 160, 12
    Dn = synth.random_traces((ns, n, nt), 1).astype(np.float32)
    Xn = synth.random_traces((n, n, nt), 2).astype(np.float32)
    Rn = synth.random_traces((nb, n, nt), 3).astype(np.float32)
    ia, ib = synth.random_indices(ns, nb, 4), synth.random_indices(ns, nb, 5)
    plan = binding.MDCPlan(_cuda(Dn), n, nb_max=nb, precision=binding.MDC_PREC_BF16X3)
    plan.set_config(fft_variant=0, gemm_fwd=binding.MDC_GEMM_TC, gemm_adj=binding.MDC_GEMM_TC)
    X, R = _cuda(Xn), _cuda(Rn)
    Ua = plan.forward(X, _cuda(ia, torch.int32)).clone()
    assert plan.sync_status() == binding.MDC_OK

    binding.mdc_plan_set_wait_probe(plan.handle, PROBE_CYCLES)
    # forward on another batch: the products are not written, so the inverse transform reads the batch
    # spectra of the previous call and returns its result unchanged
    Ub = plan.forward(X, _cuda(ib, torch.int32))
    assert plan.sync_status() == binding.MDC_ERR_TIMEOUT
    assert torch.equal(Ub, Ua)
    # adjoint: the gradient spectra share the buffer of the model spectra the forward call left, so the
    # inverse transform returns the model itself (up to FFT rounding) instead of a gradient
    G = torch.empty_like(X)
    if recip:
        binding.smdd_step(plan.handle, G.copy_(X), _cuda(np.zeros((ns, n, nt), np.float32)),
                          _cuda(ib, torch.int32), 0.0, binding.SMDD_RECIPROCITY)
        assert plan.sync_status() == binding.MDC_ERR_TIMEOUT
    else:
        plan.adjoint(R, _cuda(ib, torch.int32), out=G)
        assert plan.sync_status() == binding.MDC_ERR_TIMEOUT
        assert oracle.rel_l2(G.double().cpu().numpy(), Xn) <= 1e-5
    assert plan.sync_status() == binding.MDC_OK          # the status word was cleared by the read

    binding.mdc_plan_set_wait_probe(plan.handle, 0)
    U = plan.forward(X, _cuda(ib, torch.int32)).double().cpu().numpy()
    G = plan.adjoint(R, _cuda(ib, torch.int32)).double().cpu().numpy()
    assert plan.sync_status() == binding.MDC_OK
    assert oracle.rel_l2(U, oracle.mdc_forward(Dn, Xn, ib)) <= 1e-4
    assert oracle.rel_l2(G, oracle.mdc_adjoint(Dn, Rn, ib)) <= 1e-4


def test_wait_probe_arguments():
    plan = binding.MDCPlan(_cuda(synth.random_traces((4, 3, 16), 1)), 3, precision=binding.MDC_PREC_BF16X3)
    for bad in (-1, 10 ** 9):
        with pytest.raises(binding.MDCError) as e:
            binding.mdc_plan_set_wait_probe(plan.handle, bad)
        assert e.value.status == binding.MDC_ERR_INVALID_ARG
    binding.mdc_plan_set_wait_probe(plan.handle, 0)

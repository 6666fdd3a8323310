"""GPU parity of the full-gradient LSQR solver (smdd_lsqr) against the oracle's LSQR (Paige & Saunders)
on the same preconditioned operator.

Bar: relative L2 <= 1e-4 on X and on the residual-norm estimates after 10 iterations (the stated FP32
operator bound of 1e-5 per application, carried through the recurrence's 20 operator applications in
FP32 vectors with FP64 norms)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_04486_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    binding.load_library()


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("recip,use_mute", [(False, False), (True, False), (True, True), (False, True)])
def test_lsqr_matches_oracle(recip, use_mute):
    nt, n, ns = 128, 32, 32
    p = synth.make_problem(nt, n, n, ns, dx=40.0, n_reflectors=3, n_multiples=2, seed=3)
    D = p.D.astype(np.float32).astype(np.float64)
    U = oracle.mdc_forward(D, p.X_true.astype(np.float32).astype(np.float64), np.arange(ns))
    U = (U + 0.05 * np.sqrt(np.mean(U ** 2)) * p.noise).astype(np.float32).astype(np.float64)
    mute = synth.direct_arrival_mute(n, n, nt, dx=40.0) if use_mute else None
    X_ref, n_ref = oracle.mdc_lsqr(D, np.zeros((n, n, nt)), U, 10, recip=recip, mute=mute)
    plan = binding.MDCPlan(_cuda(D), n, nb_max=ns)
    X = torch.zeros((n, n, nt), device="cuda")
    norms = torch.zeros(11, device="cuda", dtype=torch.float64)
    binding.smdd_lsqr(plan.handle, X, _cuda(U), 10, binding.SMDD_RECIPROCITY if recip else 0,
                      None if mute is None else _cuda(mute, torch.int32), norms)
    assert plan.sync_status() == binding.MDC_OK
    assert oracle.rel_l2(X.double().cpu().numpy(), X_ref) <= 1e-4
    assert oracle.rel_l2(norms.cpu().numpy(), np.array(n_ref)) <= 1e-4
    assert n_ref[-1] < 0.5 * n_ref[0]
    if recip:
        Xh = X.cpu().numpy()
        np.testing.assert_allclose(Xh, np.transpose(Xh, (1, 0, 2)), rtol=0, atol=1e-6 * np.abs(Xh).max())


def test_lsqr_from_nonzero_start_and_errors():
    nt, nr, nv, ns = 100, 12, 9, 15
    D = synth.random_traces((ns, nr, nt), 5).astype(np.float32).astype(np.float64)
    U = synth.random_traces((ns, nv, nt), 6).astype(np.float32).astype(np.float64)
    X0 = synth.random_traces((nv, nr, nt), 7).astype(np.float32).astype(np.float64)
    X_ref, _ = oracle.mdc_lsqr(D, X0, U, 6)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=ns)
    X = _cuda(X0)
    binding.smdd_lsqr(plan.handle, X, _cuda(U), 6)
    assert plan.sync_status() == binding.MDC_OK
    assert oracle.rel_l2(X.double().cpu().numpy(), X_ref) <= 1e-4
    small = binding.MDCPlan(_cuda(D), nv, nb_max=4)          # cannot hold every source in one batch
    with pytest.raises(binding.MDCError) as e:
        binding.smdd_lsqr(small.handle, X, _cuda(U), 2)
    assert e.value.status == binding.MDC_ERR_SHAPE
    with pytest.raises(binding.MDCError) as e:
        binding.smdd_lsqr(plan.handle, X, _cuda(U), 2, binding.SMDD_RECIPROCITY)   # nr != nv
    assert e.value.status == binding.MDC_ERR_SHAPE

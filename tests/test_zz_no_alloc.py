"""The allocation-free forward entry point (mdc_forward_static) against the plan-based mdc_forward and
the FP64 oracle.

mdc_forward_static serves callers that may not allocate device memory (their device memory belongs to
another allocator or pool, or they cannot afford an allocation's latency); it keeps its intermediates in
a static device array.  Its output must match the plan path within the tolerance of the parity tests,
on consecutive calls that reuse the same array.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_04486_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
ELEM = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    binding.load_library()


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("shape", [(130, 21, 19, 23, 7), (128, 32, 32, 32, 8)], ids=["ragged", "aligned"])
def test_forward_static_matches_plan_on_consecutive_calls(shape):
    nt, nr, nv, ns, nb = shape
    Dn = synth.random_traces((ns, nr, nt), 1).astype(np.float32)
    D = _cuda(Dn)
    plan = binding.MDCPlan(D, nv, nb_max=nb, scale=0.5)
    for call in range(2):
        Xn = synth.random_traces((nv, nr, nt), 10 + call).astype(np.float32)
        idxn = synth.random_indices(ns, nb, 20 + call)
        X = _cuda(Xn)
        idx = _cuda(idxn, torch.int32)
        ref = plan.forward(X, idx).double()
        U = torch.full((nb, nv, nt), float("nan"), device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        binding.mdc_forward_static(D, X, idx, U, scale=0.5, dev_status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        # against the plan-based entry point
        err = (U.double() - ref)
        rel = (err.norm() / ref.norm()).item()
        elem = (err.abs().max() / ref.abs().max()).item()
        assert rel <= REL_L2, (call, rel)
        assert elem <= ELEM, (call, elem)
        # and against the FP64 direct sums of the oracle
        exact = oracle.mdc_forward(Dn, Xn, idxn, scale=0.5)
        Un = U.double().cpu().numpy()
        assert oracle.rel_l2(Un, exact) <= REL_L2, call
        assert np.abs(Un - exact).max() <= ELEM * np.abs(exact).max(), call


def test_forward_static_reports_index_errors():
    """An index outside [0, ns) sets the caller's status word and gives zero rows; the next call with
    valid indices is unaffected (the status word is the caller's, cleared by the caller)."""
    nt, nr, nv, ns, nb = 64, 5, 3, 4, 3
    Dn = synth.random_traces((ns, nr, nt), 2).astype(np.float32)
    Xn = synth.random_traces((nv, nr, nt), 3).astype(np.float32)
    D, X = _cuda(Dn), _cuda(Xn)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    U = torch.full((nb, nv, nt), float("nan"), device="cuda")
    binding.mdc_forward_static(D, X, _cuda(np.array([1, ns, 2]), torch.int32), U, dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 1
    assert torch.all(U[1] == 0)
    exact = oracle.mdc_forward(Dn, Xn, np.array([1, 2]))
    assert oracle.rel_l2(U[[0, 2]].double().cpu().numpy(), exact) <= REL_L2
    status.zero_()
    binding.mdc_forward_static(D, X, _cuda(np.array([0, 3, 2]), torch.int32), U, dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert oracle.rel_l2(U.double().cpu().numpy(), oracle.mdc_forward(Dn, Xn, np.array([0, 3, 2]))) <= REL_L2


def test_forward_static_rejects_problems_beyond_its_scratch():
    nt, nr, nv, ns, nb = 4096, 64, 64, 64, 4     # model spectra alone need about 134 MB
    D = torch.zeros((ns, nr, nt), device="cuda")
    X = torch.zeros((nv, nr, nt), device="cuda")
    idx = torch.zeros(nb, dtype=torch.int32, device="cuda")
    U = torch.zeros((nb, nv, nt), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(binding.MDCError) as e:
        binding.mdc_forward_static(D, X, idx, U, dev_status=status)
    assert e.value.status == binding.MDC_ERR_UNSUPPORTED

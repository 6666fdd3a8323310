"""The allocation-free forward entry point (mdc_forward_static) against the plan-based mdc_forward.

mdc_forward_static serves callers that may not allocate device memory (their device memory belongs to
another allocator or pool, or they cannot afford an allocation's latency); it keeps its intermediates in
a static device array.  Its output must match the plan path within the tolerance of the parity tests,
on consecutive calls that reuse the same array.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

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
    D = _cuda(synth.random_traces((ns, nr, nt), 1))
    plan = binding.MDCPlan(D, nv, nb_max=nb, scale=0.5)
    for call in range(2):
        X = _cuda(synth.random_traces((nv, nr, nt), 10 + call))
        idx = _cuda(synth.random_indices(ns, nb, 20 + call), torch.int32)
        ref = plan.forward(X, idx).double()
        U = torch.full((nb, nv, nt), float("nan"), device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        binding.mdc_forward_static(D, X, idx, U, scale=0.5, dev_status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        err = (U.double() - ref)
        rel = (err.norm() / ref.norm()).item()
        elem = (err.abs().max() / ref.abs().max()).item()
        assert rel <= REL_L2, (call, rel)
        assert elem <= ELEM, (call, elem)


def test_forward_static_rejects_problems_beyond_its_scratch():
    nt, nr, nv, ns, nb = 4096, 64, 64, 64, 4     # model spectra alone need about 134 MB
    D = torch.zeros((ns, nr, nt), device="cuda")
    X = torch.zeros((nv, nr, nt), device="cuda")
    idx = torch.zeros(nb, dtype=torch.int32, device="cuda")
    U = torch.zeros((nb, nv, nt), device="cuda")
    with pytest.raises(binding.MDCError) as e:
        binding.mdc_forward_static(D, X, idx, U)
    assert e.value.status == binding.MDC_ERR_UNSUPPORTED

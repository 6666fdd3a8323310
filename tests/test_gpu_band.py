"""Band-limited products (mdc_plan_set_band): the GPU operator restricted to the bins f < band against the
oracle's band-limited Tier B (FP32 bar: relative L2 <= 1e-5), and its error against the exact operator on
the Ricker workload with the band at 3 f0 (stated and bounded: <= 1e-2)."""
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


@pytest.mark.parametrize("precision", [binding.MDC_PREC_FP32, binding.MDC_PREC_BF16X3], ids=["fp32", "bf16x3"])
@pytest.mark.parametrize("recip", [False, True])
def test_band_limited_operator(precision, recip):
    nt, n, ns, nb = 128, 32, 40, 8
    p = synth.make_problem(nt, n, n, ns, dx=10.0, n_reflectors=3, n_multiples=2, seed=0)
    D = p.D.astype(np.float32).astype(np.float64)
    X = p.X_true.astype(np.float32).astype(np.float64)
    R = synth.random_traces((nb, n, nt), 5).astype(np.float32).astype(np.float64)
    idx = synth.random_indices(ns, nb, 6)
    nfft = oracle.default_nfft(nt)
    band = int(np.ceil(3 * synth.F0 * nfft * synth.DT)) + 1        # bins up to 3 f0
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb, precision=precision)
    plan.set_band(band)
    ti = _cuda(idx, torch.int32)
    U = plan.forward(_cuda(X), ti).double().cpu().numpy()
    G = plan.adjoint(_cuda(R), ti).double().cpu().numpy()
    tol = 1e-5 if precision == binding.MDC_PREC_FP32 else 1e-4
    U_band = oracle.mdc_forward_fft(D, X, idx, band=band)
    assert oracle.rel_l2(U, U_band) <= tol
    assert oracle.rel_l2(G, oracle.mdc_adjoint_fft(D, R, idx, band=band)) <= tol
    # approximation error of the band limit on band-limited (Ricker) data
    assert oracle.rel_l2(U_band, oracle.mdc_forward(D, X, idx)) <= 1e-2
    # a step with the band limit equals the oracle's step with the same band; set_band(0) restores
    U_obs = oracle.mdc_forward(D, X, np.arange(ns)).astype(np.float32).astype(np.float64)
    alpha = 0.3 / oracle.sigma2_max(D)
    Xg = torch.zeros((n, n, nt), device="cuda")
    binding.smdd_step(plan.handle, Xg, _cuda(U_obs), ti, alpha, binding.SMDD_RECIPROCITY if recip else 0)
    Rr = oracle.mdc_forward_fft(D, np.zeros((n, n, nt)), idx, band=band) - U_obs[idx]
    g = oracle.mdc_adjoint_fft(D, Rr, idx, band=band)
    if recip:
        g = oracle.reciprocity(g)
    assert oracle.rel_l2(Xg.double().cpu().numpy(), -alpha * g) <= tol
    plan.set_band(0)
    U0 = plan.forward(_cuda(X), ti).double().cpu().numpy()
    assert oracle.rel_l2(U0, oracle.mdc_forward(D, X, idx)) <= tol
    assert plan.sync_status() == binding.MDC_OK

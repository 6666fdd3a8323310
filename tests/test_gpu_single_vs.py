"""Single virtual source (nv = 1, the matrix-vector regime of the per-frequency products) on the Volve-like
line of 180 receivers and 110 sources, nt = 1024: forward, adjoint and SGD / N-SGD steps against the FP64
oracle with the FP32 bar (relative L2 <= 1e-5, elementwise <= 2e-5 of max|ref|), for both precisions
of the products (split BF16: 1e-4)."""
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
def test_single_virtual_source(precision):
    w = synth.WORKLOADS["smdd_nt1024_nr180_nv1_ns110_nb16"]
    nt, nr, nv, ns, nb = w["nt"], w["nr"], w["nv"], w["ns"], w["nb"]
    p = synth.make_problem(nt, nr, nv, ns, dx=w["dx"], n_reflectors=w["n_reflectors"], n_multiples=w["n_multiples"],
                           seed=0)
    D = p.D.astype(np.float32).astype(np.float64)
    Xt = p.X_true.astype(np.float32).astype(np.float64)
    idx = synth.epoch_batches(ns, nb, 1, seed=0)[0][0]
    R = synth.random_traces((nb, nv, nt), 3).astype(np.float32).astype(np.float64)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, precision=precision)
    ti = _cuda(idx, torch.int32)
    tol = 1e-5 if precision == binding.MDC_PREC_FP32 else 1e-4
    U = plan.forward(_cuda(Xt), ti).double().cpu().numpy()
    U_ref = oracle.mdc_forward(D, Xt, idx)
    assert oracle.rel_l2(U, U_ref) <= tol
    assert np.max(np.abs(U - U_ref)) <= 2 * tol * np.max(np.abs(U_ref))
    G = plan.adjoint(_cuda(R), ti).double().cpu().numpy()
    assert oracle.rel_l2(G, oracle.mdc_adjoint(D, R, idx)) <= tol
    # a few SGD and N-SGD steps from zero
    U_obs = oracle.mdc_forward_fft(D, Xt, np.arange(ns)).astype(np.float32).astype(np.float64)
    alpha = 0.5 * 2.0 / oracle.sigma2_max(D)
    batches = synth.epoch_batches(ns, nb, 1, seed=1)[0][:3]
    Xs, Xn, V = (torch.zeros((nv, nr, nt), device="cuda") for _ in range(3))
    Xr, Xnr, Vr = np.zeros((nv, nr, nt)), np.zeros((nv, nr, nt)), np.zeros((nv, nr, nt))
    Ug = _cuda(U_obs)
    for k, b in enumerate(batches):
        bi = _cuda(b, torch.int32)
        fl = binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
        binding.smdd_step(plan.handle, Xs, Ug, bi, alpha, fl)
        Xr, _ = oracle.sgd_step(D, Xr, U_obs, b, alpha, fft=True)
    plan2 = binding.MDCPlan(_cuda(D), nv, nb_max=nb, precision=precision)
    for k, b in enumerate(batches):
        bi = _cuda(b, torch.int32)
        fl = binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0) | binding.SMDD_NESTEROV
        binding.smdd_step_ex(plan2.handle, Xn, Ug, bi, alpha, fl, V=V, mu=0.9)
        Xnr, Vr, _ = oracle.nsgd_step(D, Xnr, Vr, U_obs, b, alpha, 0.9, fft=True)
    assert plan.sync_status() == binding.MDC_OK and plan2.sync_status() == binding.MDC_OK
    assert oracle.rel_l2(Xs.double().cpu().numpy(), Xr) <= tol
    assert oracle.rel_l2(Xn.double().cpu().numpy(), Xnr) <= tol


@pytest.mark.parametrize("shape", [(1024, 180, 1, 110, 16), (257, 37, 3, 41, 7), (130, 8, 8, 12, 5), (64, 70, 5, 80, 70)],
                         ids=lambda s: "x".join(map(str, s)))
def test_matrix_vector_kernels(shape):
    """The matrix-vector products for few virtual sources (MDC_GEMM_GEMV) against the oracle; with
    reciprocity (nr = nv <= 8) and with a band limit the call falls back to the tiled kernels."""
    nt, nr, nv, ns, nb = shape
    seed = sum(shape)
    D = synth.random_traces((ns, nr, nt), seed).astype(np.float32).astype(np.float64)
    X = synth.random_traces((nv, nr, nt), seed + 1).astype(np.float32).astype(np.float64)
    R = synth.random_traces((nb, nv, nt), seed + 2).astype(np.float32).astype(np.float64)
    idx = synth.random_indices(ns, nb, seed + 3, replace=nb > ns)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    plan.set_config(gemm_fwd=binding.MDC_GEMM_GEMV, gemm_adj=binding.MDC_GEMM_GEMV)
    ti = _cuda(idx, torch.int32)
    U = plan.forward(_cuda(X), ti).double().cpu().numpy()
    G = plan.adjoint(_cuda(R), ti).double().cpu().numpy()
    assert plan.sync_status() == binding.MDC_OK
    U_ref, G_ref = oracle.mdc_forward(D, X, idx), oracle.mdc_adjoint(D, R, idx)
    assert oracle.rel_l2(U, U_ref) <= 1e-5 and np.max(np.abs(U - U_ref)) <= 2e-5 * np.max(np.abs(U_ref))
    assert oracle.rel_l2(G, G_ref) <= 1e-5 and np.max(np.abs(G - G_ref)) <= 2e-5 * np.max(np.abs(G_ref))
    if nr == nv:   # reciprocity step: the adjoint runs the tiled kernel
        U_obs = synth.random_traces((ns, nv, nt), seed + 4).astype(np.float32).astype(np.float64)
        alpha = 0.3 / oracle.sigma2_max(D)
        Xg = _cuda(X)
        binding.smdd_step(plan.handle, Xg, _cuda(U_obs), ti, alpha, binding.SMDD_RECIPROCITY)
        Xr, _ = oracle.sgd_step(D, X, U_obs, idx, alpha, recip=True)
        assert plan.sync_status() == binding.MDC_OK
        assert oracle.rel_l2(Xg.double().cpu().numpy(), Xr) <= 1e-5
    plan.set_band(plan.nf // 2)          # band limit: the tiled kernels, with zero bins above the band
    Ub = plan.forward(_cuda(X), ti).double().cpu().numpy()
    assert oracle.rel_l2(Ub, oracle.mdc_forward_fft(D, X, idx, band=plan.nf // 2)) <= 1e-5


def test_matrix_vector_kernels_need_few_virtual_sources():
    D = _cuda(synth.random_traces((5, 4, 16), 9))
    plan = binding.MDCPlan(D, 9, nb_max=2)
    with pytest.raises(binding.MDCError) as e:
        plan.set_config(gemm_fwd=binding.MDC_GEMM_GEMV)
    assert e.value.status == binding.MDC_ERR_UNSUPPORTED

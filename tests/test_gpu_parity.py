"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle, element by element.

Tolerances (FP32 path, derived from the arithmetic): every output is a sum of products formed through
two length-N FP32 FFTs and an FP32 complex product of inner length K; the rounding error of such a
result is of order eps32 * (log2 N + sqrt K) times the magnitude of the largest terms, i.e. a few 1e-6
of max|output| for the sizes here.  The bar is the one stated for the FP32 path:
  * relative L2 error <= 1e-5 for U and for the gradient, and
  * elementwise |gpu - oracle| <= 2e-5 * max|oracle| (a uniform bound, since FFT rounding errors spread
    over all samples of a trace instead of scaling with each sample).
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


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _check(gpu, ref, what, rel=REL_L2, elem=ELEM):
    gpu = np.asarray(gpu, dtype=np.float64)
    r = oracle.rel_l2(gpu, ref)
    m = np.max(np.abs(gpu - ref)) / max(np.max(np.abs(ref)), 1e-30)
    assert r <= rel, f"{what}: relative L2 {r:.3e} > {rel:.1e}"
    assert m <= elem, f"{what}: max elementwise error {m:.3e} of max|ref| > {elem:.1e}"
    return r, m


# (nt, nr, nv, ns, nb): several tiles of every kernel, ragged tails, odd sizes, every FFT length
SHAPES = [
    (128, 32, 32, 32, 8),        # small workload shape (nfft 256)
    (100, 37, 29, 41, 5),        # ragged everything
    (1, 3, 2, 4, 3),             # a single time sample
    (33, 5, 7, 6, 9),            # nb > ns: duplicate sources
    (257, 17, 19, 23, 17),       # odd nt, nfft 1024, two batch tiles in the forward product
    (600, 20, 20, 20, 4),        # nfft 2048
    (1500, 6, 5, 7, 3),          # nfft 3072 (radix 8 * 8 * 3 * 8)
    (1536, 5, 6, 4, 5),          # nfft 3072, nt = M: no zero padding inside the first half
    (1800, 6, 5, 7, 3),          # nfft 4096
    (2500, 3, 2, 4, 2),          # nfft 8192
    (64, 70, 65, 80, 20),        # several 64x64 adjoint tiles, two forward batch tiles
    (16, 300, 260, 10, 3),       # nv > 256: two forward row blocks
    (6, 4, 3, 5, 2),             # nt = 2 mod 4: traces not 16-byte aligned (scalar time I/O)
    (130, 9, 11, 12, 7),         # nt = 2 mod 4, nfft 512
]


def _problem(nt, nr, nv, ns, nb, seed):
    D = _f32(synth.random_traces((ns, nr, nt), seed))
    X = _f32(synth.random_traces((nv, nr, nt), seed + 1))
    R = _f32(synth.random_traces((nb, nv, nt), seed + 2))
    idx = synth.random_indices(ns, nb, seed + 3, replace=nb > ns)
    return D, X, R, idx


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_forward_matches_oracle(shape):
    nt, nr, nv, ns, nb = shape
    D, X, _, idx = _problem(nt, nr, nv, ns, nb, seed=sum(shape))
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, scale=0.5)
    U = plan.forward(_cuda(X), _cuda(idx, torch.int32)).cpu().numpy()
    assert plan.sync_status() == binding.MDC_OK
    _check(U, oracle.mdc_forward(D, X, idx, 0.5), f"U {shape}")


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_adjoint_matches_oracle(shape):
    nt, nr, nv, ns, nb = shape
    D, _, R, idx = _problem(nt, nr, nv, ns, nb, seed=2 * sum(shape))
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, scale=0.5)
    G = plan.adjoint(_cuda(R), _cuda(idx, torch.int32)).cpu().numpy()
    assert plan.sync_status() == binding.MDC_OK
    _check(G, oracle.mdc_adjoint(D, R, idx, 0.5), f"G {shape}")


@pytest.mark.parametrize("shape", [(128, 32, 32, 32, 8), (257, 17, 19, 23, 17), (512, 40, 33, 50, 16)])
def test_dot_product_on_gpu(shape):
    """<P x, y> = <x, P^H y> for the GPU operator pair, inner products in FP64."""
    nt, nr, nv, ns, nb = shape
    D, X, Y, idx = _problem(nt, nr, nv, ns, nb, seed=7)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    ti = _cuda(idx, torch.int32)
    U = plan.forward(_cuda(X), ti).double().cpu().numpy()
    G = plan.adjoint(_cuda(Y), ti).double().cpu().numpy()
    lhs, rhs = np.vdot(U, Y), np.vdot(X, G)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(U) * np.linalg.norm(Y)


def test_delta_kernel_shifts_model_on_gpu():
    n, nt, nv, k = 6, 40, 5, 3
    D = np.zeros((n, n, nt))
    for s in range(n):
        D[s, s, k] = 1.0
    X = _f32(synth.random_traces((nv, n, nt), 5))
    idx = np.array([5, 0, 2, 2], np.int32)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=4)
    U = plan.forward(_cuda(X), _cuda(idx, torch.int32)).cpu().numpy().astype(np.float64)
    ref = np.zeros_like(U)
    for b, s in enumerate(idx):
        ref[b, :, k:] = X[:, s, :nt - k]
    assert np.max(np.abs(U - ref)) <= 1e-5 * np.max(np.abs(X))


@pytest.mark.parametrize("recip", [False, True])
@pytest.mark.parametrize("shape", [(128, 32, 32, 32, 8), (100, 37, 37, 41, 5), (64, 70, 70, 80, 20)])
def test_smdd_step_matches_oracle(shape, recip):
    nt, nr, nv, ns, nb = shape
    D, X, _, idx = _problem(nt, nr, nv, ns, nb, seed=11)
    if recip:
        X = _f32(0.5 * (X + X.transpose(1, 0, 2)))
    U_obs = _f32(synth.random_traces((ns, nv, nt), 12))
    alpha = 1e-4
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    Xg = _cuda(X)
    loss = torch.zeros((), device="cuda", dtype=torch.float64)
    plan.step(Xg, _cuda(U_obs), _cuda(idx, torch.int32), alpha,
              binding.SMDD_RECIPROCITY if recip else 0, loss)
    assert plan.sync_status() == binding.MDC_OK
    g, l_ref, _ = oracle.gradient(D, X, U_obs, idx)
    if recip:
        g = oracle.reciprocity(g)
    _check((X - Xg.double().cpu().numpy()) / alpha, g, f"step gradient {shape} recip={recip}", rel=1e-4, elem=2e-4)
    Xn_ref = X - alpha * g
    assert oracle.rel_l2(Xg.double().cpu().numpy(), Xn_ref) <= 1e-6
    assert abs(loss.item() - l_ref) <= 1e-5 * l_ref
    if recip:
        Xo = Xg.cpu().numpy()
        np.testing.assert_array_equal(Xo, Xo.transpose(1, 0, 2))


def test_step_gradient_exact_parity_via_adjoint():
    """The gradient the fused step applies equals adjoint(forward(X) - U_obs) at FP32 parity with the oracle,
    measured with alpha = 1 so that the difference X - X_new carries the full gradient."""
    nt, nr, nv, ns, nb = 128, 32, 32, 32, 8
    D, X, _, idx = _problem(nt, nr, nv, ns, nb, seed=21)
    X = np.zeros_like(X)
    U_obs = _f32(synth.random_traces((ns, nv, nt), 22))
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    Xg = _cuda(X)
    plan.step(Xg, _cuda(U_obs), _cuda(idx, torch.int32), 1.0, 0)
    g, _, _ = oracle.gradient(D, X, U_obs, idx)
    _check(-Xg.double().cpu().numpy(), g, "gradient at X=0")


def test_gathered_uobs_and_reuse_of_model_spectra():
    nt, nr, nv, ns, nb = 128, 24, 24, 30, 6
    D, X, _, _ = _problem(nt, nr, nv, ns, nb, seed=31)
    U_obs = _f32(synth.random_traces((ns, nv, nt), 32))
    batches = synth.epoch_batches(ns, nb, 2, seed=3)
    plan_a = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    plan_b = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    Xa, Xb = _cuda(X), _cuda(X)
    Ug = _cuda(U_obs)
    la = torch.zeros((), device="cuda", dtype=torch.float64)
    lb = torch.zeros((), device="cuda", dtype=torch.float64)
    first = True
    for ep in batches:
        for idx in ep:
            ti = _cuda(idx, torch.int32)
            plan_a.step(Xa, Ug, ti, 2e-4, binding.SMDD_RECIPROCITY, la)
            fl = binding.SMDD_RECIPROCITY | binding.SMDD_KEEP_XHAT | binding.SMDD_UOBS_GATHERED
            if not first:
                fl |= binding.SMDD_REUSE_XHAT
            plan_b.step(Xb, Ug[ti.long()].contiguous(), ti, 2e-4, fl, lb)
            first = False
            assert abs(la.item() - lb.item()) <= 1e-6 * la.item()
    assert oracle.rel_l2(Xb.double().cpu().numpy(), Xa.double().cpu().numpy()) <= 1e-6


def test_trajectory_small_workload_matches_oracle():
    """50 epochs of SGD with batches of 8 on the nt=128, 32x32x32 Ricker workload, against the FP64 oracle
    trajectory from the same batches.  Relative L2 of the final model and of the per-step losses."""
    w = synth.WORKLOADS["smdd_nt128_n32_nb8"]
    p = synth.make_problem(w["nt"], 32, 32, 32, dx=w["dx"], n_reflectors=w["n_reflectors"],
                           n_multiples=w["n_multiples"], seed=0)
    D = _f32(p.D)
    U_obs = _f32(oracle.mdc_forward(D, _f32(p.X_true), np.arange(32)))
    batches = synth.epoch_batches(32, w["nb"], 50, seed=0)
    alpha = 0.5 * 2.0 / oracle.sigma2_max(D)
    X_ref, l_ref = oracle.run_epochs(D, np.zeros_like(p.X_true), U_obs, batches, alpha, fft=True)

    plan = binding.MDCPlan(_cuda(D), 32, nb_max=w["nb"])
    Xg = torch.zeros((32, 32, w["nt"]), device="cuda")
    Ug = _cuda(U_obs)
    losses = torch.zeros(len(l_ref), device="cuda", dtype=torch.float64)
    k = 0
    for ep in batches:
        for idx in ep:
            fl = binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
            binding.smdd_step(plan.handle, Xg, Ug, _cuda(idx, torch.int32), alpha, fl, losses[k])
            k += 1
    assert plan.sync_status() == binding.MDC_OK
    assert oracle.rel_l2(Xg.double().cpu().numpy(), X_ref) <= 1e-4
    assert oracle.rel_l2(losses.cpu().numpy(), np.array(l_ref)) <= 1e-4
    assert l_ref[-1] < 0.2 * l_ref[0]


def test_sigma2_power_iteration_matches_oracle():
    p = synth.make_problem(128, 24, 24, 30, dx=10.0, seed=4)
    D = _f32(p.D)
    plan = binding.MDCPlan(_cuda(D), 24, nb_max=8, scale=0.7)
    s2 = plan.sigma2_max(200)
    ref = oracle.sigma2_max(D, scale=0.7)
    assert s2 <= ref * (1 + 1e-5)
    assert s2 >= ref * (1 - 1e-3)


def test_large_workload_sampled_columns():
    """nt=512, 201x201x201, batch 16 with reciprocity (the configuration the benchmark times): every
    output of the fused step is checked on sampled traces against the oracle's direct sums."""
    w = synth.WORKLOADS["smdd_nt512_n201_nb16_recip"]
    n, nt, nb = 201, w["nt"], w["nb"]
    p = synth.make_problem(nt, n, n, n, dx=w["dx"], n_reflectors=w["n_reflectors"], n_multiples=w["n_multiples"],
                           seed=0)
    D = _f32(p.D)
    X = _f32(0.3 * p.X_true)                                   # symmetric
    U_obs = _f32(synth.random_traces((n, n, nt), 9))
    idx = synth.epoch_batches(n, nb, 1, seed=0)[0][0]
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb)
    Xg = _cuda(X)
    ti = _cuda(idx, torch.int32)
    # forward on sampled virtual sources
    U = plan.forward(Xg, ti).cpu().numpy()
    vs = np.array([0, 1, 77, 150, 200])
    _check(U[:, vs], oracle.mdc_forward(D, X, idx, vsel=vs), "U sampled")
    # adjoint on sampled virtual sources
    R = _f32(synth.random_traces((nb, n, nt), 10))
    G = plan.adjoint(_cuda(R), ti).cpu().numpy()
    _check(G[vs], oracle.mdc_adjoint(D, R, idx, vsel=vs), "G sampled")
    # fused step with reciprocity: sampled (v, r) pairs need G[v, r] and G[r, v]
    alpha = 1e-5
    loss = torch.zeros((), device="cuda", dtype=torch.float64)
    plan.step(Xg, _cuda(U_obs), ti, alpha, binding.SMDD_RECIPROCITY, loss)
    assert plan.sync_status() == binding.MDC_OK
    Xn = Xg.double().cpu().numpy()
    np.testing.assert_array_equal(Xn.astype(np.float32), Xn.astype(np.float32).transpose(1, 0, 2))
    cols = np.array([3, 100, 199])
    # G[:, v] depends on the residual of column v only, so the sampled columns need only their residuals
    Rsub = oracle.mdc_forward(D, X, idx, vsel=cols) - U_obs[idx][:, cols]
    Gc = oracle.mdc_adjoint(D, Rsub, idx, vsel=np.arange(len(cols)))   # (3, nr, nt): G[v=cols]
    for a_, va in enumerate(cols):
        for b_, vb in enumerate(cols):
            g_sym = 0.5 * (Gc[a_, vb] + Gc[b_, va])               # 1/2 (G[va, vb] + G[vb, va])
            got = (X[va, vb] - Xn[va, vb]) / alpha
            err = np.max(np.abs(got - g_sym)) / np.max(np.abs(Gc))
            assert err <= 2e-4, (va, vb, err)
    l_ref = oracle.loss(oracle.mdc_forward_fft(D, X, idx) - U_obs[idx])   # FFT tier, pinned to the direct sums
    assert abs(loss.item() - l_ref) <= 1e-5 * l_ref


def test_device_index_error_reported():
    nt, nr, nv, ns = 32, 4, 4, 5
    D, X, _, _ = _problem(nt, nr, nv, ns, 2, seed=41)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=4)
    bad = _cuda(np.array([1, 7], np.int32), torch.int32)
    plan.forward(_cuda(X), bad)
    assert plan.sync_status() == binding.MDC_ERR_INDEX_RANGE
    assert plan.sync_status() == binding.MDC_OK     # cleared
    plan.forward(_cuda(X), _cuda(np.array([1, 4], np.int32), torch.int32))
    assert plan.sync_status() == binding.MDC_OK


def test_host_errors():
    nt, nr, nv, ns = 32, 4, 3, 5
    D, X, _, _ = _problem(nt, nr, nv, ns, 2, seed=42)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=2)
    idx3 = _cuda(np.array([0, 1, 2], np.int32), torch.int32)
    with pytest.raises(binding.MDCError) as e:
        plan.forward(_cuda(X), idx3)
    assert e.value.status == binding.MDC_ERR_SHAPE
    with pytest.raises(binding.MDCError) as e:
        plan.step(_cuda(X), _cuda(np.zeros((ns, nv, nt))), idx3[:2], 1e-3, binding.SMDD_RECIPROCITY)
    assert e.value.status == binding.MDC_ERR_SHAPE
    with pytest.raises(binding.MDCError) as e:
        binding.MDCPlan(_cuda(np.zeros((2, 2, 5000))), 2)
    assert e.value.status == binding.MDC_ERR_UNSUPPORTED


def test_stage_timing_and_launch_counts():
    nt, nr, nv, ns, nb = 128, 32, 32, 32, 8
    D, X, _, idx = _problem(nt, nr, nv, ns, nb, seed=51)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    binding.mdc_plan_set_profiling(plan.handle, True)
    binding.mdc_plan_stage_times(plan.handle, reset=True)
    n0 = binding.mdc_plan_launch_count(plan.handle)
    Xg, Ug, ti = _cuda(X), _cuda(np.zeros((ns, nv, nt))), _cuda(idx, torch.int32)
    for k in range(3):
        plan.step(Xg, Ug, ti, 1e-4, binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0))
    t = binding.mdc_plan_stage_times(plan.handle, reset=True)
    assert binding.mdc_plan_launch_count(plan.handle) - n0 == 1 + 4 * 3
    assert t["rfft"][1] == 1 and t["cgemm_fwd"][1] == 3 and t["update"][1] == 3
    assert all(t[s][0] > 0 for s in ("rfft", "cgemm_fwd", "residual", "cgemm_adj", "update"))

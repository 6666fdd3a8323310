"""GPU parity of the Adam update fused into the update kernel (smdd_step_ex with SMDD_ADAM) against the FP64
oracle's adam_step (Kingma & Ba 2015, Algorithm 1, on the preconditioned batch gradient of Eq. 6).

Tolerance, from the arithmetic.  The FP32 gradient carries a relative error of at most 1e-5 (the bar of
the single-step parity tests; elementwise 2e-5 of max|g|).  One Adam step is x - alpha * m_hat /
(sqrt(v_hat) + eps), whose derivative with respect to g is at most alpha / eps per element, while the step
itself is at least alpha |g| / (max|g| + eps).  With eps = c max|g| the relative error of a step is
therefore at most 1e-5 (1 + c) / c, and of X after n steps from zero at most n times that.  The tests use
c = 1 (2e-5 per step).  With a small eps (1e-8, Kingma & Ba's default) Adam divides by |g| itself, so where
|g| lies near its own rounding error the sign of the step is decided by rounding: there the parity is
checked only on the elements whose gradient is far above that floor.
"""
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


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _check(gpu, ref, what, rel, elem):
    gpu = np.asarray(gpu, dtype=np.float64)
    r = oracle.rel_l2(gpu, ref)
    m = np.max(np.abs(gpu - ref)) / max(np.max(np.abs(ref)), 1e-30)
    assert r <= rel, f"{what}: relative L2 {r:.3e} > {rel:.1e}"
    assert m <= elem, f"{what}: max elementwise error {m:.3e} of max|ref| > {elem:.1e}"


def _problem(shape, seed):
    nt, nr, nv, ns, nb = shape
    p = synth.make_problem(nt, nr, nv, ns, dx=60.0, n_reflectors=3, n_multiples=2, seed=seed)
    D = _f32(p.D)
    U_obs = _f32(oracle.mdc_forward(D, _f32(p.X_true), np.arange(ns)))
    return D, U_obs


@pytest.mark.parametrize("shape,recip,use_mute", [
    ((128, 24, 24, 30, 8), True, True),
    ((257, 17, 19, 23, 7), False, True),
    ((100, 12, 12, 15, 5), True, False),
    ((130, 10, 13, 9, 3), False, False),      # nt = 2 mod 4: scalar time I/O for X, m and v
    ((1024, 16, 16, 20, 4), False, False),    # nfft 2048 (the plan's default there is the two-pass FFT)
], ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_adam_steps_match_oracle(shape, recip, use_mute):
    nt, nr, nv, ns, nb = shape
    seed = sum(shape)
    D, U_obs = _problem(shape, seed)
    mute = synth.direct_arrival_mute(nr, nv, nt, dx=60.0) if use_mute else None
    if use_mute:
        assert (mute > 0).any()
    idxs = [synth.random_indices(ns, nb, seed + k) for k in range(3)]
    g0, _, _ = oracle.gradient(D, np.zeros((nv, nr, nt)), U_obs, idxs[0])
    g0 = oracle.precondition(g0, recip=recip, mute=mute)
    eps = float(np.abs(g0).max())                 # c = 1
    alpha, b1, b2 = 1e-3, 0.9, 0.999
    X, M, V = np.zeros((nv, nr, nt)), np.zeros((nv, nr, nt)), np.zeros((nv, nr, nt))
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    Xg, Mg, Vg, Ug = _cuda(X), _cuda(M), _cuda(V), _cuda(U_obs)
    mg = None if mute is None else _cuda(mute, torch.int32)
    losses = torch.zeros(3, device="cuda", dtype=torch.float64)
    l_ref = []
    for k, idx in enumerate(idxs):
        fl = (binding.SMDD_RECIPROCITY if recip else 0) | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
        plan.step_adam(Xg, Mg, Vg, Ug, _cuda(idx, torch.int32), alpha, k + 1, beta1=b1, beta2=b2, eps=eps, flags=fl,
                       mute=mg, loss=losses[k])
        X, M, V, l = oracle.adam_step(D, X, M, V, U_obs, idx, alpha, k + 1, beta1=b1, beta2=b2, eps=eps,
                                      recip=recip, mute=mute)
        l_ref.append(l)
    assert plan.sync_status() == binding.MDC_OK
    n = len(idxs)
    _check(Xg.cpu().numpy(), X, "X", rel=n * 2e-5, elem=n * 4e-5)
    _check(Mg.cpu().numpy(), M, "m", rel=1e-5, elem=2e-5)
    _check(Vg.cpu().numpy(), V, "v", rel=2e-5, elem=4e-5)
    np.testing.assert_allclose(losses.cpu().numpy(), l_ref, rtol=1e-5)
    Xc = Xg.cpu().numpy()
    if use_mute:
        muted = np.arange(nt)[None, None, :] < mute[:, :, None]
        assert np.all(Xc[muted] == 0.0) and np.all(Mg.cpu().numpy()[muted] == 0.0)
    if recip:
        assert np.array_equal(Xc, Xc.transpose(1, 0, 2))


def test_adam_default_eps_on_well_conditioned_elements():
    """eps = 1e-8: two steps.  With eps << sqrt(v_hat) a step is alpha m_hat / sqrt(v_hat), and a gradient
    error |dg| <= d (d = 2e-5 max|g|, the FP32 bar) moves it by at most alpha (d / sqrt(v_hat) +
    |m_hat| |dv_hat| / (2 v_hat^1.5)) <= alpha (d / max|g|) (1 / c + 1.0013 / c^2) where every gradient of
    the element is at least c max|g| (|m_hat| <= 1.0013 sqrt(v_hat) for beta1 = 0.9, beta2 = 0.999 at
    t <= 2, by Cauchy-Schwarz on the bias-corrected weights).  With c = 0.1 that is 2.2e-3 alpha per
    step; elsewhere the sign of the step can be decided by rounding and is not compared.  Every element
    moved by at most 1.0013 alpha per step."""
    shape = (256, 20, 20, 24, 6)
    nt, nr, nv, ns, nb = shape
    D, U_obs = _problem(shape, 5)
    alpha = 2e-3
    X, M, V = np.zeros((nv, nr, nt)), np.zeros((nv, nr, nt)), np.zeros((nv, nr, nt))
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    Xg, Mg, Vg, Ug = _cuda(X), _cuda(M), _cuda(V), _cuda(U_obs)
    good = np.ones(X.shape, bool)
    for k in range(2):
        idx = synth.random_indices(ns, nb, 50 + k)
        g, _, _ = oracle.gradient(D, X, U_obs, idx)
        good &= np.abs(g) >= 0.1 * np.abs(g).max()
        plan.step_adam(Xg, Mg, Vg, Ug, _cuda(idx, torch.int32), alpha, k + 1)
        X, M, V, _ = oracle.adam_step(D, X, M, V, U_obs, idx, alpha, k + 1)
    assert plan.sync_status() == binding.MDC_OK
    Xc = Xg.double().cpu().numpy()
    assert good.mean() > 0.05
    assert np.max(np.abs(Xc - X)[good]) <= 2 * 2e-5 * (1 / 0.1 + 1.0013 / 0.1 ** 2) * alpha
    assert np.max(np.abs(Xc)) <= 2 * 1.0013 * alpha * (1 + 1e-6)


def test_adam_argument_errors():
    nt, n, ns, nb = 64, 6, 8, 2
    plan = binding.MDCPlan(_cuda(synth.random_traces((ns, n, nt), 1)), n, nb_max=nb)
    X, U = torch.zeros((n, n, nt), device="cuda"), torch.zeros((ns, n, nt), device="cuda")
    M, V = torch.zeros_like(X), torch.zeros_like(X)
    idx = torch.zeros(nb, dtype=torch.int32, device="cuda")
    bad = [
        dict(flags=binding.SMDD_ADAM, V=M, S=None, t=1),                              # no second moment
        dict(flags=binding.SMDD_ADAM, V=M, S=V, t=0),                                 # step count from 1
        dict(flags=binding.SMDD_ADAM, V=M, S=M, t=1),                                 # m and v the same array
        dict(flags=binding.SMDD_ADAM | binding.SMDD_NESTEROV, V=M, S=V, t=1, mu=0.5),  # two solvers
        dict(flags=binding.SMDD_ADAM, V=M, S=V, t=1, beta1=1.0),                      # beta outside [0, 1)
        dict(flags=binding.SMDD_ADAM, V=M, S=V, t=1, eps=0.0),                        # eps > 0
        dict(flags=0, V=None, S=V, t=0),                                              # moment without Adam
    ]
    for kw in bad:
        with pytest.raises(binding.MDCError) as e:
            binding.smdd_step_ex(plan.handle, X, U, idx, 1e-3, **kw)
        assert e.value.status == binding.MDC_ERR_INVALID_ARG, kw
    assert plan.sync_status() == binding.MDC_OK

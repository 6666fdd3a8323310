"""GPU parity of the N-SGD step (Nesterov momentum on the look-ahead point) and of the causality mute
(smdd_step_ex) against the FP64 oracle's nsgd_step / causal_mute.

Bar: the FP32 one of the single-step tests (relative L2 <= 1e-5, elementwise <= 2e-5 of max|ref|) on X
and V after a few steps; 1e-4 relative L2 on a 30-epoch trajectory (rounding compounds over steps, as
in the SGD trajectory test).
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


def _check(gpu, ref, what, rel=1e-5, elem=2e-5):
    gpu = np.asarray(gpu, dtype=np.float64)
    r = oracle.rel_l2(gpu, ref)
    m = np.max(np.abs(gpu - ref)) / max(np.max(np.abs(ref)), 1e-30)
    assert r <= rel, f"{what}: relative L2 {r:.3e} > {rel:.1e}"
    assert m <= elem, f"{what}: max elementwise error {m:.3e} of max|ref| > {elem:.1e}"


@pytest.mark.parametrize("shape,recip,use_mute,nesterov", [
    ((128, 24, 24, 30, 8), True, True, True),
    ((257, 17, 19, 23, 7), False, True, True),
    ((100, 12, 12, 15, 5), True, False, True),
    ((600, 9, 9, 11, 4), False, True, False),
    ((130, 10, 13, 9, 3), False, False, True),     # nt = 2 mod 4: scalar time I/O for X and V
], ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_nsgd_steps_match_oracle(shape, recip, use_mute, nesterov):
    nt, nr, nv, ns, nb = shape
    seed = sum(shape)
    p = synth.make_problem(nt, nr, nv, ns, dx=60.0, n_reflectors=3, n_multiples=2, seed=seed)
    D = _f32(p.D)
    U_obs = _f32(oracle.mdc_forward(D, _f32(p.X_true), np.arange(ns)))
    mute = synth.direct_arrival_mute(nr, nv, nt, dx=60.0) if use_mute else None
    if use_mute:
        assert (mute > 0).any()
    X = np.zeros((nv, nr, nt))
    V = np.zeros_like(X)
    alpha, mu = 0.4 / oracle.sigma2_max(D), 0.9
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    Xg, Vg, Ug = _cuda(X), _cuda(V), _cuda(U_obs)
    mg = None if mute is None else _cuda(mute, torch.int32)
    losses = torch.zeros(3, device="cuda", dtype=torch.float64)
    l_ref = []
    for k in range(3):
        idx = synth.random_indices(ns, nb, seed + k)
        fl = (binding.SMDD_RECIPROCITY if recip else 0) | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
        if nesterov:
            binding.smdd_step_ex(plan.handle, Xg, Ug, _cuda(idx, torch.int32), alpha, fl | binding.SMDD_NESTEROV,
                                 V=Vg, mu=mu, mute=mg, loss=losses[k])
            X, V, l = oracle.nsgd_step(D, X, V, U_obs, idx, alpha, mu, recip=recip, mute=mute)
        else:
            binding.smdd_step_ex(plan.handle, Xg, Ug, _cuda(idx, torch.int32), alpha, fl, mute=mg, loss=losses[k])
            g, l, _ = oracle.gradient(D, X, U_obs, idx)
            X = X - alpha * oracle.precondition(g, recip=recip, mute=mute)
        l_ref.append(l)
    assert plan.sync_status() == binding.MDC_OK
    _check(Xg.cpu().numpy(), X, "X")
    if nesterov:
        _check(Vg.cpu().numpy(), V, "V")
    np.testing.assert_allclose(losses.cpu().numpy(), l_ref, rtol=1e-5)
    if use_mute:
        t = np.arange(nt)
        muted = t[None, None, :] < mute[:, :, None]
        assert np.all(Xg.cpu().numpy()[muted] == 0.0)


def test_zero_momentum_equals_sgd_step():
    nt, n, ns, nb = 128, 20, 24, 6
    D = _cuda(synth.random_traces((ns, n, nt), 1))
    U = _cuda(synth.random_traces((ns, n, nt), 2))
    X0 = _cuda(synth.random_traces((n, n, nt), 3))
    idx = _cuda(synth.random_indices(ns, nb, 4), torch.int32)
    plan = binding.MDCPlan(D, n, nb_max=nb)
    Xa, Xb, V = X0.clone(), X0.clone(), torch.zeros_like(X0)
    binding.smdd_step(plan.handle, Xa, U, idx, 1e-4, binding.SMDD_RECIPROCITY)
    binding.smdd_step_ex(plan.handle, Xb, U, idx, 1e-4, binding.SMDD_RECIPROCITY | binding.SMDD_NESTEROV, V=V, mu=0.0)
    assert plan.sync_status() == binding.MDC_OK
    torch.testing.assert_close(Xb, Xa, rtol=0, atol=1e-7 * X0.abs().max().item())
    torch.testing.assert_close(Xb - X0, V, rtol=1e-5, atol=1e-6 * V.abs().max().item())


def test_nsgd_trajectory_small_workload():
    """30 epochs of N-SGD (mu 0.9) with batches of 8 on the nt=128, 32^3 workload against the oracle's
    trajectory from the same batches; N-SGD reaches a lower loss than SGD with the same step size."""
    w = synth.WORKLOADS["smdd_nt128_n32_nb8"]
    p = synth.make_problem(w["nt"], 32, 32, 32, dx=w["dx"], n_reflectors=w["n_reflectors"],
                           n_multiples=w["n_multiples"], seed=0)
    D = _f32(p.D)
    U_obs = _f32(oracle.mdc_forward(D, _f32(p.X_true), np.arange(32)))
    batches = synth.epoch_batches(32, w["nb"], 30, seed=0)
    alpha, mu = 0.25 * 2.0 / oracle.sigma2_max(D), 0.9
    X, V = np.zeros((32, 32, w["nt"])), np.zeros((32, 32, w["nt"]))
    l_ref = []
    for ep in batches:
        for idx in ep:
            X, V, l = oracle.nsgd_step(D, X, V, U_obs, idx, alpha, mu, fft=True)
            l_ref.append(l)
    plan = binding.MDCPlan(_cuda(D), 32, nb_max=w["nb"])
    Xg, Vg, Ug = torch.zeros((32, 32, w["nt"]), device="cuda"), torch.zeros((32, 32, w["nt"]), device="cuda"), _cuda(U_obs)
    Xs = torch.zeros_like(Xg)
    losses = torch.zeros(len(l_ref), device="cuda", dtype=torch.float64)
    ls = torch.zeros(len(l_ref), device="cuda", dtype=torch.float64)
    plan_s = binding.MDCPlan(_cuda(D), 32, nb_max=w["nb"])
    k = 0
    for ep in batches:
        for idx in ep:
            ii = _cuda(idx, torch.int32)
            fl = binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
            binding.smdd_step_ex(plan.handle, Xg, Ug, ii, alpha, fl | binding.SMDD_NESTEROV, V=Vg, mu=mu, loss=losses[k])
            binding.smdd_step(plan_s.handle, Xs, Ug, ii, alpha, fl, ls[k])
            k += 1
    assert plan.sync_status() == binding.MDC_OK
    assert oracle.rel_l2(Xg.double().cpu().numpy(), X) <= 1e-4
    assert oracle.rel_l2(losses.cpu().numpy(), np.array(l_ref)) <= 1e-4
    n_ep = len(batches[0])
    assert losses[-n_ep:].sum().item() < ls[-n_ep:].sum().item()


def test_step_ex_host_errors():
    D = _cuda(synth.random_traces((5, 4, 16), 1))
    plan = binding.MDCPlan(D, 4, nb_max=2)
    X = torch.zeros((4, 4, 16), device="cuda")
    V = torch.zeros_like(X)
    U = torch.zeros((5, 4, 16), device="cuda")
    idx = torch.tensor([0, 1], device="cuda", dtype=torch.int32)
    cases = [
        dict(flags=binding.SMDD_NESTEROV, V=None, mu=0.5),          # momentum without a velocity
        dict(flags=0, V=V, mu=0.5),                                  # a velocity without the flag
        dict(flags=binding.SMDD_NESTEROV, V=V, mu=1.0),              # mu out of range
        dict(flags=binding.SMDD_NESTEROV, V=X, mu=0.5),              # V aliases X
        dict(flags=128, V=None, mu=0.0),                             # unknown flag
    ]
    for c in cases:
        with pytest.raises(binding.MDCError) as e:
            binding.smdd_step_ex(plan.handle, X, U, idx, 0.1, c["flags"], V=c["V"], mu=c["mu"])
        assert e.value.status == binding.MDC_ERR_INVALID_ARG, c
    D2 = _cuda(synth.random_traces((5, 4, 16), 2))
    p2 = binding.MDCPlan(D2, 3, nb_max=2)
    with pytest.raises(binding.MDCError) as e:
        binding.smdd_step_ex(p2.handle, torch.zeros((3, 4, 16), device="cuda"), torch.zeros((5, 3, 16), device="cuda"),
                             idx, 0.1, binding.SMDD_RECIPROCITY)
    assert e.value.status == binding.MDC_ERR_SHAPE


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_nsgd_and_mute_under_every_fft_variant(variant):
    """The momentum / mute update runs the default radix order whatever FFT variant the plan holds; the
    other kernels of the step run the plan's variant.  Both must agree on the trace tiling."""
    nt, n, ns, nb = 257, 12, 15, 5        # nfft 1024: all three variants exist
    p = synth.make_problem(nt, n, n, ns, dx=60.0, n_reflectors=3, n_multiples=2, seed=77)
    D = _f32(p.D)
    U_obs = _f32(oracle.mdc_forward(D, _f32(p.X_true), np.arange(ns)))
    mute = synth.direct_arrival_mute(n, n, nt, dx=60.0)
    alpha, mu = 0.4 / oracle.sigma2_max(D), 0.9
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb)
    plan.set_config(fft_variant=variant)
    X, V = np.zeros((n, n, nt)), np.zeros((n, n, nt))
    Xg, Vg = _cuda(X), _cuda(V)
    for k in range(2):
        idx = synth.random_indices(ns, nb, 80 + k)
        fl = binding.SMDD_RECIPROCITY | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
        binding.smdd_step_ex(plan.handle, Xg, _cuda(U_obs), _cuda(idx, torch.int32), alpha, fl | binding.SMDD_NESTEROV,
                             V=Vg, mu=mu, mute=_cuda(mute, torch.int32))
        X, V, _ = oracle.nsgd_step(D, X, V, U_obs, idx, alpha, mu, recip=True, mute=mute)
    assert plan.sync_status() == binding.MDC_OK
    _check(Xg.cpu().numpy(), X, f"X (variant {variant})")
    _check(Vg.cpu().numpy(), V, f"V (variant {variant})")

"""GPU parity of the kernel configurations (FFT radix order, product kernels), the autotuner, and the
batched, graph-captured epochs of many independent problems.

Every configuration computes the same operator, so each is held to the FP32 bar of the single-plan
tests against the FP64 oracle (relative L2 <= 1e-5, elementwise <= 2e-5 of max|ref|).  The batched
epochs replay exactly the kernels that separate smdd_step calls launch, in the same order per member,
so each member's model and losses must equal those of the separate calls bit for bit; they are also
held against the oracle's SGD trajectory from the same permutations.
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


# every FFT length where the reversed radix order (variant 1) differs from the default (M = 32, 128,
# 256, 1024, 1536, 2048) or the two-pass FFT (variant 2) exists (M = 128 .. 1024), ragged sizes, odd nt
# and nt = 2 mod 4 (scalar time I/O)
VARIANT_SHAPES = [
    (30, 7, 5, 9, 4),         # nfft 64
    (100, 37, 29, 41, 5),     # nfft 256
    (200, 12, 10, 14, 6),     # nfft 512
    (257, 17, 19, 23, 17),    # nfft 1024, odd nt
    (600, 20, 20, 20, 4),     # nfft 2048
    (1500, 6, 5, 7, 3),       # nfft 3072 (radix 8 * 8 * 3 * 8, reversed 8 * 3 * 8 * 8)
    (1025, 9, 7, 8, 5),       # nfft 3072, odd nt
    (1800, 6, 5, 7, 3),       # nfft 4096
    (130, 9, 9, 12, 7),       # nfft 512, scalar time I/O
    (1024, 33, 35, 40, 9),    # nfft 2048, nt = M: no zero padding inside the first half
]


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("shape", [
    (1500, 48, 44, 20, 4),    # nfft 3072: 264 tiles of 8 traces, more than one per persistent CTA
    (600, 64, 70, 20, 4),     # nfft 2048: 1120 tiles of 4 traces
    (1023, 40, 41, 12, 3),    # nfft 2048, odd nt, a ragged last tile
], ids=lambda s: "x".join(map(str, s)))
def test_prefetch_update_walks_many_tiles(shape, order):
    """The persistent prefetching update when every CTA walks several tiles (the double buffer
    alternates): two fused steps against the oracle's SGD steps."""
    nt, nr, nv, ns, nb = shape
    seed = sum(shape) + order
    D = _f32(synth.random_traces((ns, nr, nt), seed))
    X = _f32(synth.random_traces((nv, nr, nt), seed + 1))
    U_obs = _f32(synth.random_traces((ns, nv, nt), seed + 2))
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    plan.set_config(fft_variant=order, fft_prefetch=1)
    assert plan.get_config()["fft_prefetch"] == 1
    alpha = 0.3 / oracle.sigma2_max(D)
    Xg, Ug, Xr = _cuda(X), _cuda(U_obs), X.copy()
    for k in range(2):
        ii = synth.random_indices(ns, nb, seed + 3 + k)
        fl = binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
        binding.smdd_step(plan.handle, Xg, Ug, _cuda(ii, torch.int32), alpha, fl)
        Xr, _ = oracle.sgd_step(D, Xr, U_obs, ii, alpha)
    assert plan.sync_status() == binding.MDC_OK
    _check(Xg.cpu().numpy(), Xr, f"X after two steps {shape}")


@pytest.mark.parametrize("variant", [1, 2, "prefetch0", "prefetch1"])
@pytest.mark.parametrize("shape", VARIANT_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_fft_variants_match_oracle(shape, variant):
    nt, nr, nv, ns, nb = shape
    seed = sum(shape)
    D = _f32(synth.random_traces((ns, nr, nt), seed))
    X = _f32(synth.random_traces((nv, nr, nt), seed + 1))
    R = _f32(synth.random_traces((nb, nv, nt), seed + 2))
    idx = synth.random_indices(ns, nb, seed + 3)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, scale=0.5)
    M = plan.nfft // 2
    if isinstance(variant, str):   # the persistent prefetching update with radix order 0 or 1
        order = int(variant[-1])
        plan.set_config(fft_variant=order, fft_prefetch=1)
        assert plan.get_config()["fft_prefetch"] == (1 if M <= 1536 else 0)
    else:
        plan.set_config(fft_variant=variant)
        # variant 1 falls back to 0 where both radix orders coincide; variant 2 exists for 128 <= M <= 1024
        # (two passes) and M = 1536 (three passes)
        expected = {0, 1} if variant == 1 else ({2} if 128 <= M <= 1024 or M == 1536 else {0})
        assert plan.get_config()["fft_variant"] in expected
    ti = _cuda(idx, torch.int32)
    _check(plan.forward(_cuda(X), ti).cpu().numpy(), oracle.mdc_forward(D, X, idx, 0.5), f"U {shape}")
    _check(plan.adjoint(_cuda(R), ti).cpu().numpy(), oracle.mdc_adjoint(D, R, idx, 0.5), f"G {shape}")
    # the fused step (model transform kept for the next step) with this variant, twice
    U_obs = _f32(synth.random_traces((ns, nv, nt), seed + 4))
    alpha = 0.3 / oracle.sigma2_max(D, scale=0.5)
    Xg, Ug = _cuda(X), _cuda(U_obs)
    Xr = X.copy()
    idx2 = synth.random_indices(ns, nb, seed + 5)
    for k, ii in enumerate((idx, idx2)):
        fl = binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
        binding.smdd_step(plan.handle, Xg, Ug, _cuda(ii, torch.int32), alpha, fl)
        Xr, _ = oracle.sgd_step(D, Xr, U_obs, ii, alpha, scale=0.5)
    assert plan.sync_status() == binding.MDC_OK
    _check(Xg.cpu().numpy(), Xr, f"X after two steps {shape}")


@pytest.mark.parametrize("adj", [binding.MDC_GEMM_SIMT32, binding.MDC_GEMM_SIMT64])
@pytest.mark.parametrize("recip", [False, True])
def test_adjoint_tiles_match_oracle(adj, recip):
    nt, n, ns, nb = 64, 70, 80, 20
    D = _f32(synth.random_traces((ns, n, nt), 31))
    X = _f32(synth.random_traces((n, n, nt), 32))
    U_obs = _f32(synth.random_traces((ns, n, nt), 33))
    idx = synth.random_indices(ns, nb, 34)
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb)
    plan.set_config(gemm_adj=adj)
    R = _f32(synth.random_traces((nb, n, nt), 35))
    _check(plan.adjoint(_cuda(R), _cuda(idx, torch.int32)).cpu().numpy(), oracle.mdc_adjoint(D, R, idx), "G")
    alpha = 0.3 / oracle.sigma2_max(D)
    Xg = _cuda(X)
    binding.smdd_step(plan.handle, Xg, _cuda(U_obs), _cuda(idx, torch.int32), alpha,
                      binding.SMDD_RECIPROCITY if recip else 0)
    Xr, _ = oracle.sgd_step(D, X, U_obs, idx, alpha, recip=recip)
    assert plan.sync_status() == binding.MDC_OK
    _check(Xg.cpu().numpy(), Xr, "X")


@pytest.mark.parametrize("fwd,adj", [(binding.MDC_GEMM_SIMT, binding.MDC_GEMM_TC),
                                     (binding.MDC_GEMM_TC, binding.MDC_GEMM_SIMT)])
def test_mixed_kernels_on_split_bf16_plan(fwd, adj):
    """A BF16X3 plan may run the FP32 kernels for either product; both combinations stay inside the
    split-BF16 bound (1e-4) and the FP32 product inside the FP32 bound."""
    nt, n, ns, nb = 128, 150, 160, 24
    D = _f32(synth.random_traces((ns, n, nt), 41))
    X = _f32(synth.random_traces((n, n, nt), 42))
    R = _f32(synth.random_traces((nb, n, nt), 43))
    idx = synth.random_indices(ns, nb, 44)
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb, precision=binding.MDC_PREC_BF16X3)
    plan.set_config(gemm_fwd=fwd, gemm_adj=adj)
    ti = _cuda(idx, torch.int32)
    U = plan.forward(_cuda(X), ti).cpu().numpy()
    G = plan.adjoint(_cuda(R), ti).cpu().numpy()
    assert plan.sync_status() == binding.MDC_OK
    bu = REL_L2 if fwd == binding.MDC_GEMM_SIMT else 1e-4
    bg = REL_L2 if adj == binding.MDC_GEMM_SIMT else 1e-4
    _check(U, oracle.mdc_forward(D, X, idx), "U", rel=bu, elem=20 * bu)
    _check(G, oracle.mdc_adjoint(D, R, idx), "G", rel=bg, elem=20 * bg)


def test_config_errors():
    D = _cuda(synth.random_traces((4, 3, 16), 1))
    plan = binding.MDCPlan(D, 3, nb_max=2)
    cfg = plan.get_config()
    assert cfg == {"fft_variant": 0, "gemm_fwd": binding.MDC_GEMM_SIMT, "gemm_adj": binding.MDC_GEMM_SIMT,
                   "fft_prefetch": 0}
    with pytest.raises(binding.MDCError) as e:
        plan.set_config(gemm_fwd=binding.MDC_GEMM_TC)
    assert e.value.status == binding.MDC_ERR_UNSUPPORTED
    with pytest.raises(binding.MDCError) as e:
        plan.set_config(fft_variant=3)
    assert e.value.status == binding.MDC_ERR_INVALID_ARG
    with pytest.raises(binding.MDCError) as e:
        plan.set_config(gemm_adj=7)
    assert e.value.status == binding.MDC_ERR_INVALID_ARG
    with pytest.raises(binding.MDCError) as e:
        plan.autotune(nb=3)
    assert e.value.status == binding.MDC_ERR_SHAPE
    assert plan.get_config() == cfg
    b16 = binding.MDCPlan(D, 3, nb_max=2, precision=binding.MDC_PREC_BF16X3)
    assert b16.get_config() == {"fft_variant": 0, "gemm_fwd": binding.MDC_GEMM_TC, "gemm_adj": binding.MDC_GEMM_TC,
                                "fft_prefetch": 0}


@pytest.mark.parametrize("precision", [binding.MDC_PREC_FP32, binding.MDC_PREC_BF16X3])
def test_autotune_keeps_parity(precision):
    nt, n, ns, nb = 600, 40, 48, 16
    D = _f32(synth.random_traces((ns, n, nt), 51))
    X = _f32(synth.random_traces((n, n, nt), 52))
    U_obs = _f32(synth.random_traces((ns, n, nt), 53))
    idx = synth.random_indices(ns, nb, 54)
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb, precision=precision)
    best = plan.autotune(nb, binding.SMDD_RECIPROCITY, reps=3)
    assert best == plan.get_config()
    assert best["fft_variant"] in (0, 1, 2) and best["fft_prefetch"] in (0, 1)
    if precision == binding.MDC_PREC_FP32:
        assert best["gemm_fwd"] == binding.MDC_GEMM_SIMT and best["gemm_adj"] in (1, 2)
    alpha = 0.3 / oracle.sigma2_max(D)
    Xg = _cuda(X)
    binding.smdd_step(plan.handle, Xg, _cuda(U_obs), _cuda(idx, torch.int32), alpha, binding.SMDD_RECIPROCITY)
    Xr, _ = oracle.sgd_step(D, X, U_obs, idx, alpha, recip=True)
    assert plan.sync_status() == binding.MDC_OK
    tol = REL_L2 if precision == binding.MDC_PREC_FP32 else 1e-4
    _check(Xg.cpu().numpy(), Xr, "X after the autotuned step", rel=tol, elem=20 * tol)


# ------------------------------------------------------------------------------------------------
# batched epochs under one graph
# ------------------------------------------------------------------------------------------------
MEMBERS = [   # (nt, nr, nv, ns, nb, reciprocity)
    (128, 32, 32, 32, 8, False),
    (100, 19, 23, 41, 6, False),
    (257, 12, 12, 15, 4, True),
    (40, 50, 9, 70, 32, False),
    (600, 6, 7, 9, 9, False),
]


def _member_data(k, shape, n_perm):
    nt, nr, nv, ns, nb, recip = shape
    p = synth.make_problem(nt, nr, nv, ns, dx=15.0, n_reflectors=3, n_multiples=2, seed=100 + k)
    D = _f32(p.D)
    U_obs = _f32(oracle.mdc_forward(D, _f32(p.X_true), np.arange(ns)))
    batches = synth.epoch_batches(ns, nb, n_perm, seed=100 + k)
    perm = np.stack([np.concatenate(ep) for ep in batches]).astype(np.int32)
    alpha = 0.5 * 2.0 / oracle.sigma2_max(D)
    X0 = np.zeros((nv, nr, nt))
    if recip:
        X0 = _f32(0.1 * oracle.reciprocity(synth.random_traces((nv, nr, nt), 7 + k)))
    return D, U_obs, perm, alpha, X0


def test_batched_epochs_equal_separate_steps_and_oracle():
    n_epochs, n_perm, loss_rows = 3, 2, 3   # rows of the permutation table are re-used: epoch e -> e % 2
    data, members, refs = [], [], []
    for k, shape in enumerate(MEMBERS):
        nt, nr, nv, ns, nb, recip = shape
        D, U_obs, perm, alpha, X0 = _member_data(k, shape, n_perm)
        plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
        steps = oracle.steps_per_epoch(ns, nb)
        # the reciprocity member starts symmetric: its update runs on the upper triangle (SMDD_SYMMETRIC)
        m = dict(plan=plan, X=_cuda(X0), U_obs=_cuda(U_obs), perm=_cuda(perm, torch.int32), nb=nb, alpha=alpha,
                 flags=(binding.SMDD_RECIPROCITY | binding.SMDD_SYMMETRIC) if recip else 0,
                 loss=torch.full((loss_rows, steps), -1.0, device="cuda", dtype=torch.float64))
        members.append(m)
        data.append((D, U_obs, perm, alpha, X0, recip, steps))
    batch = binding.MDCBatch(members, n_branches=3)
    assert batch.n_branches == 3
    # kernels per epoch: begin + end, plus per member 5 launches in its first step and 4 in the others, and
    # for the symmetric member the copy of the spectra below the block diagonal after every update
    n_sym = sum(s for s, shape in zip(batch.steps, MEMBERS) if shape[5])
    assert batch.kernels_per_epoch == 2 + sum(4 * s + 1 for s in batch.steps) + n_sym
    batch.run(0, 2)
    batch.run(2, 1)
    torch.cuda.synchronize()

    for k, (m, (D, U_obs, perm, alpha, X0, recip, steps)) in enumerate(zip(members, data)):
        assert m["plan"].sync_status() == binding.MDC_OK
        nt, nr, nv, ns, nb, _ = MEMBERS[k]
        # the same steps issued one by one
        plan2 = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
        Xs, Us = _cuda(X0), _cuda(U_obs)
        ls = torch.zeros((n_epochs, steps), device="cuda", dtype=torch.float64)
        for e in range(n_epochs):
            row = perm[e % n_perm]
            for s in range(steps):
                fl = m["flags"] | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if s else 0)
                binding.smdd_step(plan2.handle, Xs, Us, _cuda(row[s * nb:(s + 1) * nb], torch.int32), alpha, fl,
                                  ls[e, s])
        assert torch.equal(m["X"], Xs), f"member {k}: batched model differs from separate steps"
        assert torch.equal(m["loss"], ls), f"member {k}: batched losses differ from separate steps"
        # the oracle's trajectory from the same permutations
        batches = [[perm[e % n_perm][s * nb:(s + 1) * nb] for s in range(steps)] for e in range(n_epochs)]
        X_ref, l_ref = oracle.run_epochs(D, X0, U_obs, batches, alpha, recip=recip, fft=True)
        assert oracle.rel_l2(m["X"].double().cpu().numpy(), X_ref) <= 1e-4, f"member {k}"
        assert oracle.rel_l2(m["loss"].cpu().numpy().ravel(), np.array(l_ref)) <= 1e-4, f"member {k}"
    batch.close()


@pytest.mark.parametrize("fwd", [binding.MDC_GEMM_TC, binding.MDC_GEMM_TC_STREAM])
def test_queue_epochs_equal_branch_epochs(fwd):
    """The work-queue layout (waves of persistent kernels taking (problem, tile) items) runs the same steps
    with the same arithmetic as the branch layout: models and step losses equal bit for bit after three
    epochs, on split-BF16 plans of uneven sizes (FFT lengths 256 .. 2048, one with reciprocity, mixed FFT
    variants), and within 1e-3 of the oracle's trajectories (the split-BF16 bar of the trajectory test)."""
    n_epochs, n_perm = 3, 2
    runs = {}
    for mode in (binding.MDC_BATCH_BRANCHES, binding.MDC_BATCH_QUEUE):
        members, data = [], []
        for k, shape in enumerate(MEMBERS):
            nt, nr, nv, ns, nb, recip = shape
            D, U_obs, perm, alpha, X0 = _member_data(k, shape, n_perm)
            plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, precision=binding.MDC_PREC_BF16X3)
            plan.set_config(fft_variant=[0, 1, 2][k % 3], gemm_fwd=fwd, gemm_adj=binding.MDC_GEMM_TC)
            steps = oracle.steps_per_epoch(ns, nb)
            members.append(dict(plan=plan, X=_cuda(X0), U_obs=_cuda(U_obs), perm=_cuda(perm, torch.int32), nb=nb,
                                alpha=alpha, flags=binding.SMDD_RECIPROCITY if recip else 0,
                                loss=torch.full((n_epochs, steps), -1.0, device="cuda", dtype=torch.float64)))
            data.append((D, U_obs, perm, alpha, X0, recip, steps))
        batch = binding.MDCBatch(members, n_branches=3, mode=mode)
        if mode == binding.MDC_BATCH_QUEUE:
            assert batch.kernels_per_epoch < 2 + sum(4 * s + 1 for s in batch.steps)
        batch.run(0, n_epochs)
        torch.cuda.synchronize()
        for m in members:
            assert m["plan"].sync_status() == binding.MDC_OK
        runs[mode] = ([m["X"].clone() for m in members], [m["loss"].clone() for m in members], data)
        batch.close()
    Xb, Lb, data = runs[binding.MDC_BATCH_BRANCHES]
    Xq, Lq, _ = runs[binding.MDC_BATCH_QUEUE]
    for k in range(len(MEMBERS)):
        assert torch.equal(Xq[k], Xb[k]), f"member {k}: queue model differs from the branch model"
        assert torch.equal(Lq[k], Lb[k]), f"member {k}: queue losses differ"
        D, U_obs, perm, alpha, X0, recip, steps = data[k]
        nb = MEMBERS[k][4]
        batches = [[perm[e % n_perm][s * nb:(s + 1) * nb] for s in range(steps)] for e in range(n_epochs)]
        X_ref, _ = oracle.run_epochs(D, X0, U_obs, batches, alpha, recip=recip, fft=True)
        assert oracle.rel_l2(Xq[k].double().cpu().numpy(), X_ref) <= 1e-3, f"member {k}"


def test_queue_mode_requires_tensor_core_products():
    nt, nr, nv, ns, nb, _ = MEMBERS[0]
    plan = binding.MDCPlan(_cuda(synth.random_traces((ns, nr, nt), 3)), nv, nb_max=nb)   # FP32 plan
    m = dict(plan=plan, X=torch.zeros((nv, nr, nt), device="cuda"), U_obs=torch.zeros((ns, nv, nt), device="cuda"),
             perm=torch.arange(ns, device="cuda", dtype=torch.int32)[None], nb=nb, alpha=0.1)
    with pytest.raises(binding.MDCError) as e:
        binding.MDCBatch([m], mode=binding.MDC_BATCH_QUEUE)
    assert e.value.status == binding.MDC_ERR_UNSUPPORTED
    with pytest.raises(binding.MDCError) as e:
        binding.MDCBatch([m], mode=7)
    assert e.value.status == binding.MDC_ERR_INVALID_ARG


def test_batch_replay_is_repeatable_and_reports_index_errors():
    shape = MEMBERS[1]
    nt, nr, nv, ns, nb, _ = shape
    D, U_obs, perm, alpha, X0 = _member_data(1, shape, 1)
    outs = []
    for _ in range(2):
        plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
        m = dict(plan=plan, X=_cuda(X0), U_obs=_cuda(U_obs), perm=_cuda(perm, torch.int32), nb=nb, alpha=alpha)
        batch = binding.MDCBatch([m], n_branches=4)
        assert batch.n_branches == 1      # clamped to the member count
        batch.run(5, 2)
        torch.cuda.synchronize()
        outs.append(m["X"].clone())
        batch.close()
    assert torch.equal(outs[0], outs[1])
    bad = perm.copy()
    bad[0, 3] = ns + 5
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    m = dict(plan=plan, X=_cuda(X0), U_obs=_cuda(U_obs), perm=_cuda(bad, torch.int32), nb=nb, alpha=alpha)
    batch = binding.MDCBatch([m])
    batch.run(0, 1)
    assert plan.sync_status() == binding.MDC_ERR_INDEX_RANGE
    batch.close()


def test_batch_host_errors():
    nt, nr, nv, ns, nb, _ = MEMBERS[0]
    D = _cuda(synth.random_traces((ns, nr, nt), 3))
    plan = binding.MDCPlan(D, nv, nb_max=nb)
    X = torch.zeros((nv, nr, nt), device="cuda")
    U = torch.zeros((ns, nv, nt), device="cuda")
    perm = torch.arange(ns, device="cuda", dtype=torch.int32)[None]
    base = dict(plan=plan, X=X, U_obs=U, perm=perm, nb=nb, alpha=0.1)
    with pytest.raises(binding.MDCError) as e:
        binding.MDCBatch([dict(base, nb=nb + 1)])
    assert e.value.status == binding.MDC_ERR_SHAPE
    with pytest.raises(binding.MDCError) as e:
        binding.MDCBatch([base, dict(base)])        # the same plan twice
    assert e.value.status == binding.MDC_ERR_INVALID_ARG
    with pytest.raises(binding.MDCError) as e:
        binding.MDCBatch([dict(base, flags=binding.SMDD_KEEP_XHAT)])
    assert e.value.status == binding.MDC_ERR_INVALID_ARG
    p2 = binding.MDCPlan(_cuda(synth.random_traces((5, 4, 8), 4)), 3, nb_max=2)
    with pytest.raises(binding.MDCError) as e:
        binding.MDCBatch([dict(plan=p2, X=torch.zeros((3, 4, 8), device="cuda"),
                               U_obs=torch.zeros((5, 3, 8), device="cuda"),
                               perm=torch.arange(5, device="cuda", dtype=torch.int32)[None], nb=2, alpha=0.1,
                               flags=binding.SMDD_RECIPROCITY)])
    assert e.value.status == binding.MDC_ERR_SHAPE

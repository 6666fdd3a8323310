"""The update of a symmetric model (SMDD_SYMMETRIC with reciprocity): only the traces on and above the
block diagonal are transformed and each result is written to (v, r) and (r, v); the spectra below the
block diagonal are filled by a transposed copy, and the adjoint product skips the mirrored copies of its
off-diagonal tiles.

On a symmetric model every trace of the full update is computed from the same inputs by the same
arithmetic as its mirror, so the flag must give the same bits as the step without it: X, the loss, and
(through SMDD_REUSE_XHAT) the model spectra used by the next step.  The FP64 oracle bounds the result
as for the plain step (relative L2 <= 1e-5, FP32 path)."""
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


# (nt, n, ns, nb): square model grids over the FFT lengths (and traces per CTA) of the radix kernels,
# n not a multiple of the traces per CTA nor of the 32-wide mirror tiles, several 128-wide adjoint tiles
SHAPES = [
    (128, 45, 37, 8),       # nfft 256
    (512, 70, 40, 16),      # nfft 1024
    (1000, 133, 30, 9),     # nfft 2048, two adjoint tile rows
    (1500, 150, 20, 7),     # nfft 3072 (radix 8 * 8 * 3 * 8)
    (1800, 21, 12, 5),      # nfft 4096
]


def _problem(nt, n, ns, seed):
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((ns, n, nt)).astype(np.float32) * 0.1
    X = rng.standard_normal((n, n, nt)).astype(np.float32)
    X = (0.5 * (X + X.transpose(1, 0, 2))).astype(np.float32)   # exactly symmetric in (v, r)
    U = rng.standard_normal((ns, n, nt)).astype(np.float32)
    return D, X, U


@pytest.mark.parametrize("prec", [binding.MDC_PREC_FP32, binding.MDC_PREC_BF16X3], ids=["fp32", "bf16x3"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{s[0]}x{s[1]}" for s in SHAPES])
@pytest.mark.parametrize("variant", [0, 1])
def test_symmetric_update_bit_identical(shape, prec, variant):
    nt, n, ns, nb = shape
    D, X, U = _problem(nt, n, ns, seed=nt + n)
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb, precision=prec)
    plan.set_config(fft_variant=variant, fft_prefetch=0)   # variant 1 falls back to 0 where it is the same plan
    alpha = 0.3 / plan.sigma2_max(30)
    rng = np.random.default_rng(7)
    batches = [rng.permutation(ns)[:nb].astype(np.int32) for _ in range(3)]
    Ug = _cuda(U)
    outs = []
    for sym in (False, True):
        Xg = _cuda(X)
        losses = []
        for k, b in enumerate(batches):
            fl = binding.SMDD_RECIPROCITY | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
            if sym:
                fl |= binding.SMDD_SYMMETRIC
            loss = torch.zeros((), dtype=torch.float64, device="cuda")
            plan.step(Xg, Ug, _cuda(b, torch.int32), alpha, fl, loss)
            losses.append(loss.item())
        assert plan.sync_status() == binding.MDC_OK
        outs.append((Xg.cpu().numpy(), losses))
    (Xa, la), (Xb, lb) = outs
    assert np.array_equal(Xa, Xb), f"max diff {np.max(np.abs(Xa - Xb))}"
    assert la == lb
    assert np.array_equal(Xb, Xb.transpose(1, 0, 2))   # exactly symmetric
    plan.close()


@pytest.mark.parametrize("shape", SHAPES[:4], ids=[f"{s[0]}x{s[1]}" for s in SHAPES[:4]])
def test_symmetric_step_matches_oracle(shape):
    nt, n, ns, nb = shape
    D, X, U = _problem(nt, n, ns, seed=3 * nt + n)
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb)
    # the register FFT where the plan has one: the symmetric update then runs the radix plan instead
    plan.set_config(fft_variant=2)
    alpha = 0.3 / plan.sigma2_max(30)
    idx = np.random.default_rng(5).permutation(ns)[:nb].astype(np.int32)
    Xg = _cuda(X)
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    plan.step(Xg, _cuda(U), _cuda(idx, torch.int32), alpha, binding.SMDD_RECIPROCITY | binding.SMDD_SYMMETRIC, loss)
    assert plan.sync_status() == binding.MDC_OK
    Xn_ref, l_ref = oracle.sgd_step(D, X, U, idx, alpha, recip=True)
    G = (X.astype(np.float64) - Xg.double().cpu().numpy()) / alpha
    G_ref = (X.astype(np.float64) - Xn_ref) / alpha
    assert oracle.rel_l2(G, G_ref) <= 1e-4, oracle.rel_l2(G, G_ref)
    assert oracle.rel_l2(Xg.double().cpu().numpy(), Xn_ref) <= 1e-5
    assert abs(loss.item() - l_ref) <= 1e-5 * l_ref
    plan.close()


def test_symmetric_flag_ignored_without_reciprocity():
    nt, n, ns, nb = 128, 20, 10, 4
    D, X, U = _problem(nt, n, ns, seed=11)
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb)
    idx = _cuda(np.arange(nb, dtype=np.int32), torch.int32)
    Xa, Xb = _cuda(X), _cuda(X)
    plan.step(Xa, _cuda(U), idx, 1e-3, 0)
    plan.step(Xb, _cuda(U), idx, 1e-3, binding.SMDD_SYMMETRIC)
    assert torch.equal(Xa, Xb)
    plan.close()


@pytest.mark.parametrize("solver", ["nsgd", "adam"])
@pytest.mark.parametrize("shape", [(512, 70, 40, 16), (1500, 45, 20, 7)], ids=lambda s: "x".join(map(str, s)))
def test_symmetric_momentum_and_adam_bit_identical(shape, solver):
    """N-SGD (velocity) and Adam (moments) with the causality mute on a symmetric model: the flagged steps
    mirror the state arrays too, and give the bits of the unflagged steps (X and the state, three steps)."""
    nt, n, ns, nb = shape
    D, X, U = _problem(nt, n, ns, seed=nt + 7)
    mute = _cuda(synth.direct_arrival_mute(n, n, nt), torch.int32)
    rng = np.random.default_rng(4)
    batches = [rng.permutation(ns)[:nb].astype(np.int32) for _ in range(3)]
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb)
    alpha = 0.2 / plan.sigma2_max(30)
    outs = []
    for sym in (False, True):
        Xg, Ug = _cuda(X), _cuda(U)
        A, B = torch.zeros_like(Xg), torch.zeros_like(Xg)
        for k, b in enumerate(batches):
            fl = binding.SMDD_RECIPROCITY | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
            fl |= binding.SMDD_SYMMETRIC if sym else 0
            ib = _cuda(b, torch.int32)
            if solver == "nsgd":
                plan.step_nsgd(Xg, A, Ug, ib, alpha, mu=0.9, flags=fl, mute=mute)
            else:
                plan.step_adam(Xg, A, B, Ug, ib, 1e-3, k + 1, flags=fl, mute=mute)
        assert plan.sync_status() == binding.MDC_OK
        outs.append([t.cpu().numpy() for t in (Xg, A, B)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert np.array_equal(outs[1][0], outs[1][0].transpose(1, 0, 2))
    plan.close()


def test_lower_spectra_read_transposed_or_copied_when_the_kernel_changes():
    """With the tile forward product the spectra below the block diagonal are not copied: the next
    forward product reads them transposed.  A plan switched to another forward kernel between two steps
    copies them into place first.  Either way the steps equal the steps without the flag bit for bit."""
    nt, n, ns, nb = 512, 70, 40, 16
    D, X, U = _problem(nt, n, ns, seed=21)
    rng = np.random.default_rng(9)
    batches = [rng.permutation(ns)[:nb].astype(np.int32) for _ in range(4)]
    kernels = [binding.MDC_GEMM_TC, binding.MDC_GEMM_TC, binding.MDC_GEMM_SIMT, binding.MDC_GEMM_TC]
    outs = []
    for sym in (False, True):
        plan = binding.MDCPlan(_cuda(D), n, nb_max=nb, precision=binding.MDC_PREC_BF16X3)
        alpha = 0.3 / plan.sigma2_max(30)
        Xg, Ug = _cuda(X), _cuda(U)
        for k, (b, fwd) in enumerate(zip(batches, kernels)):
            plan.set_config(fft_variant=0, fft_prefetch=0, gemm_fwd=fwd, gemm_adj=binding.MDC_GEMM_TC)
            fl = binding.SMDD_RECIPROCITY | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
            plan.step(Xg, Ug, _cuda(b, torch.int32), alpha, fl | (binding.SMDD_SYMMETRIC if sym else 0))
        assert plan.sync_status() == binding.MDC_OK
        outs.append(Xg.cpu().numpy())
        plan.close()
    assert np.array_equal(outs[0], outs[1])

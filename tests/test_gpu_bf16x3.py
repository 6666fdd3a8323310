"""Split-BF16 tensor-core products (MDC_PREC_BF16X3) against the FP64 oracle.

Tolerance (stated for this path): relative L2 error <= 1e-4.  Derivation: hi + lo keeps about 16
significant bits of each FP32 operand (relative error ~2^-17 each), the dropped lo*lo term is ~2^-16
smaller still, and the FP32 accumulation adds the FP32 rounding of the plain path; so an output carries
~1e-5 relative error, summed over K with random signs.  Elementwise: |gpu - oracle| <= 2e-4 max|oracle|.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_04486_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu
REL, ELEM = 1e-4, 2e-4


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


def _check(gpu, ref, what, rel=REL, elem=ELEM):
    gpu = np.asarray(gpu, dtype=np.float64)
    r = oracle.rel_l2(gpu, ref)
    m = np.max(np.abs(gpu - ref)) / max(np.max(np.abs(ref)), 1e-30)
    assert r <= rel, f"{what}: relative L2 {r:.3e}"
    assert m <= elem, f"{what}: elementwise {m:.3e}"


SHAPES = [
    (128, 32, 32, 32, 8),       # one M tile, one K chunk, batch tile 16
    (100, 37, 29, 41, 5),       # ragged
    (257, 130, 140, 150, 20),   # two M tiles, three K chunks, batch tile 32
    (64, 70, 65, 80, 70),       # batch 70: two batch tiles of 64, two adjoint K chunks
    (33, 5, 7, 6, 9),           # duplicates, tiny
]


def _problem(nt, nr, nv, ns, nb, seed):
    D = _f32(synth.random_traces((ns, nr, nt), seed))
    X = _f32(synth.random_traces((nv, nr, nt), seed + 1))
    R = _f32(synth.random_traces((nb, nv, nt), seed + 2))
    idx = synth.random_indices(ns, nb, seed + 3, replace=nb > ns)
    return D, X, R, idx


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_bf16x3_forward_and_adjoint(shape):
    nt, nr, nv, ns, nb = shape
    D, X, R, idx = _problem(nt, nr, nv, ns, nb, seed=3 * sum(shape))
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, scale=0.5, precision=binding.MDC_PREC_BF16X3)
    ti = _cuda(idx, torch.int32)
    U = plan.forward(_cuda(X), ti).cpu().numpy()
    G = plan.adjoint(_cuda(R), ti).cpu().numpy()
    assert plan.sync_status() == binding.MDC_OK
    _check(U, oracle.mdc_forward(D, X, idx, 0.5), f"U {shape}")
    _check(G, oracle.mdc_adjoint(D, R, idx, 0.5), f"G {shape}")


@pytest.mark.parametrize("shape", [(128, 32, 32, 32, 8), (64, 150, 150, 160, 24)])
def test_bf16x3_step_with_reciprocity(shape):
    nt, nr, nv, ns, nb = shape
    D, X, _, idx = _problem(nt, nr, nv, ns, nb, seed=5)
    X = _f32(0.5 * (X + X.transpose(1, 0, 2)))
    U_obs = _f32(synth.random_traces((ns, nv, nt), 6))
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, precision=binding.MDC_PREC_BF16X3)
    Xg = _cuda(X)
    loss = torch.zeros((), device="cuda", dtype=torch.float64)
    alpha = 1e-4
    plan.step(Xg, _cuda(U_obs), _cuda(idx, torch.int32), alpha, binding.SMDD_RECIPROCITY, loss)
    assert plan.sync_status() == binding.MDC_OK
    g, l_ref, _ = oracle.gradient(D, X, U_obs, idx)
    g = oracle.reciprocity(g)
    _check((X - Xg.double().cpu().numpy()) / alpha, g, f"step gradient {shape}", rel=3e-4, elem=6e-4)
    assert abs(loss.item() - l_ref) <= 1e-4 * l_ref
    Xo = Xg.cpu().numpy()
    np.testing.assert_array_equal(Xo, Xo.transpose(1, 0, 2))


def test_bf16x3_dot_product():
    nt, nr, nv, ns, nb = 200, 60, 50, 70, 12
    D, X, Y, idx = _problem(nt, nr, nv, ns, nb, seed=9)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, precision=binding.MDC_PREC_BF16X3)
    ti = _cuda(idx, torch.int32)
    U = plan.forward(_cuda(X), ti).double().cpu().numpy()
    G = plan.adjoint(_cuda(Y), ti).double().cpu().numpy()
    assert abs(np.vdot(U, Y) - np.vdot(X, G)) <= 1e-4 * np.linalg.norm(U) * np.linalg.norm(Y)


STREAM_SHAPES = SHAPES + [
    (64, 301, 301, 40, 32),     # nr = 301: five K chunks, the last one 45 wide; v tail of 45 rows
    (40, 20, 300, 90, 65),      # three v tiles, two batch tiles of 64 (the second with one column)
    (24, 16, 16, 20, 1),        # batch of one
]


@pytest.mark.parametrize("shape", STREAM_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("band", [0, 5], ids=["full", "band5"])
def test_streamed_forward_equals_tile_kernel(shape, band):
    """MDC_GEMM_TC_STREAM (persistent, fed by tensor-memory-accelerator copies) splits the same values
    and issues the same MMAs in the same order as MDC_GEMM_TC, so the two forward products agree bit for
    bit; both meet the split-BF16 bar against the oracle (with a band limit, the oracle's band-limited
    Tier B)."""
    nt, nr, nv, ns, nb = shape
    D, X, _, idx = _problem(nt, nr, nv, ns, nb, seed=7 * sum(shape) + band)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, precision=binding.MDC_PREC_BF16X3)
    if band:
        plan.set_band(band)
    ti, Xg = _cuda(idx, torch.int32), _cuda(X)
    plan.set_config(gemm_fwd=binding.MDC_GEMM_TC, gemm_adj=binding.MDC_GEMM_TC)
    U_tile = plan.forward(Xg, ti).cpu().numpy()
    plan.set_config(gemm_fwd=binding.MDC_GEMM_TC_STREAM, gemm_adj=binding.MDC_GEMM_TC)
    U = plan.forward(Xg, ti).cpu().numpy()
    assert plan.sync_status() == binding.MDC_OK
    np.testing.assert_array_equal(U, U_tile)
    ref = oracle.mdc_forward_fft(D, X, idx, band=band) if band else oracle.mdc_forward(D, X, idx)
    _check(U, ref, f"U {shape}")


def test_streamed_forward_reports_index_errors():
    nt, nr, nv, ns, nb = 64, 40, 40, 30, 8
    D, X, _, idx = _problem(nt, nr, nv, ns, nb, seed=11)
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, precision=binding.MDC_PREC_BF16X3)
    plan.set_config(gemm_fwd=binding.MDC_GEMM_TC_STREAM, gemm_adj=binding.MDC_GEMM_TC)
    bad = idx.copy()
    bad[3] = ns + 2
    plan.forward(_cuda(X), _cuda(bad, torch.int32))
    assert plan.sync_status() == binding.MDC_ERR_INDEX_RANGE
    U = plan.forward(_cuda(X), _cuda(idx, torch.int32)).cpu().numpy()
    assert plan.sync_status() == binding.MDC_OK
    _check(U, oracle.mdc_forward(D, X, idx), "U after the error")
    fp32 = binding.MDCPlan(_cuda(D), nv, nb_max=nb)
    with pytest.raises(binding.MDCError) as e:
        fp32.set_config(gemm_fwd=binding.MDC_GEMM_TC_STREAM)
    assert e.value.status == binding.MDC_ERR_UNSUPPORTED


@pytest.mark.parametrize("shape", [(100, 37, 29, 41, 5), (64, 150, 140, 160, 24), (257, 130, 130, 70, 40),
                                   (64, 140, 140, 80, 64)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("recip", [False, True])
def test_adjoint_operand_images_equal_inline_split(shape, recip):
    """The adjoint products from the per-step operand images (plans for batches up to 64) against the
    products that load and split their operands themselves (a plan for larger batches): the same split and
    the same MMAs in the same order, so bit-identical gradients and steps; ragged blocks, one and two K
    chunks, an out-of-range source index reported."""
    nt, nr, nv, ns, nb = shape
    if recip:
        nv = nr
    seed = sum(shape) + recip
    D = _f32(synth.random_traces((ns, nr, nt), seed))
    R = _f32(synth.random_traces((nb, nv, nt), seed + 1))
    X = _f32(oracle.reciprocity(synth.random_traces((nv, nr, nt), seed + 2))) if recip else \
        _f32(synth.random_traces((nv, nr, nt), seed + 2))
    U = _f32(synth.random_traces((ns, nv, nt), seed + 3))
    idx = synth.random_indices(ns, nb, seed + 4)
    ti = _cuda(idx, torch.int32)
    out = []
    for nb_max in (nb, 65):   # images held / not held
        plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb_max, precision=binding.MDC_PREC_BF16X3)
        plan.set_config(gemm_fwd=binding.MDC_GEMM_TC, gemm_adj=binding.MDC_GEMM_TC)
        G = plan.adjoint(_cuda(R), ti)
        Xg = _cuda(X)
        plan.step(Xg, _cuda(U), ti, 1e-3, binding.SMDD_RECIPROCITY if recip else 0)
        assert plan.sync_status() == binding.MDC_OK
        out.append((G.cpu().numpy(), Xg.cpu().numpy()))
        plan.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    _check(out[0][0], oracle.mdc_adjoint(D, R, idx), "G")
    # an out-of-range index is reported by the image construction; its batch entry contributes nothing
    plan = binding.MDCPlan(_cuda(D), nv, nb_max=nb, precision=binding.MDC_PREC_BF16X3)
    plan.set_config(gemm_adj=binding.MDC_GEMM_TC)
    bad = idx.copy()
    bad[0] = ns + 3
    G = plan.adjoint(_cuda(R), _cuda(bad, torch.int32)).cpu().numpy()
    assert plan.sync_status() == binding.MDC_ERR_INDEX_RANGE
    keep = np.arange(1, nb)
    _check(G, oracle.mdc_adjoint(D, R[keep], bad[keep]), "G without the bad entry")
    plan.close()

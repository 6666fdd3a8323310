"""Pins for the FP64 oracle: each check is fixed by the paper or by mathematics, not by the oracle itself.

A plausible mistake in the oracle (a dropped term, a sign, a transposed operand, an off-by-one in the
causal window or in the correlation lag, a wrong source index) fails at least one of these.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2202_04486_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_operator(D, idx, nv, scale=1.0):
    """Dense matrix of the batch MDC built from scipy Toeplitz blocks (independent of the oracle's loops).

    Rows: (b, v, t) of U; columns: (v', r, tau) of X.  Block (b, v; v', r) = delta_{v v'} * T(D[idx_b, r]),
    T(d) the lower-triangular Toeplitz matrix with first column d (causal convolution, truncated)."""
    ns, nr, nt = D.shape
    nb = len(idx)
    A = np.zeros((nb * nv * nt, nv * nr * nt))
    for b, s in enumerate(idx):
        for r in range(nr):
            T = scipy.linalg.toeplitz(D[s, r], np.zeros(nt))
            for v in range(nv):
                A[(b * nv + v) * nt:(b * nv + v + 1) * nt, (v * nr + r) * nt:(v * nr + r + 1) * nt] = scale * T
    return A


# ------------------------------------------------------------------------------------------ 1D case
@pytest.mark.parametrize("nt", [1, 2, 7, 33])
def test_1d_forward_is_numpy_convolve(nt):
    d = synth.random_traces((1, 1, nt), seed=nt)
    x = synth.random_traces((1, 1, nt), seed=100 + nt)
    U = oracle.mdc_forward(d, x, [0])
    np.testing.assert_allclose(U[0, 0], np.convolve(d[0, 0], x[0, 0])[:nt], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("nt", [1, 2, 7, 33])
def test_1d_adjoint_is_numpy_correlate(nt):
    d = synth.random_traces((1, 1, nt), seed=nt)
    r = synth.random_traces((1, 1, nt), seed=200 + nt)
    G = oracle.mdc_adjoint(d, r, [0])
    # correlate(r, d, 'full')[nt-1+tau] = sum_t r[t+tau] d[t]  ->  G[tau] = sum_t d[t-tau] r[t]
    ref = np.correlate(r[0, 0], d[0, 0], mode="full")[nt - 1:]
    np.testing.assert_allclose(G[0, 0], ref, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------------------------------------ delta kernel
@pytest.mark.parametrize("k", [0, 1, 5])
def test_delta_kernel_shifts_model(k):
    """D[s, r, t] = delta_{sr} delta_{t,k}: U[b, v, t] = X[v, idx_b, t - k] (zero filled, truncated)."""
    n, nt, nv = 5, 12, 3
    D = np.zeros((n, n, nt))
    for s in range(n):
        D[s, s, k] = 1.0
    X = synth.random_traces((nv, n, nt), seed=3)
    idx = np.array([4, 0, 2, 2])
    U = oracle.mdc_forward(D, X, idx)
    ref = np.zeros_like(U)
    for b, s in enumerate(idx):
        ref[b, :, k:] = X[:, s, :nt - k]
    np.testing.assert_array_equal(U, ref)
    # and the adjoint moves the residual back by k into receiver idx_b
    R = synth.random_traces((len(idx), nv, nt), seed=4)
    G = oracle.mdc_adjoint(D, R, idx)
    refG = np.zeros((nv, n, nt))
    for b, s in enumerate(idx):
        refG[:, s, :nt - k] += R[b, :, k:]
    np.testing.assert_allclose(G, refG, rtol=0, atol=1e-15)


# ------------------------------------------------------------------------------------------ brute force
@pytest.mark.parametrize("shape", [(1, 2, 1, 3, 2), (4, 2, 3, 3, 3), (6, 3, 2, 4, 2), (5, 2, 2, 2, 4)])
def test_dense_operator_brute_force(shape):
    nt, nr, nv, ns, nb = shape
    D = synth.random_traces((ns, nr, nt), seed=11)
    X = synth.random_traces((nv, nr, nt), seed=12)
    R = synth.random_traces((nb, nv, nt), seed=13)
    idx = synth.random_indices(ns, nb, seed=14, replace=True)
    A = _dense_operator(D, idx, nv, scale=0.7)
    U = oracle.mdc_forward(D, X, idx, scale=0.7)
    np.testing.assert_allclose(U.ravel(), A @ X.ravel(), rtol=1e-12, atol=1e-12)
    G = oracle.mdc_adjoint(D, R, idx, scale=0.7)
    np.testing.assert_allclose(G.ravel(), A.T @ R.ravel(), rtol=1e-12, atol=1e-12)


def test_virtual_source_selection_matches_full():
    D = synth.random_traces((6, 4, 9), seed=1)
    X = synth.random_traces((5, 4, 9), seed=2)
    R = synth.random_traces((3, 5, 9), seed=3)
    idx = np.array([5, 1, 3])
    vsel = np.array([4, 0, 2])
    np.testing.assert_array_equal(oracle.mdc_forward(D, X, idx, vsel=vsel), oracle.mdc_forward(D, X, idx)[:, vsel])
    np.testing.assert_array_equal(oracle.mdc_adjoint(D, R, idx, vsel=vsel), oracle.mdc_adjoint(D, R, idx)[vsel])


def test_invalid_index_rejected():
    D = np.zeros((3, 2, 4))
    X = np.zeros((2, 2, 4))
    with pytest.raises(ValueError):
        oracle.mdc_forward(D, X, [3])
    with pytest.raises(ValueError):
        oracle.mdc_adjoint(D, np.zeros((1, 2, 4)), [-1])


# ------------------------------------------------------------------------------------------ dot test
@pytest.mark.parametrize("shape", [(16, 5, 4, 7, 3), (37, 3, 6, 5, 5)])
def test_adjoint_dot_product(shape):
    nt, nr, nv, ns, nb = shape
    D = synth.random_traces((ns, nr, nt), seed=21)
    X = synth.random_traces((nv, nr, nt), seed=22)
    Y = synth.random_traces((nb, nv, nt), seed=23)
    idx = synth.random_indices(ns, nb, seed=24)
    lhs = np.vdot(oracle.mdc_forward(D, X, idx), Y)
    rhs = np.vdot(X, oracle.mdc_adjoint(D, Y, idx))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


# ------------------------------------------------------------------------------------------ finite sum
def test_finite_sum_identity():
    """Eq. 5/6: the batch gradients over a partition of the sources add up to the full gradient."""
    nt, nr, nv, ns, nb = 20, 4, 3, 11, 4
    D = synth.random_traces((ns, nr, nt), seed=31)
    X = synth.random_traces((nv, nr, nt), seed=32)
    U = synth.random_traces((ns, nv, nt), seed=33)
    g_full, l_full, _ = oracle.gradient(D, X, U, np.arange(ns))
    batches = synth.epoch_batches(ns, nb, 1, seed=5)[0]
    assert len(batches) == oracle.steps_per_epoch(ns, nb) == 3
    parts = [oracle.gradient(D, X, U, b) for b in batches]
    g_sum = sum(p[0] for p in parts)
    l_sum = sum(p[1] for p in parts)
    assert np.linalg.norm(g_sum - g_full) <= 1e-13 * np.linalg.norm(g_full)
    assert abs(l_sum - l_full) <= 1e-13 * l_full
    # duplicates count twice, exactly as in the sum of Eq. 6
    g_dup, _, _ = oracle.gradient(D, X, U, [2, 2])
    g_one, _, _ = oracle.gradient(D, X, U, [2])
    np.testing.assert_allclose(g_dup, 2 * g_one, rtol=1e-14, atol=1e-14)


def test_gradient_is_derivative_of_loss():
    """g_B is the gradient of 1/2||P_B X - U_B||^2 (central differences; the loss is quadratic so they are exact)."""
    nt, nr, nv, ns = 8, 3, 2, 4
    D = synth.random_traces((ns, nr, nt), seed=41)
    X = synth.random_traces((nv, nr, nt), seed=42)
    U = synth.random_traces((ns, nv, nt), seed=43)
    idx = [3, 1]
    g, _, _ = oracle.gradient(D, X, U, idx)
    E = synth.random_traces(X.shape, seed=44)
    h = 1e-3
    lp = oracle.gradient(D, X + h * E, U, idx)[1]
    lm = oracle.gradient(D, X - h * E, U, idx)[1]
    assert abs((lp - lm) / (2 * h) - np.vdot(g, E)) <= 1e-9 * max(1.0, abs(np.vdot(g, E)))


# ------------------------------------------------------------------------------------------ Tier B
@pytest.mark.parametrize("shape", [(1, 1, 1, 1, 1), (13, 3, 4, 5, 2), (64, 6, 5, 7, 4), (100, 2, 3, 3, 3)])
def test_tier_b_fft_matches_direct_sums(shape):
    nt, nr, nv, ns, nb = shape
    D = synth.random_traces((ns, nr, nt), seed=51)
    X = synth.random_traces((nv, nr, nt), seed=52)
    R = synth.random_traces((nb, nv, nt), seed=53)
    idx = synth.random_indices(ns, nb, seed=54)
    assert oracle.rel_l2(oracle.mdc_forward_fft(D, X, idx, 1.3), oracle.mdc_forward(D, X, idx, 1.3)) < 1e-12
    assert oracle.rel_l2(oracle.mdc_adjoint_fft(D, R, idx, 1.3), oracle.mdc_adjoint(D, R, idx, 1.3)) < 1e-12


def test_nfft_too_short_is_circular_and_rejected():
    with pytest.raises(AssertionError):
        oracle.mdc_forward_fft(np.zeros((1, 1, 8)), np.zeros((1, 1, 8)), [0], nfft=8)


# ------------------------------------------------------------------------------------------ Landweber (App. B)
def test_landweber_toy():
    g = json.load(open(os.path.join(GOLDEN, "landweber_toy.json")))
    A = np.array(g["A"], float)
    x = np.array(g["x"], float)
    s2 = np.linalg.norm(A, 2) ** 2
    assert round(s2) == g["sigma2_printed"]
    assert abs(s2 - (67 + math.sqrt(1525)) / 2) < 1e-12
    y = A @ x
    ok = oracle.landweber(A, y, g["bound_fraction_converges"] / s2, 400)
    bad = oracle.landweber(A, y, g["bound_fraction_diverges"] / s2, 400)
    assert np.linalg.norm(ok[-1] - x) < 1e-6
    assert np.linalg.norm(bad[-1] - x) > 1e3
    # the residual of the divergent run grows geometrically at the rate |1 - alpha sigma^2| = 1.05
    e = [np.linalg.norm(it - x) for it in bad[-20:]]
    assert 1.04 < (e[-1] / e[0]) ** (1 / 19) < 1.06


def test_sigma2_bounds_operator_norm():
    """sigma_max of the truncated time-domain operator <= max_f sigma_max(Dh_f) (its circulant embedding),
    and the bound tightens as the record gets longer than the kernel support."""
    rng_D = synth.random_traces((3, 2, 6), seed=61)
    ratios = []
    for nt in (6, 24, 96):
        D = np.zeros((3, 2, nt))
        D[:, :, :6] = rng_D
        A = _dense_operator(D, [0, 1, 2], nv=1)
        s2_op = np.linalg.norm(A, 2) ** 2
        s2_k = oracle.sigma2_max(D)
        assert s2_op <= s2_k * (1 + 1e-12)
        ratios.append(s2_op / s2_k)
    assert ratios[0] < ratios[1] < ratios[2] and ratios[2] > 0.95


def test_sigma2_scaled_operator():
    """With scale != 1 the operator is scale * P, so its squared norm is scale^2 times that of P: the
    bound of the scaled dense operator (built here independently, scale inside every Toeplitz block) keeps
    the same ratio to oracle.sigma2_max(D, scale=...) as at scale 1, and tightens the same way with a
    long record.  A factor of scale instead of scale^2 moves the ratio by 0.7 and fails."""
    rng_D = synth.random_traces((3, 2, 6), seed=62)
    for scale in (0.7, 2.5):
        D = np.zeros((3, 2, 96))
        D[:, :, :6] = rng_D
        A = _dense_operator(D, [0, 1, 2], nv=1, scale=scale)
        s2_op = np.linalg.norm(A, 2) ** 2
        s2_k = oracle.sigma2_max(D, scale=scale)
        assert s2_op <= s2_k * (1 + 1e-12)
        assert s2_op / s2_k > 0.95


def test_sgd_full_batch_is_landweber_and_converges_to_lstsq():
    """Full-batch SGD with alpha < 2/sigma^2 is the Landweber iteration; from 0 on a consistent system it
    converges to the minimum-norm least-squares solution (numpy.linalg.lstsq on the dense operator)."""
    nt, nr, nv, ns = 5, 2, 2, 4
    D = synth.random_traces((ns, nr, nt), seed=71)
    Xt = synth.random_traces((nv, nr, nt), seed=72)
    U = oracle.mdc_forward(D, Xt, np.arange(ns))
    A = _dense_operator(D, np.arange(ns), nv)
    s2 = np.linalg.norm(A, 2) ** 2
    X = np.zeros_like(Xt)
    alpha = 1.9 / s2
    for _ in range(4000):
        X, _ = oracle.sgd_step(D, X, U, np.arange(ns), alpha)
    x_ls = np.linalg.lstsq(A, U.ravel(), rcond=None)[0]
    assert np.linalg.norm(X.ravel() - x_ls) < 1e-6 * np.linalg.norm(x_ls)


def test_sgd_minibatch_converges_on_consistent_problem():
    nt, nr, nv, ns, nb = 5, 2, 2, 6, 2
    D = synth.random_traces((ns, nr, nt), seed=81)
    Xt = synth.random_traces((nv, nr, nt), seed=82)
    U = oracle.mdc_forward(D, Xt, np.arange(ns))
    A = _dense_operator(D, np.arange(ns), nv)
    alpha = 0.5 / (np.linalg.norm(A, 2) ** 2)
    X, losses = oracle.run_epochs(D, np.zeros_like(Xt), U, synth.epoch_batches(ns, nb, 1500, seed=1), alpha)
    x_ls = np.linalg.lstsq(A, U.ravel(), rcond=None)[0]
    assert np.linalg.norm(X.ravel() - x_ls) < 1e-5 * np.linalg.norm(x_ls)
    assert losses[-1] < 1e-12 * losses[0]


# ------------------------------------------------------------------------------------------ reciprocity
def test_reciprocity_keeps_model_symmetric():
    n, nt, ns = 4, 10, 5
    D = synth.random_traces((ns, n, nt), seed=91)
    Xt = synth.random_traces((n, n, nt), seed=92)
    Xt = Xt + Xt.transpose(1, 0, 2)
    U = oracle.mdc_forward(D, Xt, np.arange(ns))
    X = np.zeros_like(Xt)
    for idx in synth.epoch_batches(ns, 2, 3, seed=2)[0]:
        g, _, _ = oracle.gradient(D, X, U, idx)
        Xn, _ = oracle.sgd_step(D, X, U, idx, 1e-3, recip=True)
        np.testing.assert_array_equal(Xn, Xn.transpose(1, 0, 2))
        np.testing.assert_allclose((X - Xn) / 1e-3, 0.5 * (g + g.transpose(1, 0, 2)), rtol=1e-9, atol=1e-12)
        X = Xn


def test_reciprocity_is_orthogonal_projection():
    G = synth.random_traces((3, 3, 4), seed=93)
    P = oracle.reciprocity(G)
    np.testing.assert_allclose(oracle.reciprocity(P), P, rtol=0, atol=0)
    H = synth.random_traces((3, 3, 4), seed=94)
    assert abs(np.vdot(oracle.reciprocity(G), H) - np.vdot(G, oracle.reciprocity(H))) < 1e-12


# ------------------------------------------------------------------------------------------ epoch + metrics
def test_steps_per_epoch_golden():
    g = json.load(open(os.path.join(GOLDEN, "epoch_counts.json")))
    for c in g["printed"] + g["reading_cases"]:
        assert oracle.steps_per_epoch(c["ns"], c["nb"]) == c["steps"]
        b = synth.epoch_batches(c["ns"], c["nb"], 2, seed=0)
        assert all(len(e) == c["steps"] for e in b)
        for e in b:
            assert sorted(np.concatenate(e).tolist()) == list(range(c["ns"]))


def test_rmse_reading():
    x = synth.random_traces((3, 4, 5), seed=95)
    assert oracle.rmse(x, x) == 0.0
    assert oracle.rmse(x, 3.0 * x) < 1e-15
    y = np.zeros_like(x)
    y.flat[0] = 1.0
    a = x / np.max(np.abs(x))
    assert abs(oracle.rmse(x, y) - math.sqrt(np.sum((a - y) ** 2))) < 1e-14


def test_generator_reciprocal_and_seeded():
    p = synth.make_problem(64, 6, 6, 7, seed=3)
    np.testing.assert_array_equal(p.X_true, p.X_true.transpose(1, 0, 2))
    q = synth.make_problem(64, 6, 6, 7, seed=3)
    np.testing.assert_array_equal(p.D, q.D)
    assert np.max(np.abs(p.D)) > 0.5 and np.max(np.abs(p.X_true)) > 0.1


# ------------------------------------------------------------------------------------------------
# N-SGD (Nesterov momentum after Sutskever et al. 2013) and the causality mute
# ------------------------------------------------------------------------------------------------
def _dense_quadratic(seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((12, 7)) @ np.diag([3, 2, 1.5, 1, 0.7, 0.5, 0.3])
    b = rng.standard_normal(12)
    return A, b


def test_nsgd_lookahead_form_equals_sutskever_form():
    """With nt = 1 and one virtual source the MDC is a dense product, U[s] = sum_r D[s, r] x[r], so the
    oracle's N-SGD steps on f(x) = 1/2 ||A x - b||^2 (A = D[:, :, 0]) can be checked against Sutskever's
    form iterated directly: gradient at x + mu v, x' = x + v'; the oracle's X is y = x + mu v."""
    A, b = _dense_quadratic(5)
    alpha, mu = 0.02, 0.9
    D = A[:, :, None]
    U = b[:, None, None]
    grad = lambda z: A.T @ (A @ z - b)
    x, v = np.zeros(7), np.zeros(7)
    Y, W = np.zeros((1, 7, 1)), np.zeros((1, 7, 1))
    for _ in range(40):
        v = mu * v - alpha * grad(x + mu * v)
        x = x + v
        Y, W, _ = oracle.nsgd_step(D, Y, W, U, np.arange(12), alpha, mu)
        np.testing.assert_allclose(Y.ravel(), x + mu * v, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(W.ravel(), v, rtol=1e-11, atol=1e-12)


def test_nsgd_with_zero_momentum_is_sgd():
    nt, nr, nv, ns = 20, 4, 3, 6
    D = synth.random_traces((ns, nr, nt), 1)
    X = synth.random_traces((nv, nr, nt), 2)
    U = synth.random_traces((ns, nv, nt), 3)
    idx = np.array([4, 1, 2])
    Xs, ls = oracle.sgd_step(D, X, U, idx, 0.01)
    g, _, _ = oracle.gradient(D, X, U, idx)
    Xn, Vn, ln = oracle.nsgd_step(D, X, np.zeros_like(X), U, idx, 0.01, 0.0)
    np.testing.assert_array_equal(Xn, Xs)
    np.testing.assert_array_equal(Vn, -0.01 * g)
    assert ln == ls


def test_nsgd_full_batch_converges_to_min_norm_solution():
    """Full-batch N-SGD from zero on a tiny consistent 1-source-per-row problem converges to the
    minimum-norm least-squares solution of the dense operator (numpy.linalg.lstsq)."""
    nt, nr, nv, ns = 6, 2, 1, 5      # condition number ~8: converged to rounding in 3000 steps
    D = synth.random_traces((ns, nr, nt), 11)
    Xt = synth.random_traces((nv, nr, nt), 12)
    U = oracle.mdc_forward(D, Xt, np.arange(ns))
    A = np.zeros((ns * nv * nt, nv * nr * nt))
    for j in range(nv * nr * nt):
        e = np.zeros(nv * nr * nt)
        e[j] = 1.0
        A[:, j] = oracle.mdc_forward(D, e.reshape(nv, nr, nt), np.arange(ns)).ravel()
    x_ls = np.linalg.lstsq(A, U.ravel(), rcond=None)[0]
    s2 = np.linalg.norm(A, 2) ** 2
    X, V = np.zeros((nv, nr, nt)), np.zeros((nv, nr, nt))
    for _ in range(3000):
        X, V, _ = oracle.nsgd_step(D, X, V, U, np.arange(ns), 0.5 / s2, 0.9)
    assert np.linalg.norm(X.ravel() - x_ls) <= 1e-6 * np.linalg.norm(x_ls)


def test_adam_against_element_loop():
    """Three Adam steps of the oracle against Kingma & Ba's Algorithm 1 written out element by element,
    on a gradient taken from the dense Toeplitz operator (independent of the oracle's sums), with
    reciprocity and a causality mute so that the preconditioned gradient is what the moments see."""
    n, nt, ns = 3, 7, 4
    D = synth.random_traces((ns, n, nt), 91)
    Xt = synth.random_traces((n, n, nt), 92)
    Xt = 0.5 * (Xt + Xt.transpose(1, 0, 2))
    U = oracle.mdc_forward(D, Xt, np.arange(ns)) + 0.1 * synth.random_traces((ns, n, nt), 93)
    first = np.array([[0, 2, 4], [2, 0, 1], [4, 1, 0]])
    idx = np.array([3, 1])
    A = _dense_operator(D, idx, n)
    alpha, b1, b2, eps = 0.01, 0.8, 0.95, 1e-6
    X, M, V = np.zeros((n, n, nt)), np.zeros((n, n, nt)), np.zeros((n, n, nt))
    x, m, v = X.ravel().copy(), M.ravel().copy(), V.ravel().copy()
    for t in range(1, 4):
        g = (A.T @ (A @ x - U[idx].ravel())).reshape(n, n, nt)
        g = 0.5 * (g + g.transpose(1, 0, 2))
        g = g.ravel()
        for j in range(x.size):
            vv, rr, tt = np.unravel_index(j, (n, n, nt))
            gj = 0.0 if tt < first[vv, rr] else g[j]
            m[j] = b1 * m[j] + (1 - b1) * gj
            v[j] = b2 * v[j] + (1 - b2) * gj * gj
            mh = m[j] / (1 - b1 ** t)
            vh = v[j] / (1 - b2 ** t)
            x[j] = x[j] - alpha * mh / (math.sqrt(vh) + eps)
        X, M, V, _ = oracle.adam_step(D, X, M, V, U, idx, alpha, t, beta1=b1, beta2=b2, eps=eps, recip=True, mute=first)
        np.testing.assert_allclose(X.ravel(), x, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(M.ravel(), m, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(V.ravel(), v, rtol=1e-12, atol=1e-16)
    # the model stays symmetric and zero above the mute
    np.testing.assert_array_equal(X, X.transpose(1, 0, 2))
    assert np.all(X[np.arange(nt)[None, None, :] < first[:, :, None]] == 0.0)


def test_adam_first_step_has_size_alpha():
    """From zero moments the bias corrections make the first step alpha * g / (|g| + eps): of size alpha
    wherever |g| >> eps, whatever the scale of the gradient (a dropped correction gives (1-beta1)/sqrt(1-beta2))."""
    nt, nr, nv, ns = 16, 3, 2, 5
    D = 1e3 * synth.random_traces((ns, nr, nt), 94)
    X = synth.random_traces((nv, nr, nt), 95)
    U = synth.random_traces((ns, nv, nt), 96)
    idx = np.array([0, 4])
    g, _, _ = oracle.gradient(D, X, U, idx)
    Xn, _, _, _ = oracle.adam_step(D, X, np.zeros_like(X), np.zeros_like(X), U, idx, 0.003, 1)
    big = np.abs(g) > 1e3 * 1e-8
    assert big.mean() > 0.9
    np.testing.assert_allclose(np.abs(Xn - X)[big], 0.003, rtol=1e-5)
    np.testing.assert_array_equal(np.sign(X - Xn)[big], np.sign(g)[big])


def test_adam_without_averaging_is_sign_descent():
    """beta1 = beta2 = 0: m_hat = g and v_hat = g^2 at every step, so Adam moves each element by
    alpha * g / (|g| + eps), a signed step of size ~alpha."""
    nt, nr, nv, ns = 9, 2, 2, 3
    D = synth.random_traces((ns, nr, nt), 97)
    X = synth.random_traces((nv, nr, nt), 98)
    U = synth.random_traces((ns, nv, nt), 99)
    M = synth.random_traces((nv, nr, nt), 100)
    V = np.abs(synth.random_traces((nv, nr, nt), 101))
    g, _, _ = oracle.gradient(D, X, U, [2, 0])
    Xn, Mn, Vn, _ = oracle.adam_step(D, X, M, V, U, [2, 0], 0.1, 5, beta1=0.0, beta2=0.0, eps=1e-8)
    np.testing.assert_allclose(Xn, X - 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(Mn, g, rtol=0, atol=0)
    np.testing.assert_allclose(Vn, g * g, rtol=0, atol=0)


def test_adam_full_batch_converges_to_least_squares():
    """Full-batch Adam from zero with the decaying step alpha_t = 0.2 / sqrt(t) on a tiny consistent
    over-determined problem (ns > nr: the dense operator has full column rank) converges to its unique
    least-squares solution, the true model."""
    nt, nr, nv, ns = 6, 2, 1, 5
    D = synth.random_traces((ns, nr, nt), 11)
    Xt = synth.random_traces((nv, nr, nt), 12)
    U = oracle.mdc_forward(D, Xt, np.arange(ns))
    A = _dense_operator(D, np.arange(ns), nv)
    x_ls = np.linalg.lstsq(A, U.ravel(), rcond=None)[0]
    assert np.linalg.matrix_rank(A) == A.shape[1]
    X, M, V = np.zeros((nv, nr, nt)), np.zeros((nv, nr, nt)), np.zeros((nv, nr, nt))
    for t in range(1, 3001):
        X, M, V, _ = oracle.adam_step(D, X, M, V, U, np.arange(ns), 0.2 / math.sqrt(t), t)
    assert np.linalg.norm(X.ravel() - x_ls) <= 1e-9 * np.linalg.norm(x_ls)


def test_causal_mute_against_loop():
    G = synth.random_traces((3, 4, 10), 21)
    first = np.array([[0, 3, 10, 12], [1, 0, 5, 9], [2, 2, 2, 2]])
    M = oracle.causal_mute(G, first)
    for v in range(3):
        for r in range(4):
            for t in range(10):
                assert M[v, r, t] == (0.0 if t < first[v, r] else G[v, r, t])


def test_nsgd_mute_and_reciprocity_keep_model_in_range():
    """Starting from zero with a symmetric mute table, N-SGD with C = C_r C_c keeps X symmetric and zero
    above the mute, and the unmuted samples move as the unmuted step does."""
    n, nt, ns = 5, 16, 7
    D = synth.random_traces((ns, n, nt), 31)
    U = synth.random_traces((ns, n, nt), 32)
    first = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]) * 2
    X, V = np.zeros((n, n, nt)), np.zeros((n, n, nt))
    for k in range(4):
        idx = synth.random_indices(ns, 3, 40 + k)
        X, V, _ = oracle.nsgd_step(D, X, V, U, idx, 1e-3, 0.9, recip=True, mute=first)
        np.testing.assert_array_equal(X, np.transpose(X, (1, 0, 2)))
        t = np.arange(nt)
        assert np.all(X[t[None, None, :] < first[:, :, None]] == 0.0)
    g, _, _ = oracle.gradient(D, np.zeros((n, n, nt)), U, np.array([0, 1]))
    X1, _, _ = oracle.nsgd_step(D, np.zeros((n, n, nt)), np.zeros((n, n, nt)), U, np.array([0, 1]), 1e-3, 0.5,
                                mute=first)
    keep = t[None, None, :] >= first[:, :, None]
    np.testing.assert_allclose(X1[keep], (-(1 + 0.5) * 1e-3 * g)[keep], rtol=1e-13, atol=1e-16)


def test_tier_b_with_precomputed_kernel_spectrum():
    D = synth.random_traces((9, 5, 40), 61)
    X = synth.random_traces((4, 5, 40), 62)
    R = synth.random_traces((3, 4, 40), 63)
    idx = np.array([7, 2, 2])
    Dh = oracle.kernel_spectrum(D)
    np.testing.assert_array_equal(oracle.mdc_forward_fft(D, X, idx, Dh=Dh), oracle.mdc_forward_fft(D, X, idx))
    np.testing.assert_array_equal(oracle.mdc_adjoint_fft(D, R, idx, Dh=Dh), oracle.mdc_adjoint_fft(D, R, idx))


# ------------------------------------------------------------------------------------------------
# LSQR (Paige & Saunders), the full-gradient baseline
# ------------------------------------------------------------------------------------------------
def test_lsqr_matches_scipy_iterates():
    from scipy.sparse.linalg import lsqr as scipy_lsqr
    rng = np.random.default_rng(71)
    A = rng.standard_normal((30, 12)) @ np.diag(np.linspace(3, 0.2, 12))
    b = rng.standard_normal(30)
    for k in (1, 3, 7, 10, 20):   # (k = 12 = n ends the Krylov space: both are then ill-conditioned in beta ~ 0)
        x, norms = oracle.lsqr(lambda z: A @ z, lambda r: A.T @ r, b, np.zeros(12), k)
        xs = scipy_lsqr(A, b, atol=0, btol=0, conlim=0, iter_lim=k)[0]
        np.testing.assert_allclose(x, xs, rtol=1e-10, atol=1e-12)
        assert abs(norms[-1] - np.linalg.norm(b - A @ x)) <= 1e-9 * np.linalg.norm(b)


def test_lsqr_on_mdc_reaches_least_squares_and_keeps_preconditioned_range():
    nt, n, ns = 8, 2, 3
    D = synth.random_traces((ns, n, nt), 81)
    U = synth.random_traces((ns, n, nt), 82)
    nx = n * n * nt
    A = np.zeros((ns * n * nt, nx))
    for j in range(nx):
        e = np.zeros(nx)
        e[j] = 1.0
        A[:, j] = oracle.mdc_forward(D, e.reshape(n, n, nt), np.arange(ns)).ravel()
    X, norms = oracle.mdc_lsqr(D, np.zeros((n, n, nt)), U, nx + 5)
    x_ls = np.linalg.lstsq(A, U.ravel(), rcond=None)[0]
    assert np.linalg.norm(A @ X.ravel() - U.ravel()) <= (1 + 1e-8) * np.linalg.norm(A @ x_ls - U.ravel())
    assert all(b <= a * (1 + 1e-12) for a, b in zip(norms, norms[1:]))     # monotone residual estimates
    Xr, _ = oracle.mdc_lsqr(D, np.zeros((n, n, nt)), U, 6, recip=True)
    np.testing.assert_allclose(Xr, np.transpose(Xr, (1, 0, 2)), rtol=0, atol=1e-12)


def test_band_limited_operator_is_direct_sums_with_lowpassed_kernel():
    """Zeroing the products above bin `band` equals the direct sums (Tier A) with the down-going field
    passed through the ideal low-pass filter of the same FFT length (a separate route to the same operator)."""
    nt, nr, nv, ns, band = 40, 4, 3, 5, 17
    D = synth.random_traces((ns, nr, nt), 91)
    X = synth.random_traces((nv, nr, nt), 92)
    R = synth.random_traces((3, nv, nt), 93)
    idx = np.array([4, 0, 2])
    nfft = oracle.default_nfft(nt)
    Dh = np.fft.rfft(D, n=nfft, axis=-1)
    Dh[..., band:] = 0.0
    Dlp = np.fft.irfft(Dh, n=nfft, axis=-1)          # the filtered kernel, full length nfft
    # direct sums with a kernel of length nfft: the causal sum only needs tau < nt, but the filtered
    # kernel is not causal-limited, so wrap the tail (tau in [nt, nfft)) as the circular product does
    U = np.zeros((3, nv, nt))
    G = np.zeros((nv, nr, nt))
    for b, s in enumerate(idx):
        for v in range(nv):
            for r in range(nr):
                for t in range(nt):
                    U[b, v, t] += sum(Dlp[s, r, (t - k) % nfft] * X[v, r, k] for k in range(nt))
                    G[v, r, t] += sum(Dlp[s, r, (k - t) % nfft] * R[b, v, k] for k in range(nt))
    np.testing.assert_allclose(oracle.mdc_forward_fft(D, X, idx, band=band), U, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(oracle.mdc_adjoint_fft(D, R, idx, band=band), G, rtol=1e-10, atol=1e-10)
    np.testing.assert_array_equal(oracle.mdc_forward_fft(D, X, idx, band=nfft // 2 + 1), oracle.mdc_forward_fft(D, X, idx))

"""Parity oracle for stochastic multi-dimensional deconvolution (arXiv 2202.04486).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct FP64 CPU code written from the paper, used
to check the CUDA path.  Only the tests, the smoke check and the benchmark's CPU-baseline / reference
leg may import it.  It imports nothing from the CUDA package and shares no code with it.

Tier A (the definition): direct time-domain convolution / cross-correlation sums in C
(oracle/mdc_direct.c), for the forward operator P+_t of Eq. 3 restricted to a batch of sources
(Eq. 5) and for its adjoint (the cross-correlation named in the Synthetic OBC section).

Tier B: the same operator through numpy's FP64 FFT (Appendix A: FFT along time, one matrix product per
frequency, inverse FFT), with zero padding to nfft >= 2 nt - 1 so that the circular convolution equals
the causal linear one on [0, nt).  It is pinned to Tier A in the tests and used only where Tier A is
too slow (multi-epoch trajectories).

Pins (tests/test_oracle_pins.py): the 1D case against numpy.convolve / numpy.correlate, a delta
down-going field, a dense operator built from scipy Toeplitz blocks, the adjoint dot-product test, the
finite-sum identity of Eq. 5/6, the Landweber toy of Eq. 11 (sigma^2 = 53.0256), the spectral bound on
the operator norm, SGD converging to the least-squares solution of a tiny consistent problem, and for
N-SGD: the equivalence of the look-ahead form with Sutskever's form, mu = 0 giving SGD, and convergence
to the minimum-norm least-squares solution; the causality mute against an explicit loop; LSQR against
scipy's implementation and the least-squares solution.

Readings of the paper taken here, where its text is silent or ambiguous:
  * scale: the receiver integral of Eq. 1 is a plain sum over receivers times `scale` (default 1).
  * gradient: g_B = P_B^H (P_B X - U_B), summed (not averaged) over the batch; the update is
    X <- X - alpha * C(g_B) (Eq. 6 with its leading minus folded into the residual).
  * reciprocity preconditioner C_r: 1/2 (G + G^T) with T swapping receiver and virtual source.
  * steps per epoch: ceil(ns / nb), the last batch partial.
  * RMSE (Eq. 7): plain L2 norm of the difference of the max-normalised fields.
  * N-SGD: Nesterov momentum in Sutskever's form, evaluated on the look-ahead point (nsgd_step).
  * causality preconditioner C_c: a per-trace first kept sample (the direct-arrival mute); with
    reciprocity the mute table is symmetric in (r, v).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        for name in ("oracle_mdc_forward", "oracle_mdc_adjoint"):
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [ctypes.c_int] * 4 + [dp, dp, ip, ctypes.c_int, ip, ctypes.c_int,
                                                ctypes.c_double, dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_num_threads.restype = None
        _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the direct sums use."""
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Set the OpenMP threads of the direct sums (timing only; the results do not depend on it)."""
    _load().oracle_set_num_threads(int(n))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


# ----------------------------------------------------------------------------------------------
# Tier A: direct sums
# ----------------------------------------------------------------------------------------------
def mdc_forward(D, X, idx, scale: float = 1.0, vsel=None) -> np.ndarray:
    """Forward MDC for the sources idx (Eq. 1-3 in the time domain, batch form of Eq. 5).

    U[b, j, t] = scale * sum_r sum_{tau<=t} D[idx[b], r, tau] * X[vsel[j], r, t - tau].
    D: (ns, nr, nt), X: (nv, nr, nt) -> U: (nb, len(vsel), nt).  vsel defaults to all virtual sources.
    """
    D, X = _f64(D), _f64(X)
    ns, nr, nt = D.shape
    nv = X.shape[0]
    assert X.shape == (nv, nr, nt)
    idx = _i32(idx)
    vsel = _i32(np.arange(nv) if vsel is None else vsel)
    U = np.zeros((idx.size, vsel.size, nt))
    rc = _load().oracle_mdc_forward(nt, nr, nv, ns, _ptr(D, ctypes.c_double), _ptr(X, ctypes.c_double),
                                    _ptr(idx, ctypes.c_int32), idx.size, _ptr(vsel, ctypes.c_int32),
                                    vsel.size, float(scale), _ptr(U, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_mdc_forward: invalid argument")
    return U


def mdc_adjoint(D, R, idx, scale: float = 1.0, vsel=None) -> np.ndarray:
    """Adjoint MDC: cross-correlation of the residual with the down-going field (Eq. 6).

    G[j, r, tau] = scale * sum_b sum_{t>=tau} D[idx[b], r, t - tau] * R[b, vsel[j], t].
    D: (ns, nr, nt), R: (nb, nv, nt) -> G: (len(vsel), nr, nt).
    """
    D, R = _f64(D), _f64(R)
    ns, nr, nt = D.shape
    nb, nv, _ = R.shape
    idx = _i32(idx)
    assert idx.size == nb and R.shape[2] == nt
    vsel = _i32(np.arange(nv) if vsel is None else vsel)
    G = np.zeros((vsel.size, nr, nt))
    rc = _load().oracle_mdc_adjoint(nt, nr, nv, ns, _ptr(D, ctypes.c_double), _ptr(R, ctypes.c_double),
                                    _ptr(idx, ctypes.c_int32), nb, _ptr(vsel, ctypes.c_int32),
                                    vsel.size, float(scale), _ptr(G, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_mdc_adjoint: invalid argument")
    return G


# ----------------------------------------------------------------------------------------------
# Tier B: the same operator through the FFT (Appendix A), numpy FP64
# ----------------------------------------------------------------------------------------------
def default_nfft(nt: int) -> int:
    """Smallest power of two >= 2 nt - 1 (linear, not circular, convolution on [0, nt))."""
    n = 1
    while n < 2 * nt - 1:
        n *= 2
    return n


def kernel_spectrum(D, nfft: int | None = None) -> np.ndarray:
    """rfft of every down-going trace, (ns, nr, nf): Appendix A transforms the kernel once."""
    D = _f64(D)
    return np.fft.rfft(D, n=nfft or default_nfft(D.shape[2]), axis=-1)


def mdc_forward_fft(D, X, idx, scale: float = 1.0, nfft: int | None = None, Dh=None, band: int | None = None) -> np.ndarray:
    """Tier B forward: rfft along time, per-frequency matrix product, irfft, keep t < nt.
    Dh: the kernel spectrum of D from kernel_spectrum (same nfft), or None to transform D[idx] here.
    band: only bins f < band take part in the products (the band-limited variant), None for all."""
    D, X = _f64(D), _f64(X)
    nt = D.shape[2]
    nfft = nfft or default_nfft(nt)
    assert nfft >= 2 * nt - 1
    Dh = np.fft.rfft(D[np.asarray(idx)], n=nfft, axis=-1) if Dh is None else Dh[np.asarray(idx)]   # (nb, nr, nf)
    Xh = np.fft.rfft(X, n=nfft, axis=-1)                            # (nv, nr, nf)
    Uh = np.matmul(Dh.transpose(2, 0, 1), Xh.transpose(2, 1, 0)).transpose(1, 2, 0)   # per f: [nb x nr][nr x nv]
    if band is not None:
        Uh[..., band:] = 0.0
    return scale * np.fft.irfft(Uh, n=nfft, axis=-1)[..., :nt]


def mdc_adjoint_fft(D, R, idx, scale: float = 1.0, nfft: int | None = None, Dh=None, band: int | None = None) -> np.ndarray:
    """Tier B adjoint: spectra of the residual times the conjugate down-going spectra, summed over the batch."""
    D, R = _f64(D), _f64(R)
    nt = D.shape[2]
    nfft = nfft or default_nfft(nt)
    assert nfft >= 2 * nt - 1
    Dh = np.fft.rfft(D[np.asarray(idx)], n=nfft, axis=-1) if Dh is None else Dh[np.asarray(idx)]   # (nb, nr, nf)
    Rh = np.fft.rfft(R, n=nfft, axis=-1)                            # (nb, nv, nf)
    Gh = np.matmul(Rh.transpose(2, 1, 0), np.conj(Dh).transpose(2, 0, 1)).transpose(1, 2, 0)  # per f: [nv x nb][nb x nr]
    if band is not None:
        Gh[..., band:] = 0.0
    return scale * np.fft.irfft(Gh, n=nfft, axis=-1)[..., :nt]


# ----------------------------------------------------------------------------------------------
# Stochastic MDD step (Eq. 5-6) and helpers
# ----------------------------------------------------------------------------------------------
def reciprocity(G) -> np.ndarray:
    """Reciprocity preconditioner C_r (Eq. 4): 1/2 (G + G^T), T swapping receiver and virtual source."""
    G = _f64(G)
    assert G.shape[0] == G.shape[1], "reciprocity needs nr == nv"
    return 0.5 * (G + G.transpose(1, 0, 2))


def loss(R) -> float:
    """1/2 ||R||^2 of the batch residual (the summand of Eq. 5 over the batch)."""
    R = _f64(R)
    return 0.5 * float(np.sum(R * R))


def gradient(D, X, U_obs, idx, scale: float = 1.0, fft: bool = False, Dh=None):
    """Mini-batch gradient of Eq. 6: g_B = P_B^H (P_B X - U_obs[idx]).  Returns (g, loss, residual).
    Dh (fft only): the precomputed kernel spectrum."""
    idx = np.asarray(idx)
    if fft:
        R = mdc_forward_fft(D, X, idx, scale, Dh=Dh) - _f64(U_obs)[idx]
        return mdc_adjoint_fft(D, R, idx, scale, Dh=Dh), loss(R), R
    R = mdc_forward(D, X, idx, scale) - _f64(U_obs)[idx]
    return mdc_adjoint(D, R, idx, scale), loss(R), R


def sgd_step(D, X, U_obs, idx, alpha: float, *, recip: bool = False, scale: float = 1.0,
             fft: bool = False, Dh=None):
    """One stochastic MDD step (SGD): X <- X - alpha * C(g_B), C = C_r or identity.  Returns (X_new, loss)."""
    g, l, _ = gradient(D, X, U_obs, idx, scale, fft, Dh)
    if recip:
        g = reciprocity(g)
    return _f64(X) - alpha * g, l


def run_epochs(D, X0, U_obs, batches, alpha: float, *, recip: bool = False, scale: float = 1.0,
               fft: bool = False):
    """Run the given epochs of batches (batches[epoch][step] -> source indices).  Returns (X, losses)."""
    X = _f64(X0).copy()
    losses = []
    Dh = kernel_spectrum(D) if fft else None
    for epoch in batches:
        for idx in epoch:
            X, l = sgd_step(D, X, U_obs, idx, alpha, recip=recip, scale=scale, fft=fft, Dh=Dh)
            losses.append(l)
    return X, losses


def causal_mute(G, first):
    """Causality preconditioner C_c (Eq. 4; the space-time mask of the Volve examples that mutes the
    reflection response above the direct arrival): samples t < first[v, r] of trace (v, r) set to zero.
    first: int array [nv, nr].  C_c is diagonal with 0/1 entries, so it is its own adjoint."""
    G = _f64(G).copy()
    first = np.asarray(first)
    t = np.arange(G.shape[-1])
    G[t[None, None, :] < first[:, :, None]] = 0.0
    return G


def precondition(g, *, recip: bool = False, mute=None):
    """C^T g for the chain C = C_r C_c of Eq. 4 (reciprocity and causality, either optional).  With a
    mute table symmetric in (r, v) the two commute and C_r C_c C_c^T C_r^T g = C_c C_r g: the model stays
    in the range of C when it starts there."""
    if recip:
        g = reciprocity(g)
    if mute is not None:
        g = causal_mute(g, mute)
    return g


def nsgd_step(D, X, V, U_obs, idx, alpha: float, mu: float, *, recip: bool = False, mute=None,
              scale: float = 1.0, fft: bool = False):
    """One step of SGD with Nesterov momentum (the N-SGD solver; momentum after Sutskever et al. 2013),
    written on the look-ahead point.  Sutskever's form is
        v' = mu v - alpha grad f(x + mu v),   x' = x + v';
    with y = x + mu v (the point where the gradient is taken) it becomes
        v' = mu v - alpha grad f(y),          y' = y + mu v' - alpha grad f(y),
    and X here is y.  grad f is the preconditioned mini-batch gradient C^T g_B of Eq. 6.
    Returns (X_new, V_new, loss)."""
    g, l, _ = gradient(D, X, U_obs, idx, scale, fft)
    g = precondition(g, recip=recip, mute=mute)
    V_new = mu * _f64(V) - alpha * g
    X_new = _f64(X) + mu * V_new - alpha * g
    return X_new, V_new, l


def adam_step(D, X, M, V, U_obs, idx, alpha: float, t: int, *, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8, recip: bool = False, mute=None, scale: float = 1.0, fft: bool = False):
    """One step of Adam (Kingma & Ba 2015, Algorithm 1) on the preconditioned mini-batch gradient
    C^T g_B of Eq. 6 (the paper's solvers are SGD and N-SGD; Adam is the other update asked of the fused
    kernel).  With t >= 1 the step count:
        m <- beta1 m + (1 - beta1) g,      v <- beta2 v + (1 - beta2) g^2          (biased moments)
        m_hat = m / (1 - beta1^t),         v_hat = v / (1 - beta2^t)               (bias corrections)
        x <- x - alpha m_hat / (sqrt(v_hat) + eps)                                  (element-wise)
    Returns (X_new, M_new, V_new, loss)."""
    assert t >= 1
    g, l, _ = gradient(D, X, U_obs, idx, scale, fft)
    g = precondition(g, recip=recip, mute=mute)
    M_new = beta1 * _f64(M) + (1.0 - beta1) * g
    V_new = beta2 * _f64(V) + (1.0 - beta2) * g * g
    m_hat = M_new / (1.0 - beta1 ** t)
    v_hat = V_new / (1.0 - beta2 ** t)
    X_new = _f64(X) - alpha * m_hat / (np.sqrt(v_hat) + eps)
    return X_new, M_new, V_new, l


def lsqr(apply_A, apply_At, b, x0, n_iter: int):
    """LSQR (Paige & Saunders 1982, the bidiagonalisation algorithm of their Section 4) for
    min ||A x - b||, the full-gradient MDD solver the paper compares against.  apply_A / apply_At are
    the operator and its adjoint on arrays of the shapes of x and b.  Starts from x0 (the iteration
    solves for the correction).  Returns (x, residual-norm estimates phi_bar_1 .. phi_bar_{n+1})."""
    x = _f64(x0).copy()
    u = _f64(b) - apply_A(x)
    beta = np.linalg.norm(u)
    u = u / beta if beta > 0 else u
    v = apply_At(u)
    alpha = np.linalg.norm(v)
    v = v / alpha if alpha > 0 else v
    w = v.copy()
    phi_bar, rho_bar = beta, alpha
    norms = [phi_bar]
    for _ in range(n_iter):
        # continue the bidiagonalisation
        u = apply_A(v) - alpha * u
        beta = np.linalg.norm(u)
        if beta > 0:
            u = u / beta
        v = apply_At(u) - beta * v
        alpha = np.linalg.norm(v)
        if alpha > 0:
            v = v / alpha
        # plane rotation eliminating the subdiagonal beta
        rho = np.hypot(rho_bar, beta)
        c, s = rho_bar / rho, beta / rho
        theta = s * alpha
        rho_bar = -c * alpha
        phi = c * phi_bar
        phi_bar = s * phi_bar
        # solution and search direction
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        norms.append(phi_bar)
    return x, norms


def mdc_lsqr(D, X0, U_obs, n_iter: int, *, recip: bool = False, mute=None, scale: float = 1.0):
    """Full-gradient MDD by LSQR on the preconditioned operator P C (Eq. 3-4): every source at once,
    x = C z with z from LSQR on A = P C, C = C_r C_c (each optional); the operator through Tier B.
    X0 must lie in the range of C (e.g. zero).  Returns (X, residual-norm estimates)."""
    D = _f64(D)
    ns = D.shape[0]
    idx = np.arange(ns)
    Dh = kernel_spectrum(D)
    fwd = lambda X: mdc_forward_fft(D, X, idx, scale, Dh=Dh)
    adj = lambda R: precondition(mdc_adjoint_fft(D, R, idx, scale, Dh=Dh), recip=recip, mute=mute)
    return lsqr(fwd, adj, _f64(U_obs), X0, n_iter)


def steps_per_epoch(ns: int, nb: int) -> int:
    """Number of batches in one epoch: ceil(ns / nb) (the last batch is partial)."""
    return -(-ns // nb)


def sigma2_max(D, nfft: int | None = None, scale: float = 1.0) -> float:
    """Largest squared singular value of the kernel over frequencies (Appendix B):
    max_f lambda_max(Dh_f^H Dh_f), Dh_f = unnormalised DFT of D along time at bin f, as an ns x nr matrix.
    This bounds sigma^2 of the time-domain operator from above (it is the norm of its circulant embedding)."""
    D = _f64(D)
    nt = D.shape[2]
    nfft = nfft or default_nfft(nt)
    Dh = np.fft.rfft(D, n=nfft, axis=-1)                            # (ns, nr, nf)
    s = np.linalg.svd(np.moveaxis(Dh, -1, 0), compute_uv=False)     # (nf, min(ns,nr))
    return float(scale * scale * np.max(s[:, 0] ** 2))


def landweber(A, y, alpha: float, n_iter: int, x0=None) -> np.ndarray:
    """Landweber iteration x <- x + alpha A^T (y - A x) on a dense matrix (Appendix B, Eq. 11).
    Returns the iterates, shape (n_iter + 1, n)."""
    A, y = _f64(A), _f64(y)
    x = np.zeros(A.shape[1]) if x0 is None else _f64(x0).copy()
    out = [x.copy()]
    for _ in range(n_iter):
        x = x + alpha * (A.T @ (y - A @ x))
        out.append(x.copy())
    return np.array(out)


def rmse(x_true, x_est) -> float:
    """Eq. 7 as read here: || x_true / max|x_true| - x_est / max|x_est| ||_2 (plain L2 norm)."""
    a, b = _f64(x_true), _f64(x_est)
    return float(np.linalg.norm(a / np.max(np.abs(a)) - b / np.max(np.abs(b))))


def rel_l2(a, ref) -> float:
    """||a - ref|| / ||ref|| in FP64."""
    a, ref = _f64(a), _f64(ref)
    return float(np.linalg.norm(a - ref) / max(np.linalg.norm(ref), 1e-300))

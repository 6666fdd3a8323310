"""Seeded synthetic inputs for stochastic MDD (shared by the CUDA path's tests/bench and the oracle's tests).

This module only *draws* data: it holds none of the arithmetic of the method (no convolution, no
FFT, no gradient).  Every random number the method consumes (source permutations, dot-test vectors,
noise) is produced here and passed in as an input to both sides.

The paper's datasets (finite-difference OBC modelling, SRM-redatumed subsalt fields, Volve) are not
available, so these generators stand in for them with the same geometry template: receivers, virtual
sources and sources on one line with constant spacing, a Ricker wavelet with a 20 Hz peak frequency
(Synthetic OBC example), a down-going field made of a direct arrival plus free-surface multiples, and
a reflection response made of hyperbolic events.  The reflection response is symmetric in
(receiver, virtual source), so source-receiver reciprocity (the preconditioner C_r of Eq. 4) holds
exactly.

Array conventions (time axis fastest, float64 here; callers cast):
  D[s, r, t]  down-going wavefield p+ at receiver r for source s          (ns, nr, nt)
  X[v, r, t]  reflection response R(x_r, x_v) (the unknown r_t of Eq. 3)    (nv, nr, nt)
  U[s, v, t]  up-going wavefield p- at virtual source v for source s       (ns, nv, nt)
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DT = 0.004          # 4 ms sampling
F0 = 20.0           # Ricker peak frequency (Hz), as in the Synthetic OBC example
WATER_V = 1500.0    # velocity of the direct arrival and of the multiples (m/s)
T_DIRECT = 0.06     # zero-offset time of the direct arrival (s)


def ricker(t: np.ndarray, f0: float = F0) -> np.ndarray:
    """Zero-phase Ricker wavelet (1 - 2 pi^2 f0^2 t^2) exp(-pi^2 f0^2 t^2)."""
    a = (math.pi * f0 * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


@dataclasses.dataclass
class Problem:
    nt: int
    nr: int
    nv: int
    ns: int
    dt: float
    dx: float
    D: np.ndarray          # (ns, nr, nt) float64
    X_true: np.ndarray     # (nv, nr, nt) float64
    noise: np.ndarray      # (ns, nv, nt) float64 standard normal draws (caller scales them)


def make_problem(nt: int, nr: int, nv: int, ns: int, *, dx: float = 20.0, dt: float = DT,
                 n_reflectors: int = 3, n_multiples: int = 2, seed: int = 0) -> Problem:
    """Ricker/hyperbola generator.

    X_true(v, r, t) = sum_k a_k w(t - sqrt(t0_k^2 + ((x_r - x_v)/vel_k)^2)),
        vel_k ~ U(1500, 2500) m/s, a_k ~ U(0.2, 1), t0_k ~ U(0.15, 0.85) * nt * dt.
    D(s, r, t) = w(t - sqrt(td^2 + (h/1500)^2)) + sum_{m=1..M} (-0.5)^m w(t - sqrt((td + m*Delta)^2 + (h/1500)^2)),
        td = 0.06 s, Delta = 0.2 * nt * dt, h = x_s - x_r.
    Virtual sources sit on the first nv receiver positions, so X_true is symmetric when nr == nv.
    """
    rng = np.random.default_rng(seed)
    t = np.arange(nt) * dt
    xr = np.arange(nr) * dx
    xv = np.arange(nv) * dx
    xs = np.arange(ns) * dx

    vel = rng.uniform(1500.0, 2500.0, n_reflectors)
    amp = rng.uniform(0.2, 1.0, n_reflectors)
    t0 = rng.uniform(0.15, 0.85, n_reflectors) * nt * dt
    off_vr = xr[None, :] - xv[:, None]                          # (nv, nr)
    X = np.zeros((nv, nr, nt))
    for k in range(n_reflectors):
        tk = np.sqrt(t0[k] ** 2 + (off_vr / vel[k]) ** 2)       # (nv, nr)
        X += amp[k] * ricker(t[None, None, :] - tk[:, :, None])

    delta = 0.2 * nt * dt
    off_sr = xs[:, None] - xr[None, :]                          # (ns, nr)
    D = np.zeros((ns, nr, nt))
    for m in range(n_multiples + 1):
        tm = np.sqrt((T_DIRECT + m * delta) ** 2 + (off_sr / WATER_V) ** 2)
        D += (-0.5) ** m * ricker(t[None, None, :] - tm[:, :, None])

    noise = rng.standard_normal((ns, nv, nt))
    return Problem(nt, nr, nv, ns, dt, dx, D, X, noise)


def make_problem_device(nt: int, nr: int, nv: int, ns: int, *, dx: float = 20.0, dt: float = DT,
                        n_reflectors: int = 3, n_multiples: int = 2, seed: int = 0, device=None,
                        chunk: int = 64):
    """make_problem for sizes too large for host-side float64 generation: the same formulas and the
    same random draws (the reflector parameters come from the same numpy generator, in the same
    order), evaluated with torch in float64 on `device`, chunk sources / virtual sources at a time,
    and returned as float32 tensors (D, X_true).  No noise is drawn."""
    import torch

    rng = np.random.default_rng(seed)
    vel = rng.uniform(1500.0, 2500.0, n_reflectors)
    amp = rng.uniform(0.2, 1.0, n_reflectors)
    t0 = rng.uniform(0.15, 0.85, n_reflectors) * nt * dt
    f64 = dict(device=device, dtype=torch.float64)
    t = torch.arange(nt, **f64) * dt
    xr = torch.arange(nr, **f64) * dx

    def ricker_t(x):
        a = (math.pi * F0 * x) ** 2
        return (1.0 - 2.0 * a) * torch.exp(-a)

    X = torch.empty((nv, nr, nt), device=device, dtype=torch.float32)
    for v0 in range(0, nv, chunk):
        xv = torch.arange(v0, min(nv, v0 + chunk), **f64) * dx
        off = xr[None, :] - xv[:, None]
        acc = torch.zeros((xv.numel(), nr, nt), **f64)
        for k in range(n_reflectors):
            tk = torch.sqrt(t0[k] ** 2 + (off / vel[k]) ** 2)
            acc += amp[k] * ricker_t(t[None, None, :] - tk[:, :, None])
        X[v0:v0 + xv.numel()] = acc.float()
    delta = 0.2 * nt * dt
    D = torch.empty((ns, nr, nt), device=device, dtype=torch.float32)
    for s0 in range(0, ns, chunk):
        xs = torch.arange(s0, min(ns, s0 + chunk), **f64) * dx
        off = xs[:, None] - xr[None, :]
        acc = torch.zeros((xs.numel(), nr, nt), **f64)
        for m in range(n_multiples + 1):
            tm = torch.sqrt((T_DIRECT + m * delta) ** 2 + (off / WATER_V) ** 2)
            acc += (-0.5) ** m * ricker_t(t[None, None, :] - tm[:, :, None])
        D[s0:s0 + xs.numel()] = acc.float()
    return D, X


def batch_members(n: int = 48, *, seed: int = 1000, nb: int = 32, largest=(1500, 1200, 1200, 1200)) -> list[dict]:
    """Shapes of a set of independent MDD problems of uneven sizes: n - 1 members with
    nr, nv ~ U[64, 600], ns ~ U[64, 800], nt in {256, 512, 1024, 1500} (member i drawn from seed + i and
    generated with that seed), plus one fixed largest member (nt, nr, nv, ns) = largest (None: none).
    Every member: batch nb, 20 m spacing, 8 reflectors, 4 multiple orders, no noise, reciprocity only
    where nr == nv."""
    out = []
    for i in range(n - (1 if largest else 0)):
        r = np.random.default_rng(seed + i)
        nt = int(r.choice([256, 512, 1024, 1500]))
        nr = int(r.integers(64, 601))
        nv = int(r.integers(64, 601))
        ns = int(r.integers(64, 801))
        out.append(dict(nt=nt, nr=nr, nv=nv, ns=ns, nb=nb, seed=seed + i))
    if largest:
        nt, nr, nv, ns = largest
        out.append(dict(nt=nt, nr=nr, nv=nv, ns=ns, nb=nb, seed=seed + n - 1))
    for m in out:
        m.update(dx=20.0, n_reflectors=8, n_multiples=4, reciprocity=m["nr"] == m["nv"])
    return out


def direct_arrival_mute(nr: int, nv: int, nt: int, *, dx: float = 20.0, dt: float = DT,
                        v_max: float = 2500.0, lead: float = 1.5 / F0) -> np.ndarray:
    """First kept sample of each reflection-response trace for the causality mute: the earliest
    hyperbola of the generator at offset h = |x_r - x_v| cannot arrive before h / v_max, and a Ricker
    wavelet starts about `lead` before its peak, so samples before (h / v_max - lead) / dt hold no
    signal.  Returns int32 [nv, nr]; symmetric in (r, v) on the shared positions."""
    h = np.abs(np.arange(nr)[None, :] - np.arange(nv)[:, None]) * dx
    first = np.floor((h / v_max - lead) / dt)
    return np.clip(first, 0, nt).astype(np.int32)


def epoch_batches(ns: int, nb: int, n_epochs: int, seed: int = 0) -> list[list[np.ndarray]]:
    """Source batches for n_epochs of stochastic MDD.

    Each epoch draws a fresh permutation of the ns sources (sampling without replacement) and splits it
    into ceil(ns/nb) consecutive batches, the last one partial when nb does not divide ns.
    Returns batches[epoch][step] -> int32 array of source indices.
    """
    rng = np.random.default_rng(seed + 7919)
    out = []
    for _ in range(n_epochs):
        perm = rng.permutation(ns).astype(np.int32)
        out.append([perm[i:i + nb] for i in range(0, ns, nb)])
    return out


def random_traces(shape, seed: int) -> np.ndarray:
    """Standard-normal float64 array (dot-test vectors, random models and residuals)."""
    return np.random.default_rng(seed).standard_normal(shape)


def random_indices(ns: int, nb: int, seed: int, replace: bool = False) -> np.ndarray:
    """nb source indices in [0, ns) as int32 (with replacement: duplicates allowed)."""
    rng = np.random.default_rng(seed)
    if replace:
        return rng.integers(0, ns, nb).astype(np.int32)
    return rng.permutation(ns)[:nb].astype(np.int32)


# Workload shapes (nt, nr, nv, ns, nb, dx, reflectors, multiples, noise fraction, reciprocity).
# Entries without nr / nv / ns use n for all three.
WORKLOADS = {
    "smdd_nt128_n32_nb8": dict(nt=128, nr=32, nv=32, ns=32, nb=8, dx=10.0, n_reflectors=3,
                               n_multiples=2, noise=0.0, reciprocity=False),
    "smdd_nt512_n201_nb16_recip": dict(nt=512, nr=201, nv=201, ns=201, nb=16, dx=20.0, n_reflectors=8,
                                       n_multiples=4, noise=0.05, reciprocity=True),
    "smdd_nt512_n256_nb16_recip": dict(nt=512, nr=256, nv=256, ns=256, nb=16, dx=20.0, n_reflectors=8,
                                       n_multiples=4, noise=0.0, reciprocity=True),
    "smdd_nt1024_n301_ns401_nb32": dict(nt=1024, nr=301, nv=301, ns=401, nb=32, dx=20.0, n_reflectors=8,
                                        n_multiples=4, noise=0.0, reciprocity=False),
    "smdd_nt1024_n301_ns401_nb64": dict(nt=1024, nr=301, nv=301, ns=401, nb=64, dx=20.0, n_reflectors=8,
                                        n_multiples=4, noise=0.0, reciprocity=False),
    # one virtual source on a Volve-like line of 180 receivers and 110 sources (single-virtual-source MDD)
    "smdd_nt1024_nr180_nv1_ns110_nb16": dict(nt=1024, nr=180, nv=1, ns=110, nb=16, dx=25.0, n_reflectors=8,
                                             n_multiples=4, noise=0.05, reciprocity=False),
}

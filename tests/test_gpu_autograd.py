"""Differentiable MDC (torch.autograd.Function over the C ABI): backward = the hand-written adjoint.

Checks: the autograd gradient of 1/2||MDC(C_r X) - U||^2 against the FP64 oracle's chain rule
C_r P^H (P C_r X - U); the dot-product identity through autograd; and, at the 256^3, nt = 512 size,
central finite differences (h = 1e-3) of the data term along 64 seeded random directions, with the
first-difference L1 regulariser composed by torch.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_04486_gb300 import autograd, binding, build, synth

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


def test_autograd_gradient_matches_oracle_chain_rule():
    nt, n, ns, nb = 128, 24, 30, 8
    D = _f32(synth.random_traces((ns, n, nt), 1))
    X = _f32(synth.random_traces((n, n, nt), 2))
    U = _f32(synth.random_traces((ns, n, nt), 3))
    idx = synth.random_indices(ns, nb, 4)
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb)
    Xg = _cuda(X).requires_grad_(True)
    Ub = _cuda(U[idx])
    loss = 0.5 * (autograd.mdc(autograd.reciprocity(Xg), plan, _cuda(idx, torch.int32)) - Ub).double().pow(2).sum()
    loss.backward()
    Xs = oracle.reciprocity(X)
    R = oracle.mdc_forward(D, Xs, idx) - U[idx]
    g_ref = oracle.reciprocity(oracle.mdc_adjoint(D, R, idx))
    assert oracle.rel_l2(Xg.grad.double().cpu().numpy(), g_ref) <= 1e-5
    assert abs(loss.item() - oracle.loss(R)) <= 1e-5 * oracle.loss(R)


def test_autograd_dot_product():
    nt, nr, nv, ns, nb = 100, 17, 13, 21, 5
    D = _cuda(synth.random_traces((ns, nr, nt), 11))
    X = _cuda(synth.random_traces((nv, nr, nt), 12)).requires_grad_(True)
    Y = _cuda(synth.random_traces((nb, nv, nt), 13))
    idx = _cuda(synth.random_indices(ns, nb, 14), torch.int32)
    plan = binding.MDCPlan(D, nv, nb_max=nb)
    U = autograd.mdc(X, plan, idx)
    (U.double() * Y.double()).sum().backward()
    G = plan.adjoint(Y, idx)
    torch.testing.assert_close(X.grad, G, rtol=0, atol=0)     # the backward is the adjoint kernel itself
    lhs = (U.detach().double() * Y.double()).sum().item()
    rhs = (X.detach().double() * G.double()).sum().item()
    assert abs(lhs - rhs) <= 1e-5 * U.detach().double().norm().item() * Y.double().norm().item()


def test_finite_differences_full_size():
    """Loss ||MDC(C_r X) - U||^2 + 1e-3 ||d_x X||_1 at nt = 512, nr = nv = ns = 256, batch 16."""
    nt, n, nb, lam, h = 512, 256, 16, 1e-3, 1e-3
    p = synth.make_problem(nt, n, n, n, dx=20.0, n_reflectors=8, n_multiples=4, seed=0)
    D = _cuda(p.D)
    U_obs = _cuda(0.5 * synth.random_traces((n, n, nt), 21))
    idx = _cuda(synth.epoch_batches(n, nb, 1, seed=0)[0][0], torch.int32)
    plan = binding.MDCPlan(D, n, nb_max=nb)
    Ub = U_obs[idx.long()]
    X0 = _cuda(0.3 * p.X_true)

    def data_term(X):
        return (autograd.mdc(autograd.reciprocity(X), plan, idx) - Ub).double().pow(2).sum()

    def reg_term(X):
        return lam * (X[:, 1:, :] - X[:, :-1, :]).double().abs().sum()

    X = X0.clone().requires_grad_(True)
    data_term(X).backward()
    g_data = X.grad.detach().double().clone()
    X.grad = None
    reg_term(X).backward()
    g_reg = X.grad.detach().double().clone()
    # the regulariser's gradient composed by torch: -sign(d) at r, +sign(d) at r+1
    d = torch.sign((X0[:, 1:, :] - X0[:, :-1, :]).double())
    ref = torch.zeros_like(g_reg)
    ref[:, 1:, :] += lam * d
    ref[:, :-1, :] -= lam * d
    torch.testing.assert_close(g_reg, ref, rtol=0, atol=1e-9)   # the gradient reaches X in float32

    # central differences of the data term: (L(X+hE) - L(X-hE)) / 2h, with the difference of squares
    # evaluated as <r+ + r-, r+ - r-> so that it is not lost to the rounding of L itself
    def residual(X):
        return (autograd.mdc(autograd.reciprocity(X), plan, idx) - Ub).double()

    # Both sides are inner products of FP32 operator outputs with random dense vectors, whose value is
    # ~1/sqrt(N) of the product of the norms; FP32 rounding therefore bounds the agreement relative to
    # that product (as in the dot-product test), at the FP32 tolerance 1e-5.
    gen = torch.Generator(device="cuda").manual_seed(123)
    worst = 0.0
    with torch.no_grad():
        for k in range(64):
            E = torch.randn(X0.shape, device="cuda", generator=gen)
            rp, rm = residual(X0 + h * E), residual(X0 - h * E)
            fd = ((rp + rm) * (rp - rm)).sum().item() / (2 * h)
            ad = (g_data * E.double()).sum().item()
            scale = (rp + rm).norm().item() * ((rp - rm) / (2 * h)).norm().item()
            worst = max(worst, abs(fd - ad) / scale)
    assert worst <= 1e-5, worst

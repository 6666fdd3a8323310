"""Parity at the full size of the largest member of the many-problem workload: nt = 1500, nr = nv = ns = 1200,
batch 32 (the member that dominates that workload's epoch), against the oracle's direct FP64 sums.

Without reciprocity the MDC is separable in the virtual source (U[:, v] depends only on X[v], G[v] only on
R[:, v]), so a few sampled columns of the forward output and of one SGD step are checked exactly, at the
oracle cost of a few columns.  Both precisions: FP32 (relative L2 <= 1e-5 on U and on the stepped model,
1e-4 on the gradient read back through the step) and split BF16 (1e-4 on U, 1e-3 on the gradient).  The
observed rows are seeded random traces passed already gathered (SMDD_UOBS_GATHERED); the step size comes
from the oracle's gradient (it moves the model by a tenth of its peak).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_04486_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu

NT, N, NB = 1500, 1200, 32
VSEL = np.array([0, 611, 1199])


@pytest.fixture(scope="module")
def problem():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    binding.load_library()
    D, Xt = synth.make_problem_device(NT, N, N, N, dx=20.0, n_reflectors=8, n_multiples=4, seed=1047, device="cuda")
    X0 = 0.5 * Xt
    del Xt
    idx = synth.random_indices(N, NB, 3)
    Uobs = synth.random_traces((NB, N, NT), 4).astype(np.float32)
    Dr = D[torch.from_numpy(idx).long().cuda()].double().cpu().numpy()      # the batch rows, (NB, N, NT)
    Xs = X0[torch.from_numpy(VSEL).long().cuda()].double().cpu().numpy()     # the sampled model columns
    bidx = np.arange(NB)
    U_ref = oracle.mdc_forward(Dr, Xs, bidx)                                 # (NB, len(VSEL), NT)
    G_ref = oracle.mdc_adjoint(Dr, U_ref - Uobs[:, VSEL].astype(np.float64), bidx)
    alpha = 0.1 * np.abs(Xs).max() / np.abs(G_ref).max()
    return dict(D=D, X0=X0, idx=idx, Uobs=Uobs, Xs=Xs, U_ref=U_ref, G_ref=G_ref, alpha=float(np.float32(alpha)))


def _rel(a, b):
    return oracle.rel_l2(np.asarray(a, np.float64), b)


@pytest.mark.parametrize("precision,tol_u,tol_g", [(binding.MDC_PREC_FP32, 1e-5, 1e-4),
                                                   (binding.MDC_PREC_BF16X3, 1e-4, 1e-3)], ids=["fp32", "bf16x3"])
def test_largest_member_sampled_columns(problem, precision, tol_u, tol_g):
    pr = problem
    plan = binding.MDCPlan(pr["D"], N, nb_max=NB, precision=precision)
    ti = torch.from_numpy(pr["idx"]).cuda()
    vs = torch.from_numpy(VSEL).long().cuda()
    U = plan.forward(pr["X0"], ti)[:, vs].double().cpu().numpy()
    assert _rel(U, pr["U_ref"]) <= tol_u
    X = pr["X0"].clone()
    plan.step(X, torch.from_numpy(pr["Uobs"]).cuda(), ti, pr["alpha"], binding.SMDD_UOBS_GATHERED)
    assert plan.sync_status() == binding.MDC_OK
    X1 = X[vs].double().cpu().numpy()
    del X
    plan.close()
    X1_ref = pr["Xs"] - pr["alpha"] * pr["G_ref"]
    assert _rel(X1, X1_ref) <= tol_u
    G = (pr["Xs"] - X1) / pr["alpha"]
    assert _rel(G, pr["G_ref"]) <= tol_g
    torch.cuda.empty_cache()

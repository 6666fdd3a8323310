"""smdd_step_host: the SGD step with the batch taken from host memory through the plan's two staging
slots and copy stream.  It runs the same kernels on the same values as smdd_step with device inputs, so
the models and losses agree bit for bit over a pipelined sequence of steps (slots alternate, copies of
one call overlap the previous step); one step is also checked against the FP64 oracle (FP32 bar,
relative L2 <= 1e-5)."""
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


@pytest.mark.parametrize("recip,pinned", [(True, True), (False, True), (True, False)],
                         ids=["recip-pinned", "plain-pinned", "recip-pageable"])
def test_host_steps_equal_device_steps(recip, pinned):
    nt, n, ns, nb, steps = 200, 24, 30, 7, 6
    D = _f32(synth.random_traces((ns, n, nt), 1))
    U = _f32(synth.random_traces((ns, n, nt), 2))
    alpha = 0.3 / oracle.sigma2_max(D)
    batches = [synth.random_indices(ns, nb, 10 + k) for k in range(steps)]
    batches[2] = np.array([3, 4, 5, 6, 9, 10, 0], dtype=np.int32)      # runs of consecutive sources
    batches[4] = np.array([8, 8, 2, 2, 2, 29, 28], dtype=np.int32)     # duplicates
    flags = binding.SMDD_RECIPROCITY if recip else 0
    Ud = _cuda(U)
    U_host = torch.from_numpy(U.astype(np.float32))
    if pinned:
        U_host = U_host.pin_memory()
    plan_d = binding.MDCPlan(_cuda(D), n, nb_max=nb)
    plan_h = binding.MDCPlan(_cuda(D), n, nb_max=nb)
    Xd, Xh = torch.zeros((n, n, nt), device="cuda"), torch.zeros((n, n, nt), device="cuda")
    loss_d = torch.zeros(steps, device="cuda", dtype=torch.float64)
    loss_h = torch.zeros(steps, dtype=torch.float64)
    if pinned:
        loss_h = loss_h.pin_memory()
    for k, idx in enumerate(batches):
        fl = flags | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
        binding.smdd_step(plan_d.handle, Xd, Ud, _cuda(idx, torch.int32), alpha, fl, loss_d[k])
        binding.smdd_step_host(plan_h.handle, Xh, U_host, torch.from_numpy(idx.astype(np.int32)), alpha, fl,
                               loss_h[k:k + 1])
    torch.cuda.synchronize()
    assert plan_d.sync_status() == binding.MDC_OK and plan_h.sync_status() == binding.MDC_OK
    torch.testing.assert_close(Xh, Xd, rtol=0, atol=0)
    np.testing.assert_array_equal(loss_h.numpy(), loss_d.cpu().numpy())


def test_host_step_matches_oracle():
    nt, n, ns, nb = 128, 20, 25, 6
    p = synth.make_problem(nt, n, n, ns, dx=40.0, n_reflectors=3, n_multiples=2, seed=3)
    D = _f32(p.D)
    U = _f32(oracle.mdc_forward(D, _f32(p.X_true), np.arange(ns)))
    X = _f32(0.5 * oracle.reciprocity(synth.random_traces((n, n, nt), 4)))
    idx = synth.random_indices(ns, nb, 5)
    alpha = 0.4 / oracle.sigma2_max(D)
    plan = binding.MDCPlan(_cuda(D), n, nb_max=nb)
    Xg = _cuda(X)
    loss = torch.zeros(1, dtype=torch.float64).pin_memory()
    binding.smdd_step_host(plan.handle, Xg, torch.from_numpy(U.astype(np.float32)).pin_memory(),
                           torch.from_numpy(idx.astype(np.int32)), alpha, binding.SMDD_RECIPROCITY, loss)
    torch.cuda.synchronize()
    Xr, l_ref = oracle.sgd_step(D, X, U, idx, alpha, recip=True)
    assert plan.sync_status() == binding.MDC_OK
    assert oracle.rel_l2(Xg.double().cpu().numpy(), Xr) <= 1e-5
    assert abs(loss.item() - l_ref) <= 1e-5 * l_ref


def test_host_step_errors():
    nt, n, ns, nb = 32, 4, 5, 3
    D = _cuda(synth.random_traces((ns, n, nt), 1))
    plan = binding.MDCPlan(D, n, nb_max=nb)
    X = torch.ones((n, n, nt), device="cuda")
    U_host = torch.zeros((ns, n, nt))
    for idx, status in [([0, 5, 1], binding.MDC_ERR_INDEX_RANGE), ([0, -1, 1], binding.MDC_ERR_INDEX_RANGE),
                        ([0, 1, 2, 3], binding.MDC_ERR_SHAPE)]:
        with pytest.raises(binding.MDCError) as e:
            binding.smdd_step_host(plan.handle, X, U_host, torch.tensor(idx, dtype=torch.int32), 0.1)
        assert e.value.status == status
    with pytest.raises(binding.MDCError) as e:
        binding.smdd_step_host(plan.handle, X, U_host, torch.tensor([0, 1], dtype=torch.int32), 0.1,
                               binding.SMDD_UOBS_GATHERED)
    assert e.value.status == binding.MDC_ERR_INVALID_ARG
    with pytest.raises(TypeError):
        binding.smdd_step_host(plan.handle, X, U_host.cuda(), torch.tensor([0], dtype=torch.int32), 0.1)
    torch.cuda.synchronize()
    assert plan.sync_status() == binding.MDC_OK
    assert bool((X == 1).all())      # nothing ran

"""The seeded input generators: the device generator reproduces the host generator's draws and formulas,
and the batched member shapes follow their stated ranges."""
import numpy as np
import torch

from paper_2202_04486_gb300 import synth


def test_device_generator_matches_host_generator():
    p = synth.make_problem(50, 7, 5, 9, dx=20.0, n_reflectors=8, n_multiples=4, seed=3)
    D, X = synth.make_problem_device(50, 7, 5, 9, dx=20.0, n_reflectors=8, n_multiples=4, seed=3,
                                     device="cpu", chunk=4)
    assert D.dtype == torch.float32 and X.dtype == torch.float32
    np.testing.assert_allclose(D.numpy(), p.D.astype(np.float32), rtol=0, atol=1e-6)
    np.testing.assert_allclose(X.numpy(), p.X_true.astype(np.float32), rtol=0, atol=1e-6)


def test_batch_member_shapes():
    ms = synth.batch_members(48, seed=1000)
    assert len(ms) == 48
    for m in ms[:-1]:
        assert 64 <= m["nr"] <= 600 and 64 <= m["nv"] <= 600 and 64 <= m["ns"] <= 800
        assert m["nt"] in (256, 512, 1024, 1500) and m["nb"] == 32
        assert m["reciprocity"] == (m["nr"] == m["nv"])
    assert (ms[-1]["nt"], ms[-1]["nr"], ms[-1]["nv"], ms[-1]["ns"]) == (1500, 1200, 1200, 1200)
    assert len({m["seed"] for m in ms}) == 48
    assert synth.batch_members(48, seed=1000) == ms


def test_direct_arrival_mute_keeps_true_events():
    nt, n = 256, 40
    p = synth.make_problem(nt, n, n, n, dx=20.0, n_reflectors=8, n_multiples=4, seed=0)
    first = synth.direct_arrival_mute(n, n, nt, dx=20.0)
    assert first.dtype == np.int32 and first.shape == (n, n)
    np.testing.assert_array_equal(first, first.T)
    t = np.arange(nt)
    muted = t[None, None, :] < first[:, :, None]
    assert muted.any()
    assert np.max(np.abs(p.X_true[muted])) <= 1e-3 * np.max(np.abs(p.X_true))

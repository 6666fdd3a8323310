"""The multi-rank path of the benchmark on CPU: two gloo ranks, each an independent problem replica,
combine their timings (max over ranks) and work (sum over ranks); the reference arm runs on rank 0 only."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        times, flops = bench.combine_ranks([1.0 + rank, 5.0 - rank, 0.5], 10.0 * (rank + 1))
        out[rank] = (times, flops)
    finally:
        dist.destroy_process_group()


def test_combine_ranks_gloo_world_two():
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    for rank in range(2):
        times, flops = out[rank]
        assert times == [2.0, 5.0, 0.5]       # max over ranks, per entry
        assert flops == 30.0                  # sum over ranks


def test_combine_ranks_single_process_is_identity():
    import bench
    assert bench.combine_ranks([1.5, 2.5], 7.0) == ([1.5, 2.5], 7.0)


def test_reference_arm_other_ranks_do_nothing():
    import bench

    class A:
        steps, warmup, workload, batch_n, batch_largest = 3, 3, "smdd_nt512_n201_nb16_recip", 48, 1
    assert bench.run_reference(A(), rank=1, world=2, w=bench.workload_dims(A.workload)) is None
    assert bench.run_reference_batch(A(), rank=1, world=2) is None


def test_replicas_draw_independent_batches():
    from paper_2202_04486_gb300 import synth
    a = synth.epoch_batches(201, 16, 1, seed=0)[0]
    b = synth.epoch_batches(201, 16, 1, seed=1)[0]
    assert any((x != y).any() for x, y in zip(a, b))

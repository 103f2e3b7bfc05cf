"""The N > 1 benchmark path on CPU: two gloo ranks, each with its own batch of
the same shape (weak scaling by series), whole-job throughput over the slowest
rank.  No GPU and no data-path collective are involved: series are independent
(Sec. 2.1), so only the timing and the unit count are reduced."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, out_dir, workload):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        class A:
            pass
        args = A()
        # node32 draws per-series lengths in [2000, N]
        args.workload, args.B, args.N = workload, 4, (3000 if workload == "node32" else 300)
        w, g = bench.make_workload(args, rank)
        units = bench.real_steps(w)
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        value, max_ms = bench.job_throughput(units, 3, local_ms, world, dist)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), value=value, max_ms=max_ms,
                 units=units, y0=w["y0"], times_shape=np.array(w["times"].shape),
                 g_shape=np.array(g.shape))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("workload", ["vdp", "node32"])
def test_two_gloo_ranks_weak_scaling(tmp_path, workload):
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path), workload), nprocs=world,
                       join=True, start_method="spawn")
    r = [np.load(tmp_path / f"r{k}.npz") for k in range(world)]
    units = [int(x["units"]) for x in r]
    expect = sum(units) * 3 / (15.0 / 1e3)  # all ranks' real steps over the slowest rank
    for x in r:
        assert float(x["max_ms"]) == 15.0
        assert abs(float(x["value"]) - expect) <= 1e-9 * expect
    # each rank integrates its own batch of the same shape
    assert np.array_equal(r[0]["times_shape"], r[1]["times_shape"])
    assert np.array_equal(r[0]["g_shape"], r[1]["g_shape"])
    assert not np.array_equal(r[0]["y0"], r[1]["y0"])
    if workload == "node32":  # per-series random lengths: ranks count different real steps
        assert units[0] != units[1]

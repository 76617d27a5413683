"""The benchmark's multi-rank path on the CPU: two gloo ranks (world size 2) exchange their step
times through bench.max_over_ranks and meet at bench.barrier; the whole-job value is the work of
all ranks over the slowest rank's time; the reference arm runs on rank 0 only."""
import json
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        t_local = 10.0 + 5.0 * rank          # per-rank mean step time (ms)
        t_max = bench.max_over_ranks(t_local, world)
        bench.barrier(world)
        cells = 1.0e9                        # units one replica processes per step
        value = world * cells / (t_max / 1e3)
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"t_max": t_max, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r in res:
        assert r["t_max"] == 15.0                      # every rank sees the slowest rank's time
        assert r["value"] == pytest.approx(2 * 1.0e9 / 0.015)


def test_single_rank_helpers_are_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)  # no process group needed


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse

    import bench
    args = argparse.Namespace(workload="ls_n200_l1000", N=None, L=None, steps=1, warmup=0, cpu_seconds=1.0,
                              cpu_threads=1)
    assert bench.run_reference(args, 2, 1) is None   # another rank: no work, no output
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(capsys):
    # the oracle arm's JSON line on a small instance: the contract's keys, the oracle as the
    # baseline, no host-device copies
    import argparse

    import bench
    args = argparse.Namespace(workload="ls_n200_l1000", N=60, L=80, steps=1, warmup=0, cpu_seconds=1.0,
                              cpu_threads=1)
    bench.run_reference(args, 1, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["config"]["N"] == 60 and line["config"]["L"] == 80
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] == 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}

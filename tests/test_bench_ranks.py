"""Host logic of bench.py for several ranks (replicas only: every rank runs
the whole workload on its own GPU and no collective touches the data path),
checked on the CPU with the gloo backend and world size 2: the per-rank
maximum of the timings, the whole-job throughput from it, and that the
reference arm runs on rank 0 alone."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (r + 1) * 10 ms for 5 steps; the job's time is the slowest rank's
    total = bench.per_rank_max(10.0 * (rank + 1), dist, device="cpu")
    value = bench.weak_scaling_value(world, 1000, total / 5)
    dist.barrier()
    dist.destroy_process_group()
    with open(f"{out_path}.{rank}", "w") as f:
        json.dump({"total": total, "value": value}, f)


def test_per_rank_max_and_weak_scaling_gloo(tmp_path):
    import torch.multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "r")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        d = json.load(open(f"{out}.{r}"))
        assert d["total"] == 20.0
        # 2 replicas x 1000 cells per step at 4 ms per step
        assert abs(d["value"] - 2 * 1000 / 4e-3 / 1e6) < 1e-12


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""


def test_single_rank_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.per_rank_max(3.5) == 3.5
    assert bench.weak_scaling_value(1, 8388608, 0.5) == pytest.approx(16777.216)


def test_roofline_helpers():
    """The pieces of the bench line's roofline that need no GPU: the count of
    first-order cells (the order switch, alpha <= 10 eps, fluid cells only),
    the weighted algorithmic flops, the issue-rate ceiling, the FP64-pipe
    occupancy against the DFMA peak, and the per-launch record it reads."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_1806_04960_gb300 import cases
    c = cases.c1()
    fluid, first = bench.order_mix(c, c.q)
    assert fluid == int((c.solid == 0).sum())
    assert first == int(((c.solid == 0) & (c.q[3] <= 10 * c.eps)).sum()) and 0 < first < fluid
    q = c.q.copy()
    q[3][c.solid == 0] = 10 * c.eps            # the threshold itself is first order
    assert bench.order_mix(c, q)[1] == fluid
    ops, ops1 = {"flops": 600}, {"flops": 370}
    assert bench.cell_flops(ops, ops1, 100, 25.0) == 75 * 600 + 25 * 370
    # 608 M warp instructions at 152 SMs x 4 schedulers x 2000 MHz take 0.5 ms
    ic = bench.issue_ceiling(608e6, 1.0, 2000.0, sms=152)
    assert abs(ic["min_ms"] - 0.5) < 1e-12 and abs(ic["frac"] - 0.5) < 1e-12
    assert bench.issue_ceiling(None, 1.0, 2000.0) is None
    fp = bench.fp64_pipe(64e6, 2.0, 1.0)        # 64e6 warp inst in 2 ms vs 1 TFLOP/s / 64
    assert abs(fp["achieved_per_s"] - 32e9) < 1 and abs(fp["peak_per_s"] - 1e12 / 64) < 1
    assert abs(fp["frac"] - 32e9 / (1e12 / 64)) < 1e-12
    assert bench.fp64_pipe(None, 1.0, 1.0) is None
    rec = bench.recorded_profile()
    if rec:                                     # present while the kernel sources match the record
        assert {"f32", "f64", "f32_inst", "f64_inst", "f64_fp64inst"} <= set(rec)
        assert rec["f64"] < 65 * 4096 * 2048 and rec["f32"] < 33 * 4096 * 2048

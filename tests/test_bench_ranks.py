"""Multi-rank host logic of bench.py on CPU: world_size-2 gloo ranks.

The bench runs one independent replica per GPU (the step has no exchange
between ranks); the whole-job value is the units of all ranks over the slowest
rank's time, and the reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, ws: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=ws)
    try:
        # rank r processed (r + 1) * 1000 units in (r + 1) * 10 ms
        units, ms = (rank + 1) * 1000.0, (rank + 1) * 10.0
        v, ms_max = bench.job_throughput(units, ms, ws)
        mx = bench.max_over_ranks(float(rank), ws)
        sm = bench.sum_over_ranks(float(rank + 1), ws)
        bench.barrier(ws)
        q.put((rank, v, ms_max, mx, sm))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, ms_max, mx, sm in out:
        assert ms_max == 20.0                      # the slowest rank sets the time
        assert v == pytest.approx(3000.0 / 0.020)  # all ranks' units over it
        assert mx == 1.0 and sm == 3.0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    v, ms_max = bench.job_throughput(500.0, 4.0, 1)
    assert ms_max == 4.0 and v == pytest.approx(500.0 / 0.004)


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        steps, warmup, gpus = 1, 1, 2
    # rank 1 returns at once: no oracle run, nothing printed
    assert bench.run_reference(A, {"nx": 8, "nz": 8, "name": "x"}) == 0
    assert capsys.readouterr().out == ""


def test_wide_band_workload_puts_the_antenna_inside_the_wider_domain():
    """bench --filter-strides: the particle guard grows with the filter halo ((4 + 1) x 7 = 35 cells for
    S(1:2:4)), and the antenna, which emits only inside the particle domain, moves past it"""
    import oracle
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_1009_2727_gb300 import workloads as W
    w = W.shrink(W.stage_2d(), 128, 320)
    w["order"] = 3
    ww = bench.wide_band(w, [1, 2, 4], False)
    assert ww["filter_strides"] == [1, 2, 4] and w.get("filter_strides") is None
    o = oracle.Sim(ww)
    info = o.info()
    assert info["guard"] == 3 + 35 + 2
    zlo = info["gz_lo"] * info["dz"]
    assert ww["laser"]["z_antenna"] >= zlo + 4 * info["dz"] - 1e-12


def test_reference_arm_shortens_its_sample_to_the_wall_clock_bound(monkeypatch, capsys):
    """when one oracle step projects the run past the bound, the sample drops to fewer rows (>= 96)"""
    import json
    sys.path.insert(0, ROOT)
    import bench
    from paper_1009_2727_gb300 import workloads as W
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(bench, "REF_BUDGET_S", 1e-3)
    w = W.shrink(W.stage_2d(), 64, 256)
    w["name"] = "stage_2d_narrow"

    class A:
        steps, warmup, gpus = 1, 1, 1
    assert bench.run_reference(A, w) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert "bounded sample: 96 x 64 cells" in line["config"]["workload"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"

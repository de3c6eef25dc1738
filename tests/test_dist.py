"""Multi-rank bookkeeping of the benchmark on CPU (gloo, world size 2): every
rank solves its own replica, the timing is the slowest rank's, the value is the
whole job's, and the reference arm runs on rank 0 only (others exit without
work).  The solve itself has no exchange step, so nothing else crosses ranks."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    got = bench.dist_env()
    t_local = 1.5 + rank  # rank 1 is the slow one
    t_max = bench.max_over_ranks(t_local, ws)
    value = bench.job_throughput(ws, 1000.0, 4, t_max)
    args = type("A", (), {"warmup": 1, "steps": 1, "gpus": ws})()
    buf = io.StringIO()
    if rank != 0:
        with redirect_stdout(buf):
            bench.run_reference(args)  # rank != 0: returns at once, prints nothing
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"env": got, "t_max": t_max, "value": value, "ref_out": buf.getvalue()}, f)


def test_two_rank_timing_and_value(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert d["env"] == [2, r, r]
        assert d["t_max"] == 2.5  # the slowest rank's time on every rank
        assert d["value"] == pytest.approx(2 * 1000.0 * 4 / 2.5)
    assert res[1]["ref_out"] == ""


def test_single_rank_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_throughput(1, 10.0, 3, 2.0) == 15.0


def _failing_rank_main(rank, ws, port, out_dir):
    import datetime

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws,
                            timeout=datetime.timedelta(seconds=30))
    if rank == 1:
        os._exit(3)  # a replica that dies between steps, with nothing of it in flight
    try:
        bench.max_over_ranks(1.0, ws)
        outcome = "returned"
    except Exception as e:  # the surviving rank learns of it from its next collective
        outcome = "error: " + type(e).__name__
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(outcome)


def test_a_failed_rank_ends_the_others_collective(tmp_path):
    # host-side failure detection: the timing reduction of a rank whose peer has
    # died raises within the process-group timeout instead of waiting forever
    pytest.importorskip("torch")
    import multiprocessing as mp
    import time

    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_failing_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p.is_alive() for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert not any(alive)
    assert procs[1].exitcode == 3
    assert (tmp_path / "r0.txt").read_text().startswith("error")
    assert time.time() - t0 < 120

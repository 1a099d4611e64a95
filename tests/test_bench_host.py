"""Host logic of bench.py without a GPU: the whole-job numbers of a
multi-rank run (max over ranks, pairs of all ranks) through a real
world-size-2 process group on the gloo backend, the per-rank workload seeds
of the weak-scaling run, the reference arm's rank-0-only rule and the JSON
line it prints."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out_q):
    import torch
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)

    def reduce_max(vals):
        t = torch.tensor(vals, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return [float(v) for v in t]

    dev_ms, e2e_ms = times[rank]
    res = bench.combine(dev_ms, e2e_ms, pairs_rank=1000, steps=4, world=world,
                        reduce_max=reduce_max)
    dist.barrier()
    dist.destroy_process_group()
    out_q.put((rank, res))


def test_combine_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [(8.0, 10.0), (6.0, 12.0)]  # rank 0 slower on device, rank 1 end to end
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        res = got[r]
        assert res["dev_ms"] == 8.0 and res["e2e_ms"] == 12.0
        assert res["value"] == pytest.approx(1000 * 2 * 4 / 8e-3)
        assert res["e2e_value"] == pytest.approx(1000 * 2 * 4 / 12e-3)
        assert res["ms_per_step"] == pytest.approx(2.0)


def test_single_rank_combine_is_identity():
    res = bench.combine(5.0, 7.0, pairs_rank=10, steps=5, world=1, reduce_max=lambda v: v)
    assert res["value"] == pytest.approx(10 * 5 / 5e-3) and res["ms_per_step"] == 1.0


def test_rank_seeds_distinct():
    seeds = {bench.rank_seed(r) for r in range(8)}
    assert len(seeds) == 8 and bench.rank_seed(0) == 1000 + bench.WORKLOAD


def test_reference_arm_other_ranks_print_nothing(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, ref_pixels = 1, 0, 10

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A())
    assert buf.getvalue() == ""


def test_reference_arm_line(monkeypatch):
    """Rank 0 of the reference arm prints one JSON line with the contract's
    keys: the oracle's rate is the line's value, its cpu_baseline and its
    end-to-end figure (no host-device copies)."""
    import json

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class A:
        steps, warmup, ref_pixels = 2, 1, 16

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A())
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["unit"] == "pairs/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "16 random pixels" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == bench.WORKLOAD_NAME

"""The N > 1 host path of bench.py (replicas): two gloo ranks on the CPU run
the same rank plumbing the GPU run uses with NCCL, and the reference arm's
non-zero ranks exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import bench
    r = bench.Ranks(torch, backend="gloo", device="cpu")
    # rank-dependent step times and end-to-end rates: the job takes the slowest
    ms = 10.0 + 5.0 * rank
    e2e = 1e9 / (1 + rank)
    r.barrier()
    value, ms_max, e2e_job = r.aggregate(cells=1000, ms=ms, e2e_rate=e2e)
    q.put((rank, r.ws, value, ms_max, e2e_job))
    r.close()


def test_two_gloo_ranks_aggregate_like_the_replicas_run():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, value, ms_max, e2e in out:
        assert ws == 2
        assert ms_max == 15.0                         # the slowest rank's step time
        assert value == pytest.approx(2 * 1000 / 15e-3)   # all ranks' cells over it
        assert e2e == pytest.approx(2 * 0.5e9)        # twice the slowest rank's rate
    assert out[0][2:] == out[1][2:]                   # every rank holds the same figures


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import torch
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    r = bench.Ranks(torch, backend="gloo", device="cpu")
    assert r.ws == 1 and r.rank == 0
    value, ms_max, e2e = r.aggregate(cells=500, ms=2.0, e2e_rate=None)
    assert ms_max == 2.0 and value == pytest.approx(500 / 2e-3) and e2e is None
    r.close()


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle, on the host cores) prints one
    JSON line with the contract's keys, the impl tag, a cpu_baseline that
    describes the run and an e2e entry with no host-device traffic."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0

"""The bench's multi-rank path on CPU: two gloo ranks (world size 2).  The
path shards into independent replicas, so what has to hold is the host logic:
rendezvous on 127.0.0.1, max-over-ranks timing, disjoint sampling streams per
rank and step, and the reference arm printing one line from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE="2")
    r, local, ws, d = bench.dist_init()
    try:
        got = bench.max_over_ranks(0.25 + r, d)
        q.put((r, local, ws, got, bench.replica_stream(r, 3, 1000)))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_max_and_streams():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1]
    assert all(x[2] == 2 for x in res)
    assert all(x[3] == 1.25 for x in res)              # the max over both ranks
    seeds = {x[4][0] for x in res}
    assert len(seeds) == 2                             # independent Philox keys per rank


def test_replica_streams_do_not_overlap():
    S = 1000
    ranges = {}
    for rank in range(4):
        for step in range(5):
            seed, c0 = bench.replica_stream(rank, step, S)
            ranges.setdefault(seed, []).append((c0, c0 + S))
    assert len(ranges) == 4
    for rs in ranges.values():
        rs.sort()
        assert all(a[1] <= b[0] for a, b in zip(rs, rs[1:]))


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-budget", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    assert rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["value"] > 0 and rec["e2e"]["h2d_bytes_per_step"] == 0

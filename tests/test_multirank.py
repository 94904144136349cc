"""The benchmark's multi-rank path on the CPU (gloo, world size 2): the path
has no exchange step, so N ranks run independent replicas; what must hold is
the timing protocol — a barrier, the slowest rank's time (max over ranks)
and whole-job throughput = units of all ranks / that time — and that only
rank 0 prints (the reference arm: the other ranks exit at once)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR='127.0.0.1',
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_env()
    dist = bench.init_dist(w, 'gloo')
    bench.barrier(dist)
    slowest = bench.reduce_max(dist, float(rank + 1) * 1.5)  # rank r "took" 1.5 (r + 1) s
    value = bench.aggregate(1000, slowest, w)
    out.put((r, slowest, value))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_throughput():
    ctx = mp.get_context('spawn')
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    assert [r for r, _, _ in res] == [0, 1]
    for _, slowest, value in res:
        assert slowest == 3.0           # the slowest rank's time, seen by every rank
        assert value == 1000 * 2 / 3.0  # units of both ranks over that time


@pytest.mark.parametrize('rank', [0, 1])
def test_reference_arm_prints_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE='2', MASTER_ADDR='127.0.0.1',
               MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, 'bench.py', '--impl', 'reference', '--gpus', '2', '--workload', 'shear32',
                        '--steps', '1', '--warmup', '3'], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith('{')]
    if rank != 0:
        assert lines == []
        return
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d['impl'] == 'reference' and d['value'] > 0 and d['unit'] == 'MLUPS'
    assert d['e2e']['h2d_bytes_per_step'] == 0 and d['cpu_baseline']['kind'] == 'oracle'

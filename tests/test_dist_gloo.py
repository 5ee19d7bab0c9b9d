"""Multi-process host logic of the benchmark on CPU: two gloo ranks, each with
its own population (no data-path collective), max-over-ranks timing and a sum
of the work units; the reference arm prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import bench
    from workloads import CONFIGS, make_population

    class A:
        impl = "reference"
    r, w, local, pg = bench.dist_setup(A)
    assert (r, w) == (rank, world) and pg is not None
    # each rank owns an independent population (seed + rank)
    spec = CONFIGS["tiny"]["spec"]
    nodes, _ = make_population(spec, 8, seed=100 + r)
    E, V = bench.enabled_counts(nodes, make_population(spec, 8, seed=100 + r)[1])
    dev = torch.device("cpu")
    t_max = bench.allreduce_max(pg, float(10 + r), dev)
    units = bench.allreduce_sum(pg, float(E.sum()), dev)
    digest = float(np.nansum(nodes))
    all_digests = [None] * w
    torch.distributed.all_gather_object(all_digests, digest)
    pg.destroy_process_group()
    q.put((r, t_max, units, float(E.sum()), all_digests))


def test_two_gloo_ranks_weak_scaling_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (_, t0, u0, e0, d0), (_, t1, u1, e1, d1) = res
    assert t0 == t1 == 11.0                       # max over ranks
    assert u0 == u1 == e0 + e1                    # units of all ranks
    assert d0 == d1 and d0[0] != d0[1]            # independent populations


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--config", "tiny", "--steps", "1", "--warmup", "0", "--gpus", "2"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["unit"] == "conn-evals/s" and rec["value"] > 0
    assert rec["e2e"]["h2d_bytes_per_step"] == 0

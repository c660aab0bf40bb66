"""The N-GPU benchmark runs independent replicas (no data-path collective); its only cross-rank
operations are a barrier and the max-over-ranks of the timed interval.  Covered here with
world_size-2 gloo ranks on the CPU, each solving a small replica with the oracle."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import ncpgen
    import oracle
    cfg = bench.replica_config(ncpgen.GridConfig(6, 5, 1, seed=3), rank)
    p = ncpgen.make_problem(cfg)
    b = ncpgen.normals(p.n, 2)
    o = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker, amg_max_coarse=8)
    x, info = o.fgmres(b, rtol=1e-8)
    dist.barrier()
    t = bench.max_over_ranks(float(rank + 1), dist)
    out.put((rank, t, info["iterations"], float(x.sum())))
    dist.destroy_process_group()


def test_replicas_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]          # slowest replica on every rank
    assert res[0][2] == res[1][2] and res[0][3] == res[1][3]  # identical independent replicas

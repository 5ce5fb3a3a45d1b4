"""The multi-rank host logic of the benchmark on CPU (gloo, world size 2):
each rank runs its own problem (its seed offset by the rank), the job's time
is the maximum over the ranks after a barrier, and the whole-job throughput
counts every rank's nodes.  No GPU: the data path has no collective."""
import importlib.util
import os
import socket

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    b = _bench()
    r, w, _ = b.dist_setup(None)
    from paper_1803_07822_gb300 import inputs as I
    wl = I.dynamic_channel(n=(8, 12, 8), seed=2000 + r, n_modes=4, amp=0.05, t=500.0)
    b.barrier(w)
    ms_local = 10.0 + 5.0 * r  # rank 1 is the slower one
    ms = b.reduce_max(ms_local, w)
    out[r] = (r, w, ms, float(wl["chart"].J9[8].sum()), b.whole_job_mlups(w, 1000, 10, ms))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = [out[r] for r in range(2)]
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[2] == 15.0 for x in res)  # the maximum over the ranks, on every rank
    assert res[0][3] != res[1][3]  # independent problems: the deformation differs per rank
    assert np.isclose(res[0][4], 2 * 1000 * 10 / 15e-3 / 1e6)


def test_single_rank_needs_no_group():
    b = _bench()
    os.environ.pop("WORLD_SIZE", None)
    assert b.reduce_max(3.0, 1) == 3.0
    b.barrier(1)
    assert np.isclose(b.whole_job_mlups(1, 4194304, 10, 5.0), 4194304 * 10 / 5e-3 / 1e6)

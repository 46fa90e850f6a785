"""The multi-GPU bench path runs independent replicas: every rank solves its
own conformation and only the timing is combined (max of the step time,
sum of the integrals).  Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, _ = bench.dist_init("gloo")
    assert (r, w) == (rank, world)
    wl = bench.workload_for("cluster300_sp", rank)
    # rank r claims (r + 1) units in (r + 1) * 10 ms
    value, ms_max = bench.replica_throughput(float(rank + 1), 10.0 * (rank + 1), w, "cpu")
    bench.barrier(w)
    out[rank] = (wl.mol.natom, float(wl.mol.xyz[5, 0]), wl.basis.nbf, value, ms_max)
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_replicas():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    (n0, x0, nbf0, v0, t0), (n1, x1, nbf1, v1, t1) = out[0], out[1]
    assert n0 == n1 == 300                       # same size class
    assert x0 != x1                              # different conformations (seed offset by rank)
    assert abs(nbf0 - nbf1) <= 0.1 * nbf0
    assert t0 == t1 == 20.0                      # slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(3.0 / 20e-3)  # all ranks' units over it

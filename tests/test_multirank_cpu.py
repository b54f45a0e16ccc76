"""Multi-rank design checks on CPU (gloo, world size 2).

The LOVE pre-compute shards by training point: rank r holds points X_r, the
SKI product needs one all-reduce (sum) of the m-vector W v per MVM,
K_UU is applied redundantly on every rank, and every Lanczos dot product is a
local partial plus an all-reduce.  The test phase (predict / sample) shards
test points with the cache replicated and needs no collective.  This test
runs that sharded Lanczos with the FP64 oracle's building blocks on two gloo
ranks and checks it reproduces the single-process oracle; it also checks the
max-over-ranks timing reduction bench.py uses.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _allreduce(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _sharded_lanczos(ski_r, m, k, b_r, tau=1e-12):
    """CGS2 Lanczos (as in oracle.lanczos) on sharded n-vectors."""
    grid = ski_r.grid
    nr = b_r.shape[0]
    Q = np.zeros((k, nr))
    alpha, beta = [], []
    nb = np.sqrt(_allreduce(np.array([b_r @ b_r]))[0])
    Q[0] = b_r / nb
    for j in range(k):
        u = _allreduce(ski_r.W @ Q[j])                       # the one m-vector all-reduce
        v = ski_r.WT @ grid.kuu_matmul(u) + ski_r.noise * Q[j]
        Qj = Q[: j + 1]
        c = _allreduce(Qj @ v)
        alpha.append(c[j])
        v = v - Qj.T @ c
        c2 = _allreduce(Qj @ v)
        v = v - Qj.T @ c2
        bj = np.sqrt(_allreduce(np.array([v @ v]))[0])
        if j == k - 1:
            break
        if bj <= tau * np.max(np.abs(alpha)):
            break
        beta.append(bj)
        Q[j + 1] = v / bj
    return np.array(alpha), np.array(beta)


def _worker(rank, world, port, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
        from gpu_util import small_workload
        from oracle import grid as og
        from oracle import ski as os_
        wl = small_workload(dim=1, g=60, n=3000, k=25, t=200, dtype="f64", ls=0.12)
        x = wl.x_train()
        y = wl.y_train(x)
        grid = og.grid_from_workload(wl)
        sl = slice(rank * (wl.n // world), (rank + 1) * (wl.n // world) if rank < world - 1 else wl.n)
        ski_r = os_.SKI(grid, x[sl], wl.noise, y[sl])
        # probe b = (1/m) W^T K 1, sharded by rows
        b_r = (ski_r.WT @ grid.kuu_matmul(np.ones(grid.m))) / grid.m
        alpha, beta = _sharded_lanczos(ski_r, grid.m, wl.k, b_r)
        # bench.py's reduction: max over ranks
        t = torch.tensor([float(rank + 1)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            out_q.put((alpha, beta, float(t.item())))
    finally:
        dist.destroy_process_group()


def test_sharded_lanczos_matches_single_process():
    from gpu_util import small_workload
    from oracle import grid as og
    from oracle import lanczos as LZ
    from oracle import ski as os_
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    alpha, beta, tmax = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = small_workload(dim=1, g=60, n=3000, k=25, t=200, dtype="f64", ls=0.12)
    x = wl.x_train()
    ski = os_.SKI(og.grid_from_workload(wl), x, wl.noise, wl.y_train(x))
    _, a_ref, b_ref, _ = LZ.lanczos(ski.mvm, ski.probe(), wl.k)
    kk = min(len(alpha), len(a_ref))
    np.testing.assert_allclose(alpha[:kk], a_ref[:kk], rtol=1e-9)
    np.testing.assert_allclose(beta[: kk - 1], b_ref[: kk - 1], rtol=1e-7, atol=1e-9 * np.abs(b_ref).max())
    assert tmax == 2.0

"""The column-sharded nTT (Algorithm 2 with every unfolding distributed by
columns, Section III-B) rehearsed on CPU ranks: two and three gloo processes
run the library's driver (paper_2008_01340_gb300.sharded_ntt_decompose) with
FP64 ops that restate the oracle's updates, the all-reduce of [P ; Q] per
iteration and, between stages, the exchange of H's columns that lays out the
next unfolding (reshape of H) in the same column blocks.  The cores must equal
the unsharded FP64 oracle's."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth

import paper_2008_01340_gb300 as ntt

DIMS, RANKS, ITERS, SEED = (4, 6, 5, 4), (1, 3, 4, 2, 1), 9, 17


class OracleShardOps:
    """FP64 ops of one rank with the interface of the library's ShardOps."""

    def __init__(self, m, n_shard, r, eps=1e-12):
        self.m, self.r, self.eps = m, r, eps

    def norm2(self, X):
        return torch.tensor([float(np.sum(X.numpy() ** 2))], dtype=torch.float64)

    def local_pass(self, X, W, H):
        Xn, Wn, Hn = X.numpy(), W.numpy(), H.numpy()
        Hn[:] = oracle.mu_update_H(Xn, Wn, Hn, self.eps)
        return torch.from_numpy(np.concatenate([Xn @ Hn.T, Hn @ Hn.T], axis=0))

    def update(self, pq, W, xnorm2, obj=None):
        P, Q = pq.numpy()[: self.m], pq.numpy()[self.m:]
        Wn = W.numpy()
        Wn[:] = np.maximum(0.0, Wn * P / (Wn @ Q + self.eps))
        if obj is not None:
            obj[0] = 0.5 * (xnorm2 - 2.0 * float(np.sum(Wn * P)) + float(np.sum((Wn.T @ Wn) * Q)))


def _tensor():
    A, _ = synth.tt_tensor(DIMS, RANKS, "uniform", 0.01, seed=4)
    return A.astype(np.float64)


def _init(m, n, r, stage, c0, c1):
    W0, H0 = oracle.init_factors(m, n, r, SEED, stage, 0)
    return torch.from_numpy(np.array(W0)), torch.from_numpy(np.ascontiguousarray(H0[:, c0:c1]))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = _tensor()
    X1 = A.reshape(DIMS[0], -1)
    b = ntt.shard_bounds(X1.shape[1], world)
    Xs = torch.from_numpy(np.ascontiguousarray(X1[:, b[rank]:b[rank + 1]]))

    def exchange(sends):
        every = [None] * world
        dist.all_gather_object(every, [t.contiguous() for t in sends])
        return [every[q][rank] for q in range(world)]

    cores, traces = ntt.sharded_ntt_decompose(Xs, DIMS, RANKS, ITERS, rank, world, OracleShardOps, _init,
                                              all_reduce=lambda t: dist.all_reduce(t), exchange=exchange)
    out[rank] = ([c.numpy().copy() for c in cores], [list(t) for t in traces])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_ntt_equals_unsharded_oracle(world):
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    cores_o, traces_o = oracle.ntt_decompose(_tensor(), RANKS, ITERS, seed=SEED)
    for rank in range(world):
        cores, traces = out[rank]
        assert len(cores) == len(cores_o)
        for k, (g, o) in enumerate(zip(cores, cores_o)):
            assert g.shape == o.shape, (k, g.shape, o.shape)
            assert np.allclose(g, o, rtol=1e-9, atol=1e-12), f"rank {rank} core {k}"
        for t, to in zip(traces, traces_o):
            assert np.allclose(t, to, rtol=1e-8)


@pytest.mark.parametrize("r,n,nd,world", [(3, 120, 6, 2), (4, 30, 5, 3), (2, 4, 4, 3), (5, 77, 7, 4)])
def test_handoff_plan_lays_out_the_next_unfolding(r, n, nd, world):
    """Every column of H goes to exactly one rank, and placing the received
    columns as the driver does reproduces the C-order reshape of H."""
    rng = np.random.default_rng(r * n)
    H = rng.random((r, n))
    n2, plan = ntt.handoff_plan(r, n, nd, world)
    assert n2 == n // nd
    sent = sorted(k for q in range(world) for p in range(world) for k in plan[q][p])
    assert sent == list(range(n))
    hb, xb = ntt.shard_bounds(n, world), ntt.shard_bounds(n2, world)
    Xref = H.reshape(r * nd, n2)
    for p in range(world):
        e0, e1 = xb[p], xb[p + 1]
        Xp = np.full((r * nd, e1 - e0), np.nan)
        for q in range(world):
            ks = np.array(plan[q][p], dtype=int)
            assert np.all((ks >= hb[q]) & (ks < hb[q + 1]))     # q owns what it sends
            for k in ks:
                j, c = k // n2, k % n2
                Xp[np.arange(r) * nd + j, c - e0] = H[:, k]
        assert np.array_equal(Xp, Xref[:, e0:e1])

"""Column-sharded multiplicative updates (Section III-B's 1-D column
distribution) rehearsed on CPU ranks: two and three gloo processes run the
library's own driver (paper_2008_01340_gb300.sharded_nmf_mu) with FP64 ops
that restate the oracle's updates on each rank's columns, and the only
exchange is the driver's all-reduce of [P ; Q].  The result must equal the
unsharded FP64 oracle: the H update of a column needs only W, W^T W and that
column, and X H^T, H H^T are sums over columns."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth


class OracleShardOps:
    """FP64 ops of one rank with the interface of the library's ShardOps:
    [P ; Q] is carried as one (m + r) x r tensor."""

    def __init__(self, m, r, eps=1e-12):
        self.m, self.r, self.eps = m, r, eps

    def norm2(self, X):
        return torch.tensor([float(np.sum(X.numpy() ** 2))], dtype=torch.float64)

    def local_pass(self, X, W, H):
        Xn, Wn, Hn = X.numpy(), W.numpy(), H.numpy()
        Hn[:] = oracle.mu_update_H(Xn, Wn, Hn, self.eps)      # this rank's columns only
        pq = np.concatenate([Xn @ Hn.T, Hn @ Hn.T], axis=0)
        return torch.from_numpy(pq)

    def update(self, pq, W, xnorm2, obj=None):
        P, Q = pq.numpy()[: self.m], pq.numpy()[self.m:]
        Wn = W.numpy()
        Wn[:] = np.maximum(0.0, Wn * P / (Wn @ Q + self.eps))
        if obj is not None:
            G = Wn.T @ Wn
            obj[0] = 0.5 * (xnorm2 - 2.0 * float(np.sum(Wn * P)) + float(np.sum(G * Q)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    m, n, r = 12, 301, 4
    X = synth.uniform_matrix((m, n), 5).astype(np.float64)
    W0 = synth.uniform_matrix((m, r), 6).astype(np.float64)
    H0 = synth.uniform_matrix((r, n), 7).astype(np.float64)
    return X, W0, H0


def _worker(rank, world, port, iters, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2008_01340_gb300 as ntt
    X, W0, H0 = _problem()
    n = X.shape[1]
    bounds = np.linspace(0, n, world + 1).astype(int)       # contiguous, uneven column blocks
    c0, c1 = bounds[rank], bounds[rank + 1]
    Xs = torch.from_numpy(np.ascontiguousarray(X[:, c0:c1]))
    Hs = torch.from_numpy(np.ascontiguousarray(H0[:, c0:c1]))
    W = torch.from_numpy(W0.copy())
    trace = ntt.sharded_nmf_mu(Xs, W, Hs, iters, OracleShardOps(X.shape[0], W0.shape[1]),
                               all_reduce=lambda t: dist.all_reduce(t))
    out[rank] = (c0, c1, W.numpy().copy(), Hs.numpy().copy(), trace)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_mu_equals_unsharded_oracle(world):
    iters = 7
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, iters, out), nprocs=world, join=True)
    X, W0, H0 = _problem()
    Wo, Ho, tr = oracle.nmf_mu(X, W0, H0, iters)
    H = np.zeros_like(Ho)
    for rank in range(world):
        c0, c1, W, Hs, trace = out[rank]
        assert np.allclose(W, Wo, rtol=1e-12, atol=0)          # every replica of W
        H[:, c0:c1] = Hs
        # the Gram-form objective of every rank against the oracle's direct one
        assert np.allclose(trace, tr, rtol=1e-9)
    assert np.allclose(H, Ho, rtol=1e-12, atol=0)

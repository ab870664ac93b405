"""Column-sharded multiplicative updates through the C ABI on one GPU: the
shards of one problem run one after another on the same device and the sum of
their FP64 [P ; Q] stands in for the all-reduce (ranks whose kernels wait on
each other never share a GPU; these shards do not wait).  Iterates match the
unsharded nmf_mu_step and the FP64 oracle within the FP32 bound after 10
iterations; the library's driver runs unchanged with one shard."""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ntt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2008_01340_gb300 as mod
    mod.build()
    mod.lib()
    return mod


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("m,n,r,bounds", [(32, 40000, 8, (0, 16000, 40000)),
                                          (256, 30000, 16, (0, 10000, 20004, 30000)),
                                          (100, 7777, 5, (0, 3001, 7777))])
def test_sharded_iterates_match_unsharded(ntt, m, n, r, bounds):
    rng = np.random.Generator(np.random.PCG64(m))
    X = (rng.random((m, 5)) @ rng.random((5, n)) + 0.01 * rng.random((m, n))).astype(np.float32)
    W0 = synth.uniform_matrix((m, r), 3)
    H0 = synth.uniform_matrix((r, n), 4)
    iters = 10
    shards = list(zip(bounds[:-1], bounds[1:]))
    Xs = [torch.from_numpy(np.ascontiguousarray(X[:, a:b])).cuda() for a, b in shards]
    Hs = [torch.from_numpy(np.ascontiguousarray(H0[:, a:b])).cuda() for a, b in shards]
    W = torch.from_numpy(W0.copy()).cuda()
    ops = [ntt.ShardOps(m, b - a, r) for a, b in shards]
    xn = sum(float(o.norm2(x)[0]) for o, x in zip(ops, Xs))
    # FP32 squares summed in FP64: within 2^-24 relative of the FP64 sum
    assert abs(xn - float(np.sum(X.astype(np.float64) ** 2))) <= 6e-8 * xn
    trace = []
    for _ in range(iters):
        pq = sum(o.local_pass(x, W, h).clone() for o, x, h in zip(ops, Xs, Hs))   # the all-reduce
        obj = torch.zeros(1, dtype=torch.float64, device="cuda")
        ops[0].update(pq, W, xn, obj)
        trace.append(float(obj[0]))
    Hg = np.concatenate([h.cpu().numpy() for h in Hs], axis=1)
    Wg = W.cpu().numpy()
    # against the unsharded device path and the oracle
    Wd = torch.from_numpy(W0.copy()).cuda()
    Hd = torch.from_numpy(H0.copy()).cuda()
    ntt.nmf_mu_step(torch.from_numpy(X).cuda(), Wd, Hd, iters)
    torch.cuda.synchronize()
    assert _rel(Wg, Wd.cpu().numpy()) <= 1e-5 and _rel(Hg, Hd.cpu().numpy()) <= 1e-5
    Wo, Ho, tr = oracle.nmf_mu(X.astype(np.float64), W0, H0, iters)
    assert _rel(Wg, Wo) <= 1e-4 and _rel(Hg, Ho) <= 1e-4
    assert np.allclose(trace, tr, rtol=2e-3, atol=1e-6 * xn)


def test_driver_with_one_shard_equals_nmf_mu_step(ntt):
    m, n, r = 64, 20000, 12
    X = torch.from_numpy(synth.uniform_matrix((m, n), 8)).cuda()
    W0 = synth.uniform_matrix((m, r), 9)
    H0 = synth.uniform_matrix((r, n), 10)
    W = torch.from_numpy(W0.copy()).cuda()
    H = torch.from_numpy(H0.copy()).cuda()
    trace = ntt.sharded_nmf_mu(X, W, H, 6, ntt.ShardOps(m, n, r))
    Wd = torch.from_numpy(W0.copy()).cuda()
    Hd = torch.from_numpy(H0.copy()).cuda()
    ntt.nmf_mu_step(X, Wd, Hd, 6)
    torch.cuda.synchronize()
    assert _rel(W.cpu(), Wd.cpu()) <= 1e-6 and _rel(H.cpu(), Hd.cpu()) <= 1e-6
    assert len(trace) == 6 and all(np.diff(trace) <= 1e-9 * trace[0])


def test_sharded_ntt_driver_one_rank_on_device(ntt):
    """The sharded nTT driver (stage hand-off included) with the library's
    device ShardOps on one rank: its cores against the FP64 oracle's, within
    the chained per-core bound used for every decomposition (1e-4 (k + 1))."""
    dims, ranks, iters, seed = (8, 12, 10, 9), (1, 4, 6, 3, 1), 10, 21
    A, _ = synth.tt_tensor(dims, ranks, "uniform", 0.01, seed=6)
    X1 = torch.from_numpy(np.ascontiguousarray(A.reshape(dims[0], -1).astype(np.float32))).cuda()

    def init(m, n, r, stage, c0, c1):
        W0, H0 = oracle.init_factors(m, n, r, seed, stage, 0)
        return (torch.from_numpy(np.asarray(W0, np.float32)).cuda(),
                torch.from_numpy(np.ascontiguousarray(np.asarray(H0, np.float32)[:, c0:c1])).cuda())

    cores, _ = ntt.sharded_ntt_decompose(X1, dims, ranks, iters, 0, 1, ntt.ShardOps, init)
    torch.cuda.synchronize()
    cores_o, _ = oracle.ntt_decompose(A.astype(np.float64), ranks, iters, seed=seed)
    for k, (g, o) in enumerate(zip(cores, cores_o)):
        assert tuple(g.shape) == o.shape
        assert _rel(g.cpu().numpy(), o) <= 1e-4 * (k + 1), f"core {k}"

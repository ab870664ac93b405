"""Algorithm 3 (BCD NMF) on the GPU through the C ABI against the FP64 oracle.

Tolerances, as for the multiplicative updates: iterates from identical initial
factors within 1e-4 relative (Frobenius) after 10 iterations; a whole nTT's
cores within 1e-4 x (stage index + 1) after 10 iterations per stage and its
final Eq. (3) error within 1e-3 absolute.  Every test first checks, on the
oracle's run, that each accept/reject decision is clear of rounding: the new
objective differs from the last accepted one by more than 1e-5 of it (the
device decides on the FP64 Gram form built from FP32 sums).
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_ITERATE = 1e-4


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
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _x(kind, m, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "uniform":
        return rng.random((m, n), dtype=np.float32)
    k = max(1, min(m, 5))
    X = rng.random((m, k)) @ rng.random((k, n))
    X += 0.01 * X.mean() * rng.random((m, n))
    return X.astype(np.float32)


def _decisions_clear(X, W0, H0, iters, margin=1e-5):
    info = {}
    _, _, tr, acc = oracle.bcd_nmf(X.astype(np.float64), W0, H0, iters, info=info)
    prev = 0.5 * float(np.sum(X.astype(np.float64) ** 2))
    for f, t in zip(info["f"], tr):
        if abs(f - prev) <= margin * abs(prev):
            return False
        prev = t
    return True


SHAPES = [(32, 40000, 8, "lowrank"), (24, 777, 3, "uniform"), (16, 4096, 16, "lowrank"),
          (100, 5000, 5, "lowrank"), (64, 10002, 20, "uniform"), (256, 8192, 16, "lowrank"),
          (512, 3000, 32, "lowrank"), (9, 100, 2, "uniform")]


@pytest.mark.parametrize("m,n,r,kind", SHAPES)
def test_bcd_iterates_match_oracle(ntt, m, n, r, kind):
    X = _x(kind, m, n, 7 + m)
    W0 = synth.uniform_matrix((m, r), 8)
    H0 = synth.uniform_matrix((r, n), 9)
    iters = 10
    assert _decisions_clear(X, W0, H0, iters)
    Wd = torch.from_numpy(W0.copy()).cuda()
    Hd = torch.from_numpy(H0.copy()).cuda()
    obj = torch.zeros(iters, dtype=torch.float64, device="cuda")
    ws = ntt.nmf_bcd_step(torch.from_numpy(X).cuda(), Wd, Hd, iters, obj)
    torch.cuda.synchronize()
    assert ntt.ntt_status_of_workspace(ws) == "NTT_OK"
    Wo, Ho, tr, acc = oracle.bcd_nmf(X.astype(np.float64), W0, H0, iters)
    Wg, Hg = Wd.cpu().numpy(), Hd.cpu().numpy()
    assert _rel(Wg, Wo) <= REL_ITERATE, _rel(Wg, Wo)
    assert _rel(Hg, Ho) <= REL_ITERATE, _rel(Hg, Ho)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    # the accepted-objective trace (Gram form on the device)
    xn2 = float(np.sum(X.astype(np.float64) ** 2))
    assert np.allclose(obj.cpu().numpy(), tr, rtol=2e-3, atol=1e-6 * xn2)


def test_bcd_rank_one_fixed_point(ntt):
    rng = np.random.Generator(np.random.PCG64(3))
    u = (rng.random((40, 1)) + 0.2).astype(np.float32)
    v = (rng.random((1, 3000)) + 0.2).astype(np.float32)
    X = (u @ v).astype(np.float32)
    Wd = torch.from_numpy(2.0 * u).cuda()
    Hd = torch.from_numpy(0.25 * v).cuda()
    ntt.nmf_bcd_step(torch.from_numpy(X).cuda(), Wd, Hd, 10)
    torch.cuda.synchronize()
    WH = Wd.cpu().numpy().astype(np.float64) @ Hd.cpu().numpy().astype(np.float64)
    assert _rel(WH, X) <= 1e-6


def test_bcd_monotone_and_converges_on_exact_low_rank(ntt):
    m, n, r = 48, 6000, 4
    rng = np.random.Generator(np.random.PCG64(4))
    X = (rng.random((m, r)) @ rng.random((r, n))).astype(np.float32)
    W0 = synth.uniform_matrix((m, r), 1)
    H0 = synth.uniform_matrix((r, n), 2)
    iters = 300
    Wd = torch.from_numpy(W0.copy()).cuda()
    Hd = torch.from_numpy(H0.copy()).cuda()
    obj = torch.zeros(iters, dtype=torch.float64, device="cuda")
    ntt.nmf_bcd_step(torch.from_numpy(X).cuda(), Wd, Hd, iters, obj)
    torch.cuda.synchronize()
    tr = obj.cpu().numpy()
    assert np.all(np.diff(tr) <= 0.0)
    xn2 = float(np.sum(X.astype(np.float64) ** 2))
    direct = oracle.objective(X.astype(np.float64), Wd.cpu().numpy(), Hd.cpu().numpy())
    assert direct <= 1e-5 * 0.5 * xn2
    # the same number of multiplicative updates ends higher (the paper's comparison)
    Wm = torch.from_numpy(W0.copy()).cuda()
    Hm = torch.from_numpy(H0.copy()).cuda()
    ntt.nmf_mu_step(torch.from_numpy(X).cuda(), Wm, Hm, iters)
    torch.cuda.synchronize()
    assert direct < oracle.objective(X.astype(np.float64), Wm.cpu().numpy(), Hm.cpu().numpy())


def test_bcd_repeats_bitwise(ntt):
    X = torch.from_numpy(_x("lowrank", 64, 20000, 5)).cuda()
    out = []
    for _ in range(2):
        Wd = torch.from_numpy(synth.uniform_matrix((64, 12), 6)).cuda()
        Hd = torch.from_numpy(synth.uniform_matrix((12, 20000), 7)).cuda()
        ntt.nmf_bcd_step(X, Wd, Hd, 25)
        torch.cuda.synchronize()
        out.append((Wd.cpu().numpy(), Hd.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def _decompose(ntt, A, ranks, iters, seed, solver):
    plan = ntt.ntt_plan_create(A.shape, ranks, iters, 1e-12, "f32", 0, seed, solver=solver)
    ws = ntt.empty_workspace(plan.workspace_size())
    cores = [torch.empty(s, dtype=torch.float32, device="cuda") for s in plan.core_shapes()]
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    ntt.ntt_decompose(plan, Ad, cores, ws)
    stats = ntt.ntt_plan_get_stats(plan)
    return [c.cpu().numpy() for c in cores], stats


def test_bcd_ntt_c1_per_iterate_and_final(ntt):
    c = synth.CONFIGS["c1_8x4"]
    A, _ = synth.tt_tensor(c["dims"], c["ranks"], c["core_dist"], c["noise"], c["data_seed"])
    cores_g, stats = _decompose(ntt, A, c["ranks"], 10, c["init_seed"], "bcd")
    assert stats["status"] == "NTT_OK"
    assert all(st["engine"] == "bcd_pass" for st in stats["stages"])
    cores_o, _ = oracle.ntt_decompose(A, c["ranks"], 10, seed=c["init_seed"], solver="bcd")
    for k, (g, o) in enumerate(zip(cores_g, cores_o)):
        assert _rel(g, o) <= REL_ITERATE * (k + 1), f"core {k}: {_rel(g, o):.2e}"
    cores_g, _ = _decompose(ntt, A, c["ranks"], c["iters"], c["init_seed"], "bcd")
    cores_o, _ = oracle.ntt_decompose(A, c["ranks"], c["iters"], seed=c["init_seed"], solver="bcd", record=False)
    eg, eo = oracle.rel_error(A, cores_g), oracle.rel_error(A, cores_o)
    print(f"C1 BCD: gpu {eg:.6f} oracle {eo:.6f}")
    assert abs(eg - eo) <= 1e-3
    assert all(np.all(g >= 0) and np.all(np.isfinite(g)) for g in cores_g)


def test_bcd_ntt_16x6_final_error(ntt):
    """The 32^6 recipe scaled to 16^6 with the BCD solver: final Eq. (3) error
    within 1e-3 of the oracle's, and below the multiplicative updates' at the
    same iteration count."""
    c = synth.CONFIGS["c2_32x6"]
    dims = (16,) * 6
    A, _ = synth.tt_tensor(dims, c["ranks"], c["core_dist"], c["noise"], c["data_seed"])
    cores_g, stats = _decompose(ntt, A, c["ranks"], 100, c["init_seed"], "bcd")
    assert stats["status"] == "NTT_OK"
    cores_o, _ = oracle.ntt_decompose(A, c["ranks"], 100, seed=c["init_seed"], solver="bcd", record=False)
    eg, eo = oracle.rel_error(A, cores_g), oracle.rel_error(A, cores_o)
    cores_mu, _ = _decompose(ntt, A, c["ranks"], 100, c["init_seed"], "mu")
    emu = oracle.rel_error(A, cores_mu)
    print(f"16^6 BCD: gpu {eg:.6f} oracle {eo:.6f}; MU gpu {emu:.6f}")
    assert abs(eg - eo) <= 1e-3
    assert eg < emu


def test_bcd_rejected_iteration_matches_oracle(ntt):
    """A case whose 23rd iteration is rejected (the extrapolated step raises
    the objective), with every decision of the first 26 clear by > 4e-2: the
    device rejects the same iteration (its accepted-objective trace repeats the
    previous value exactly) and the iterates after it still match."""
    rng = np.random.Generator(np.random.PCG64(6))
    m, n, r = 24, 3000, 4
    X = (rng.random((m, r)) @ rng.random((r, n))).astype(np.float32)
    X += (0.001 * rng.random((m, n))).astype(np.float32)
    W0 = synth.uniform_matrix((m, r), 8)
    H0 = synth.uniform_matrix((r, n), 9)
    iters = 26
    assert _decisions_clear(X, W0, H0, iters, margin=1e-3)
    Wo, Ho, tr, acc = oracle.bcd_nmf(X.astype(np.float64), W0, H0, iters)
    assert not acc[22] and acc[:22].all()
    Wd = torch.from_numpy(W0.copy()).cuda()
    Hd = torch.from_numpy(H0.copy()).cuda()
    obj = torch.zeros(iters, dtype=torch.float64, device="cuda")
    ntt.nmf_bcd_step(torch.from_numpy(X).cuda(), Wd, Hd, iters, obj)
    torch.cuda.synchronize()
    o = obj.cpu().numpy()
    assert o[22] == o[21] and np.all(np.diff(o)[:21] < 0)
    assert _rel(Wd.cpu().numpy(), Wo) <= REL_ITERATE
    assert _rel(Hd.cpu().numpy(), Ho) <= REL_ITERATE

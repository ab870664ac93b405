"""Algorithm 2's rank rule on the GPU (through the C ABI) against the FP64 oracle.

Tolerances:
  * eigenvalues of the Gram (sigma_i^2): |delta| <= 2e-5 * sigma_1^2 -- the
    Gram carries the FP32 rounding of its products and of runs of 256 sums
    (about 1e-6 of an entry), and an eigenvalue moves by at most the spectral
    norm of the perturbation (Weyl), below 512 x 1e-6 of the largest entry
    relative to sigma_1^2 in the worst case;
  * chosen ranks: equal (an integer decided in floating point: every eps is
    chosen so that no tail ratio lies within 1e-3 of it, relative);
  * cores of a rank-rule decomposition: the per-iterate bound of the fixed-rank
    tests, 1e-4 x (stage index + 1), after 10 iterations per stage.
"""

import math

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


def _tail_ratios(sig):
    s2 = np.asarray(sig, np.float64) ** 2
    tot = s2.sum()
    return np.array([math.sqrt(s2[k:].sum() / tot) for k in range(1, len(s2) + 1)])


def _clear(eps, ratio_sets, margin=1e-3):
    return all(np.all(np.abs(r - eps) > margin * eps) for r in ratio_sets)


def _matrix(kind, m, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "uniform":
        return rng.random((m, n), dtype=np.float32)
    k = max(1, min(m, n) // 3)
    X = rng.random((m, k)) @ rng.random((k, n)) + 0.01 * rng.random((m, n))
    return X.astype(np.float32)


SHAPES = [(1, 300, "uniform"), (7, 1000, "lowrank"), (64, 4096, "lowrank"), (65, 3000, "uniform"),
          (130, 777, "lowrank"), (300, 40, "lowrank"), (512, 2048, "lowrank"), (2000, 96, "uniform")]


@pytest.mark.parametrize("m,n,kind", SHAPES)
def test_singular_values_match_oracle(ntt, m, n, kind):
    X = _matrix(kind, m, n, 11 + m)
    sig = ntt.ntt_singular_values(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = oracle.singular_values(X)
    assert sig.shape == ref.shape
    assert np.all(np.diff(sig) <= 0.0)
    assert np.max(np.abs(sig ** 2 - ref ** 2)) <= 2e-5 * ref[0] ** 2


@pytest.mark.parametrize("m,n,kind", SHAPES)
def test_select_rank_matches_oracle(ntt, m, n, kind):
    X = _matrix(kind, m, n, 21 + m)
    ref_sig = oracle.singular_values(X)
    ratios = _tail_ratios(ref_sig)
    Xd = torch.from_numpy(X).cuda()
    checked = 0
    for eps in (0.9, 0.5, 0.3, 0.1, 0.05, 0.02, 0.01, 3e-3):
        if not _clear(eps, [ratios]):
            continue
        for cap in (0, 3):
            k = int(ntt.ntt_select_rank(Xd, eps, cap).item())
            assert k == oracle.select_rank(ref_sig, eps, cap if cap else None), (eps, cap)
        checked += 1
    assert checked >= 4


def test_select_rank_zero_matrix_is_one(ntt):
    X = torch.zeros((16, 100), dtype=torch.float32, device="cuda")
    assert int(ntt.ntt_select_rank(X, 0.1).item()) == 1


def _pick_eps(A, iters, seed, candidates, **kw):
    for eps in candidates:
        info = {}
        cores, _ = oracle.ntt_decompose(A, None, iters, seed=seed, eps_rank=eps, info=info, record=False, **kw)
        if _clear(eps, [_tail_ratios(s) for s in info["sigma"]]):
            return eps, cores
    return None, None


@pytest.mark.parametrize("dims,true_ranks,rank_cap", [((8, 8, 8, 8), (1, 3, 3, 3, 1), 0),
                                                      ((6, 7, 8, 5, 4), (1, 4, 6, 5, 3, 1), 0),
                                                      ((6, 7, 8, 5, 4), (1, 4, 6, 5, 3, 1), 3)])
def test_rank_rule_decomposition_matches_oracle(ntt, dims, true_ranks, rank_cap):
    A, _ = synth.tt_tensor(dims, true_ranks, "uniform", 0.01, seed=5)
    iters, seed = 10, 9
    eps, cores_o = _pick_eps(A, iters, seed, (0.05, 0.03, 0.02, 0.07, 0.1, 0.015, 0.04),
                             rank_cap=rank_cap or None)
    assert eps is not None
    plan = ntt.ntt_plan_create(dims, None, iters, 1e-12, "f32", 0, seed, eps_rank=eps, rank_cap=rank_cap)
    ws = ntt.empty_workspace(plan.workspace_size())
    bufs = [torch.zeros(s, dtype=torch.float32, device="cuda") for s in plan.core_shapes()]
    Ad = torch.from_numpy(A).cuda()
    ntt.ntt_decompose(plan, Ad, bufs, ws)
    stats = ntt.ntt_plan_get_stats(plan)
    assert stats["status"] == "NTT_OK"
    ranks = plan.current_ranks()
    assert ranks == tuple([1] + [c.shape[2] for c in cores_o])
    assert [st["r"] for st in stats["stages"]] == list(ranks[1:-1])
    cores_g = [c.cpu().numpy() for c in plan.core_views(bufs)]
    for k, (g, o) in enumerate(zip(cores_g, cores_o)):
        assert g.shape == o.shape
        rel = np.linalg.norm((g - o).ravel()) / np.linalg.norm(o.ravel())
        assert rel <= 1e-4 * (k + 1), f"core {k}: {rel:.2e}"
    # Eq. (3) of the result on the device agrees with the oracle's error of the GPU cores
    err = torch.zeros(3, dtype=torch.float64, device="cuda")
    ntt.ntt_rel_error(dims, ranks, [torch.from_numpy(np.ascontiguousarray(g)).cuda() for g in cores_g], Ad, err)
    assert abs(err[0].item() - oracle.rel_error(A, cores_g)) <= 1e-6
    # a second call on the same plan repeats bitwise
    bufs2 = [torch.zeros(s, dtype=torch.float32, device="cuda") for s in plan.core_shapes()]
    ntt.ntt_decompose(plan, Ad, bufs2, ws)
    torch.cuda.synchronize()
    for a, b in zip(plan.core_views(bufs), plan.core_views(bufs2)):
        assert torch.equal(a, b)


def test_rank_rule_c2_first_unfolding_full_size(ntt):
    """Stage 1 of the 32^6 workload (32 x 33,554,432): singular values of the
    full unfolding against the oracle's, from its FP64 Gram (the oracle's SVD
    of the same matrix through its 32 x 32 Gram: equal singular values), and
    the rule's rank at thresholds clear of every tail ratio."""
    c = synth.CONFIGS["c2_32x6"]
    A, _ = synth.tt_tensor(c["dims"], c["ranks"], c["core_dist"], c["noise"], c["data_seed"])
    X = A.reshape(32, -1)
    G = np.zeros((32, 32))
    for c0 in range(0, X.shape[1], 1 << 22):
        Xc = X[:, c0:c0 + (1 << 22)].astype(np.float64)
        G += Xc @ Xc.T
    ref = np.sqrt(np.maximum(0.0, np.linalg.eigvalsh(G)[::-1]))
    Xd = torch.from_numpy(X).cuda()
    sig = ntt.ntt_singular_values(Xd).cpu().numpy()
    assert np.max(np.abs(sig ** 2 - ref ** 2)) <= 2e-5 * ref[0] ** 2
    ratios = _tail_ratios(ref)
    for eps in (0.1, 0.01, 3e-3):
        if _clear(eps, [ratios]):
            assert int(ntt.ntt_select_rank(Xd, eps).item()) == oracle.select_rank(ref, eps)

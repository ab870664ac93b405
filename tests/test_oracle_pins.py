"""Pins of the FP64 oracle to facts fixed outside it (no GPU needed).

Each test checks an oracle function against something the paper or the
mathematics fixes: a printed example, a closed form, an invariant, a textbook
or library routine for a special case, or brute force on a tiny input.
"""

import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    vals = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if len(parts) == 1:
                vals.append(parts[0])
            else:
                out[parts[0]] = parts[1:]
    return out, vals


# ---------------------------------------------------------------- RNG

def test_splitmix64_published_vector():
    _, vals = _read_golden("splitmix64_seed1234567.txt")
    got = oracle.splitmix64_outputs(1234567, np.arange(5))
    assert [int(v) for v in got] == [int(v) for v in vals]


def test_uniform01_is_24bit_and_in_range():
    key = oracle.stream_key(7, 0, 0, 1)
    u = oracle.uniform01(key, np.arange(100000, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0
    scaled = u * 16777216.0
    assert np.all(scaled == np.floor(scaled))           # multiples of 2^-24
    assert np.all(u.astype(np.float32).astype(np.float64) == u)   # exact in FP32
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1.0 / 12.0) < 0.002


def test_stream_keys_distinct_and_counter_consistent():
    keys = {oracle.stream_key(3, s, r, mtx) for s in range(8) for r in range(8) for mtx in range(2)}
    assert len(keys) == 128
    W0, H0 = oracle.init_factors(5, 37, 3, seed=3, stage=2, restart=1)
    cols = np.array([0, 5, 36])
    assert np.array_equal(oracle.init_columns_H(37, 3, 3, 2, cols, restart=1), H0[:, cols])


# ---------------------------------------------------------------- Eq. (2)

def test_eq2_brute_force_tiny():
    dims, ranks = (3, 4, 2, 3), (1, 2, 3, 2, 1)
    cores = synth.tt_cores(dims, ranks, "uniform", seed=11)
    full = oracle.tt_full(cores)
    for idx in itertools.product(*[range(n) for n in dims]):
        # Eq. (2) written as the explicit sum over all rank indices k_1..k_{d-1}
        s = 0.0
        for ks in itertools.product(*[range(r) for r in ranks[1:-1]]):
            kk = (0, *ks, 0)
            p = 1.0
            for j in range(len(dims)):
                p *= cores[j][kk[j], idx[j], kk[j + 1]]
            s += p
        assert abs(full[idx] - s) <= 1e-14 * max(1.0, abs(s))
        assert abs(oracle.tt_entry(cores, idx) - s) <= 1e-14 * max(1.0, abs(s))


def test_eq2_rank_one_is_outer_product():
    dims = (3, 4, 5)
    vecs = [np.arange(1, n + 1, dtype=np.float64) for n in dims]
    cores = [v.reshape(1, -1, 1) for v in vecs]
    expect = np.einsum("i,j,k->ijk", *vecs)
    assert np.array_equal(oracle.tt_full(cores), expect)


# ---------------------------------------------------------------- Eq. (3), Eq. (4)

def test_eq3_closed_forms():
    dims, ranks = (4, 3, 5), (1, 2, 2, 1)
    cores = synth.tt_cores(dims, ranks, "uniform", seed=5)
    A = oracle.tt_full(cores)
    assert oracle.rel_error(A, cores) <= 1e-15
    c = 0.75
    scaled = [cores[0] * c] + cores[1:]
    assert abs(oracle.rel_error(A, scaled) - abs(1 - c)) <= 1e-14


def test_eq4_fig1_example():
    g, _ = _read_golden("fig1_tt_example.txt")
    dims = tuple(int(x) for x in g["dims"])
    ranks = tuple(int(x) for x in g["ranks"])
    assert sum(n * ranks[i] * ranks[i + 1] for i, n in enumerate(dims)) == int(g["params"][0])
    assert abs(oracle.compression_ratio(dims, ranks) - 600.0 / 110.0) < 1e-15


def test_eq4_config_c1():
    c = synth.CONFIGS["c1_8x4"]
    assert oracle.compression_ratio(c["dims"], c["ranks"]) == 4096.0 / 192.0


# ---------------------------------------------------------------- MU invariants

def _rand(shape, seed):
    return np.random.Generator(np.random.PCG64(seed)).random(shape)


def test_mu_fixed_point():
    Ws, Hs = _rand((9, 3), 1) + 0.1, _rand((3, 40), 2) + 0.1
    X = Ws @ Hs
    H1 = oracle.mu_update_H(X, Ws, Hs)
    W1 = oracle.mu_update_W(X, Ws, H1)
    assert np.max(np.abs(H1 - Hs) / Hs) <= 1e-12
    assert np.max(np.abs(W1 - Ws) / Ws) <= 1e-12


def test_mu_update_matches_elementwise_definition():
    # one H and one W update written element by element (small loops)
    X, W, H = _rand((5, 7), 3), _rand((5, 2), 4), _rand((2, 7), 5)
    eps = 1e-12
    Hn = np.zeros_like(H)
    for k in range(2):
        for j in range(7):
            num = sum(W[i, k] * X[i, j] for i in range(5))
            den = sum(sum(W[i, k] * W[i, l] for i in range(5)) * H[l, j] for l in range(2)) + eps
            Hn[k, j] = max(0.0, H[k, j] * num / den)
    Wn = np.zeros_like(W)
    for i in range(5):
        for k in range(2):
            num = sum(X[i, j] * Hn[k, j] for j in range(7))
            den = sum(W[i, l] * sum(Hn[l, j] * Hn[k, j] for j in range(7)) for l in range(2)) + eps
            Wn[i, k] = max(0.0, W[i, k] * num / den)
    assert np.allclose(oracle.mu_update_H(X, W, H), Hn, rtol=1e-13, atol=0)
    assert np.allclose(oracle.mu_update_W(X, W, Hn), Wn, rtol=1e-13, atol=0)
    W2, H2, tr = oracle.nmf_mu(X, W, H, 1)
    assert np.allclose(H2, Hn, rtol=1e-13) and np.allclose(W2, Wn, rtol=1e-13)
    assert abs(tr[0] - 0.5 * np.sum((X - Wn @ Hn) ** 2)) <= 1e-12 * tr[0]


def test_mu_objective_monotone_and_nonnegative():
    X = _rand((30, 200), 6) ** 2
    X[3, :] = 0.0                       # an all-zero row
    X[:, 7] = 0.0                       # and an all-zero column
    W0, H0 = _rand((30, 4), 7), _rand((4, 200), 8)
    W, H, tr = oracle.nmf_mu(X, W0, H0, 300)
    assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])
    assert np.all(W >= 0) and np.all(H >= 0)
    assert np.all(np.isfinite(W)) and np.all(np.isfinite(H))


def test_rank_one_converges_to_svd_optimum():
    # rank-1 NMF of a positive matrix: the optimum is sigma_1 u_1 v_1^T (Perron-Frobenius)
    X = _rand((12, 50), 9) + 0.5
    W0, H0 = _rand((12, 1), 10), _rand((1, 50), 11)
    W, H, tr = oracle.nmf_mu(X, W0, H0, 3000)
    s = np.linalg.svd(X, compute_uv=False)
    best = 0.5 * (np.sum(X * X) - s[0] ** 2)
    assert abs(tr[-1] - best) <= 1e-9 * np.sum(X * X)


def test_full_rank_stage_error_goes_to_zero():
    X = _rand((6, 300), 12) + 0.1
    W0, H0 = _rand((6, 6), 13), _rand((6, 300), 14)
    W, H, tr = oracle.nmf_mu(X, W0, H0, 3000)
    assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])
    assert tr[-1] <= 1e-3 * tr[0]


def test_stopping_test_limits():
    """The optional relative-change test: with tol = 0 the loop is the fixed
    count (bitwise); with tol >= 1 it must fire at its first opportunity u = 2K,
    because MU never raises the objective (Lee-Seung) and the objective is >= 0,
    so f_{u-K} - f_u <= f_{u-K} always holds; a stopped run equals a fixed-count
    run of the same length."""
    X = _rand((20, 150), 30) ** 2
    W0, H0 = _rand((20, 3), 31), _rand((3, 150), 32)
    Wf, Hf, trf = oracle.nmf_mu(X, W0, H0, 60)
    Wz, Hz, trz = oracle.nmf_mu(X, W0, H0, 60, tol=0.0, check_every=7)
    assert np.array_equal(Wf, Wz) and np.array_equal(Hf, Hz) and np.array_equal(trf, trz)
    for K in (1, 5, 7):
        Ws, Hs, trs = oracle.nmf_mu(X, W0, H0, 60, tol=1.0, check_every=K)
        assert len(trs) == 2 * K
        Wk, Hk, trk = oracle.nmf_mu(X, W0, H0, 2 * K)
        assert np.array_equal(Ws, Wk) and np.array_equal(Hs, Hk) and np.array_equal(trs, trk)
    # a stop needs a completed check: fewer than 2K iterations never stop early
    _, _, tr = oracle.nmf_mu(X, W0, H0, 9, tol=1.0, check_every=5)
    assert len(tr) == 9


def test_stopping_test_stops_where_decrease_falls_below_tol():
    """On a monotone trace the test stops at the first check whose K-iteration
    relative decrease is <= tol; a tol between two consecutive checks' decreases
    separates them, and a run to convergence of the exact-recovery case (the
    decrease shrinks towards 0) stops before the iteration cap."""
    X = _rand((20, 150), 33) ** 2
    W0, H0 = _rand((20, 3), 34), _rand((3, 150), 35)
    K = 10
    _, _, full = oracle.nmf_mu(X, W0, H0, 200)
    dec = {u: (full[u - K - 1] - full[u - 1]) / full[u - K - 1] for u in range(2 * K, 201, K)}
    # decreases of a converging MU trace shrink: pick tol between two checks
    us = sorted(dec)
    i = next(j for j in range(1, len(us)) if dec[us[j]] < 0.5 * dec[us[j - 1]])
    tol = math.sqrt(dec[us[i]] * dec[us[i - 1]])
    first = next(u for u in us if dec[u] <= tol)
    _, _, tr = oracle.nmf_mu(X, W0, H0, 200, tol=tol, check_every=K)
    assert len(tr) == first
    # noise-free rank-2 product: f -> 0, so a small tol still stops early
    Wt, Ht = _rand((12, 2), 36) + 0.1, _rand((2, 40), 37) + 0.1
    _, _, tr = oracle.nmf_mu(Wt @ Ht, _rand((12, 2), 38), _rand((2, 40), 39), 20000, tol=1e-6, check_every=K)
    assert 2 * K <= len(tr) < 20000 and len(tr) % K == 0


def test_ntt_stopping_test_per_stage():
    """Each stage's main loop stops under the test on its own trace; the
    refinement iterations of the precision form always run."""
    A = _rand((6, 5, 4), 40)
    cores, traces = oracle.ntt_decompose(A, (1, 3, 2, 1), iters=100, seed=3, tol=1.0, check_every=4)
    assert [len(t) for t in traces] == [8, 8]
    cores, traces = oracle.ntt_decompose(A, (1, 3, 2, 1), iters=100, seed=3, tol=1.0, check_every=4,
                                         x_precision="bf16", refine=3)
    assert [len(t) for t in traces] == [11, 11]


# ---------------------------------------------------------------- hand-off and Algorithm 2

def test_handoff_normalize_keeps_product():
    W, H = _rand((8, 3), 15), _rand((3, 20), 16)
    W[:, 1] = 0.0
    Wn, Hn = oracle.handoff_normalize(W, H)
    assert np.allclose(Wn @ Hn, W @ H, rtol=1e-14, atol=0)
    assert np.allclose(Wn[:, [0, 2]].sum(axis=0), 1.0, rtol=1e-15)
    assert np.all(Wn[:, 1] == 0.0) and np.array_equal(Hn[1], H[1])


def test_unfold_views_match_algorithm2_shapes():
    dims, ranks = (5, 4, 5, 6), (1, 4, 3, 2, 1)
    shapes = synth.stage_shapes(dims, ranks)
    assert shapes == [(5, 120, 4), (16, 30, 3), (15, 6, 2)]
    # C-order: element H[a, i*N + c] is row a*n + i, column c of the next unfolding
    H = np.arange(4 * 120).reshape(4, 120)
    X2 = oracle.unfold(H, 16)
    for a, i, c in [(0, 0, 0), (3, 3, 29), (2, 1, 7)]:
        assert X2[a * 4 + i, c] == H[a, i * 30 + c]


def test_ntt_d2_is_one_nmf():
    A = _rand((7, 30), 17)
    cores, traces = oracle.ntt_decompose(A, (1, 3, 1), iters=50, seed=9)
    W0, H0 = oracle.init_factors(7, 30, 3, 9, 0)
    W, H, tr = oracle.nmf_mu(A, W0, H0, 50)
    Wn, Hn = oracle.handoff_normalize(W, H)
    assert np.allclose(cores[0].reshape(7, 3), Wn, rtol=1e-13)
    assert np.allclose(cores[1].reshape(3, 30), Hn, rtol=1e-13)
    assert np.allclose(traces[0], tr, rtol=1e-13)


def test_ntt_exact_recovery_noise_free():
    # tensor built from non-negative TT cores at the true ranks: small error
    dims, ranks = (6, 6, 6), (1, 2, 2, 1)
    A, _ = synth.tt_tensor(dims, ranks, "uniform", noise=0.0, seed=21)
    cores, traces = oracle.ntt_decompose(A.astype(np.float64), ranks, iters=10000, seed=3)
    assert oracle.rel_error(A, cores) <= 1e-3
    for c in cores:
        assert np.all(c >= 0) and np.all(np.isfinite(c))
    for tr in traces:
        assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])


def test_nmf_exact_recovery_from_perturbed_truth():
    # stage-1 unfolding of a noise-free TT tensor: W* = G1, H* = (G2 G3) reshaped
    dims, ranks = (6, 6, 6), (1, 2, 2, 1)
    A, _, cores = synth.tt_tensor(dims, ranks, "uniform", noise=0.0, seed=21, return_cores=True)
    Ws = cores[0].reshape(6, 2)
    Hs = np.tensordot(cores[1], cores[2], axes=([2], [0])).reshape(2, 36)
    X = A.astype(np.float64).reshape(6, 36)
    rng = np.random.Generator(np.random.PCG64(0))
    W0 = Ws * (1 + 1e-3 * rng.random(Ws.shape))
    H0 = Hs * (1 + 1e-3 * rng.random(Hs.shape))
    W, H, tr = oracle.nmf_mu(X, W0, H0, 200)
    assert np.sqrt(2 * tr[-1]) / np.linalg.norm(X) <= 1e-5


def test_ntt_error_near_noise_level_c1():
    c = synth.CONFIGS["c1_8x4"]
    A, info = synth.tt_tensor(c["dims"], c["ranks"], c["core_dist"], c["noise"], c["data_seed"])
    cores, traces = oracle.ntt_decompose(A, c["ranks"], iters=c["iters"], seed=c["init_seed"])
    err = oracle.rel_error(A, cores)
    # noise of relative size ~1% (|N(0, (0.01 mean)^2)| has RMS 0.01 mean)
    assert err < 0.05
    assert all(np.all(g >= 0) for g in cores)
    ratio = oracle.compression_ratio(c["dims"], c["ranks"])
    assert ratio == 4096.0 / 192.0


def test_best_restart_rule():
    A = _rand((6, 6, 6), 23)
    cores1, tr1 = oracle.ntt_decompose(A, (1, 2, 2, 1), iters=20, seed=4, restarts=1)
    cores3, tr3 = oracle.ntt_decompose(A, (1, 2, 2, 1), iters=20, seed=4, restarts=3)
    assert tr3[0][-1] <= tr1[0][-1]


def test_rank_infeasible_rejected():
    with pytest.raises(ValueError):
        oracle.ntt_decompose(_rand((3, 4), 1), (1, 5, 1), iters=1)


# ---------------------------------------------------------------- synthetic inputs

def test_synth_tensor_recipe():
    dims, ranks = (4, 5, 6, 3), (1, 2, 3, 2, 1)
    A, info, cores = synth.tt_tensor(dims, ranks, "uniform", noise=0.0, seed=3, return_cores=True)
    ref = oracle.tt_full(cores)
    assert np.allclose(A, ref, rtol=1e-6, atol=0)
    assert abs(info["mean"] - ref.mean()) <= 1e-12 * ref.mean()
    An, info_n = synth.tt_tensor(dims, ranks, "uniform", noise=0.01, seed=3)
    d = An.astype(np.float64) - ref
    assert np.all(d >= -1e-6 * ref)                # |noise| is non-negative
    assert 0.3 * info_n["sigma"] < np.sqrt(np.mean(d * d)) < 3 * info_n["sigma"]
    A2, _ = synth.tt_tensor(dims, ranks, "uniform", noise=0.01, seed=3, threads=1)
    assert np.array_equal(An, A2)


def test_synth_instance_generators():
    inst = synth.batched_instances(64)
    for it in inst:
        d = len(it["dims"])
        assert 3 <= d <= 6 and all(8 <= n <= 24 for n in it["dims"])
        for k, (m, n, r) in enumerate(synth.stage_shapes(it["dims"], it["ranks"])):
            assert 1 <= r <= min(m, n)
    reqs = synth.serving_requests(50)
    for q in reqs:
        assert 4 <= len(q["dims"]) <= 7
        for (m, n, r) in synth.stage_shapes(q["dims"], q["ranks"]):
            assert 1 <= r <= min(m, n)


# ---------------------------------------------------------------- precision form

def test_bf16_round_fixed_points_and_ties():
    """Values with 8 significand bits are unchanged; halfway cases go to the even neighbour."""
    exact = np.array([1.0, 1.5, 1.0 + 2.0 ** -7, 3.0 * 2.0 ** 20, 2.0 ** -30, 255.0, 0.0, -6.5])
    assert np.array_equal(oracle.bf16_round(exact), exact)
    one = 1.0
    # 1 + 2^-8 is halfway between 1 (even) and 1 + 2^-7 (odd last bit) -> 1
    assert oracle.bf16_round(one + 2.0 ** -8) == 1.0
    # 1 + 3*2^-8 is halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even) -> 1 + 2^-6
    assert oracle.bf16_round(one + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    # just above / below a halfway point
    assert oracle.bf16_round(one + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert oracle.bf16_round(one + 2.0 ** -8 - 2.0 ** -20) == 1.0
    # carry into the next binade
    assert oracle.bf16_round(2.0 - 2.0 ** -9) == 2.0
    assert oracle.bf16_round(-(1.0 + 2.0 ** -8)) == -1.0


def test_bf16_round_matches_library_conversion():
    """Round-to-nearest-even FP32 -> bfloat16 of the library (torch, CPU) on random FP32 values."""
    torch = pytest.importorskip("torch")
    rng = np.random.Generator(np.random.PCG64(17))
    x = (rng.random(200000) * 10.0 ** rng.integers(-20, 20, 200000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.bf16_round(x.astype(np.float64)), ref)


def test_precision_form_reduces_to_fp32_form_on_bf16_exact_input():
    """With an input already representable in bfloat16 and no refinement, rounding is the
    identity at stage 1; the stage-1 core equals the FP32 form's."""
    dims, ranks = (6, 5, 4), (1, 3, 2, 1)
    A = oracle.bf16_round(synth.uniform_matrix((6, 20), 31)).reshape(dims)
    c32, _ = oracle.ntt_decompose(A, ranks, 8, seed=3, record=False)
    cbf, _ = oracle.ntt_decompose(A, ranks, 8, seed=3, record=False, x_precision="bf16")
    assert np.array_equal(c32[0], cbf[0])


def test_precision_form_refinement_lowers_the_fp64_objective():
    """The refinement iterations are plain MU on the unrounded unfolding, so they cannot
    raise its objective (MU is monotone): the stage-1 objective with refinement is no
    higher than without."""
    dims, ranks = (8, 7, 6), (1, 4, 3, 1)
    A = synth.uniform_matrix((8, 42), 5).reshape(dims)
    _, t0 = oracle.ntt_decompose(A, ranks, 20, seed=9, record=False, x_precision="bf16", refine=0)
    _, t5 = oracle.ntt_decompose(A, ranks, 20, seed=9, record=False, x_precision="bf16", refine=5)
    assert t5[0][-1] <= t0[0][-1]


# ---------------------------------------------------------------- Algorithm 2's rank rule

def test_singular_values_closed_forms():
    # [[3, 0], [4, 5]]: A^T A = [[25, 20], [20, 25]] has eigenvalues 45 and 5
    assert np.allclose(oracle.singular_values([[3.0, 0.0], [4.0, 5.0]]), [math.sqrt(45.0), math.sqrt(5.0)],
                       rtol=1e-14)
    # a rectangular diagonal matrix: the absolute diagonal, sorted
    D = np.zeros((3, 5))
    D[0, 0], D[1, 1], D[2, 2] = 1.0, -3.0, 2.0
    assert np.allclose(oracle.singular_values(D), [3.0, 2.0, 1.0], rtol=1e-14)
    # U diag(s) V^T with orthonormal U, V built by QR: exactly s
    rng = np.random.Generator(np.random.PCG64(3))
    U, _ = np.linalg.qr(rng.standard_normal((9, 4)))
    V, _ = np.linalg.qr(rng.standard_normal((13, 4)))
    s = np.array([5.0, 2.5, 0.75, 0.125])
    assert np.allclose(oracle.singular_values(U @ np.diag(s) @ V.T)[:4], s, rtol=1e-12)


def test_select_rank_hand_example():
    # sigma = (4, 2, 1, 1/2): sum of squares 21.25; tail ratios after k = 1..4:
    # sqrt(5.25/21.25) = 0.497, sqrt(1.25/21.25) = 0.2425, sqrt(0.25/21.25) = 0.1085, 0
    sig = [4.0, 2.0, 1.0, 0.5]
    for eps, k in ((1.0, 1), (0.5, 1), (0.49, 2), (0.3, 2), (0.2, 3), (0.11, 3), (0.1, 4), (0.0, 4)):
        assert oracle.select_rank(sig, eps) == k, eps
    assert oracle.select_rank(sig, 0.1, rank_cap=2) == 2
    assert oracle.select_rank([0.0, 0.0, 0.0], 0.1) == 1


def test_select_rank_brute_force_and_invariances():
    rng = np.random.Generator(np.random.PCG64(5))
    for trial in range(40):
        m, n = rng.integers(2, 9), rng.integers(2, 12)
        X = rng.random((m, n)) ** 3
        sig = oracle.singular_values(X)
        for eps in (0.3, 0.1, 0.03, 0.01):
            k = oracle.select_rank(sig, eps)
            # brute force over every candidate k: tail energy from the reversed cumulative sum
            tails = np.concatenate([np.cumsum((sig ** 2)[::-1])[::-1][1:], [0.0]])
            ok = [kk + 1 for kk in range(len(sig)) if math.sqrt(tails[kk] / np.sum(sig ** 2)) <= eps]
            assert k == min(ok)
            # scaling and transposing X change no singular value ratio
            assert oracle.select_rank(oracle.singular_values(7.5 * X.T), eps) == k


def test_select_rank_finds_exact_low_rank():
    rng = np.random.Generator(np.random.PCG64(7))
    for k in (1, 2, 5):
        X = rng.random((12, k)) @ rng.random((k, 40))
        assert oracle.select_rank(oracle.singular_values(X), 1e-8) == k


def test_ntt_rank_rule_first_stage_and_one_stage():
    # a noise-free TT tensor: X_1 has rank r_1 exactly, so a tiny eps picks r_1
    dims, ranks = (6, 5, 7), (1, 3, 2, 1)
    A = oracle.tt_full(synth.tt_cores(dims, ranks, "uniform", seed=17))
    cores, _ = oracle.ntt_decompose(A, None, 20, seed=1, eps_rank=1e-9)
    assert cores[0].shape[2] == 3
    # d = 2: one stage, the rank of the rule on A itself
    B = synth.uniform_matrix((9, 14), 4).astype(np.float64)
    for eps in (0.5, 0.2, 0.05):
        k = oracle.select_rank(oracle.singular_values(B), eps)
        cores, _ = oracle.ntt_decompose(B, None, 5, seed=1, eps_rank=eps)
        assert cores[0].shape == (1, 9, k) and cores[1].shape == (k, 14, 1)


# ---------------------------------------------------------------- Algorithm 3 (BCD)

def test_spectral_norm_is_the_two_norm():
    rng = np.random.Generator(np.random.PCG64(8))
    for n in (1, 3, 8):
        B = rng.random((n, 2 * n))
        M = B @ B.T
        assert abs(oracle.spectral_norm_sym(M) - np.linalg.norm(M, 2)) <= 1e-12 * np.linalg.norm(M, 2)


def test_bcd_first_w_step_is_least_squares_for_orthogonal_h():
    """H with disjoint row supports and equal row norms: H H^T = c I, the
    Lipschitz step 1/c makes the first W step the unconstrained least-squares
    solution X H^T (H H^T)^-1, which is non-negative here (numpy lstsq)."""
    rng = np.random.Generator(np.random.PCG64(9))
    m, r, per = 7, 3, 5
    n = r * per
    H0 = np.zeros((r, n))
    for k in range(r):
        v = rng.random(per) + 0.1
        H0[k, k * per:(k + 1) * per] = v / np.linalg.norm(v)
    X = rng.random((m, n))
    W0 = rng.random((m, r))
    W, H, tr, acc = oracle.bcd_nmf(X, W0, H0, 1)
    assert acc[0]
    Hm = H0 / np.linalg.norm(H0) * math.sqrt(np.linalg.norm(X))   # Algorithm 3's normalisation
    W_ls = np.linalg.lstsq(Hm.T, X.T, rcond=None)[0].T
    assert np.allclose(W, W_ls, rtol=1e-12, atol=1e-14)


def test_bcd_rank_one_exact_factorisation_is_a_fixed_point():
    rng = np.random.Generator(np.random.PCG64(10))
    u, v = rng.random((6, 1)) + 0.1, rng.random((1, 9)) + 0.1
    X = u @ v
    W, H, tr, acc = oracle.bcd_nmf(X, 3.0 * u, 0.5 * v, 20)
    assert np.allclose(W @ H, X, rtol=1e-12)
    assert tr[-1] <= 1e-24 * np.sum(X ** 2)


def test_bcd_objective_monotone_converges_and_rejections_restore():
    rng = np.random.Generator(np.random.PCG64(11))
    X = rng.random((10, 4)) @ rng.random((4, 30))
    W0, H0 = oracle.init_factors(10, 30, 4, seed=3, stage=0)
    W, H, tr, acc = oracle.bcd_nmf(X, W0, H0, 400)
    assert np.all(np.diff(tr) <= 0.0)                              # accepted objectives never rise
    assert tr[-1] <= 1e-6 * 0.5 * np.sum(X ** 2)                  # exact low-rank data: converges
    assert np.all(W >= 0) and np.all(H >= 0)
    assert np.allclose(oracle.objective(X, W, H), tr[-1], rtol=1e-12)
    # a rejected iteration leaves the factors where the previous iteration left them
    rej = [i for i in range(1, len(acc)) if not acc[i]]
    assert rej, "the extrapolation produced no rejected iteration on this case"
    for i in rej[:3]:
        Wa, Ha, _, _ = oracle.bcd_nmf(X, W0, H0, i)
        Wb, Hb, _, _ = oracle.bcd_nmf(X, W0, H0, i + 1)
        assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)


def test_ntt_bcd_solver_d2_is_one_bcd_nmf():
    X = synth.uniform_matrix((8, 21), 12).astype(np.float64)
    cores, tr = oracle.ntt_decompose(X, (1, 3, 1), 50, seed=6, solver="bcd")
    W0, H0 = oracle.init_factors(8, 21, 3, seed=6, stage=0)
    W, H, t2, _ = oracle.bcd_nmf(X, W0, H0, 50)
    Wn, Hn = oracle.handoff_normalize(W, H)
    assert np.allclose(cores[0].reshape(8, 3), Wn, rtol=1e-14) and np.allclose(cores[1].reshape(3, 21), Hn)
    assert np.array_equal(tr[0], t2)

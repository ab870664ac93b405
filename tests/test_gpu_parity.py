"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (all stated per test):
  * RNG initialisation: bit-exact.
  * multiplicative-update iterates from identical W0, H0: relative Frobenius
    difference <= 1e-4 after 10 updates, for W and for H (FP32 path against
    the FP64 oracle on the same FP32 input).
  * final relative reconstruction error of a whole nTT within 1e-3 absolute
    of the oracle's.
  * BF16-stored X: iterates within 1e-4 of the oracle run on the BF16-rounded
    X; error against the FP32-X oracle stated and bounded by 5e-3.
  * reconstruction (Eq. 2): relative difference <= 1e-5 per entry.
"""

import math
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_ITERATE = 1e-4
ABS_FINAL_EPS = 1e-3
REL_BF16_VS_FP64 = 5e-3


@pytest.fixture(scope="module")
def ntt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2008_01340_gb300 as mod
    mod.build()
    mod.lib()
    return mod


def _fro_rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _x_matrix(kind, m, n, seed):
    if kind == "uniform":
        return synth.uniform_matrix((m, n), seed)
    # low-rank non-negative plus noise: product of random factors
    rng = np.random.Generator(np.random.PCG64(seed))
    k = max(1, min(m, 6))
    X = rng.random((m, k)) @ rng.random((k, n))
    X += 0.01 * X.mean() * np.abs(rng.standard_normal(X.shape))
    return X.astype(np.float32)


# ------------------------------------------------------------------ RNG

@pytest.mark.parametrize("count", [1, 255, 4096, 100003])
def test_uniform_init_bit_exact(ntt, count):
    for (seed, stage, restart, mtx) in [(0, 0, 0, 0), (102, 3, 0, 1), (2**63 + 5, 7, 5, 1)]:
        out = torch.empty(count, dtype=torch.float32, device="cuda")
        ntt.ntt_uniform_init(seed, stage, restart, mtx, out)
        key = oracle.stream_key(seed, stage, restart, mtx)
        ref = oracle.uniform01(key, np.arange(count, dtype=np.uint64)).astype(np.float32)
        assert np.array_equal(out.cpu().numpy(), ref)


# ------------------------------------------------------------------ one NMF

SHAPES = [
    # (m, n, r, kind)   n % 4 == 0 -> TMA tiles, otherwise cooperative loads
    (32, 40000, 8, "lowrank"),       # MP=32, R=8, ragged last tile
    (32, 116813, 8, "uniform"),      # several tiles per CTA, odd n
    (8, 512, 3, "lowrank"),          # C1 stage 1
    (24, 777, 3, "uniform"),         # odd n, r < 8
    (16, 4096, 16, "uniform"),       # full-rank stage (r = m)
    (100, 5000, 5, "lowrank"),       # MP=128
    (64, 10000, 20, "uniform"),      # MP=64, R=32
    (256, 3000, 16, "lowrank"),      # MP=256, ragged tile
    (300, 2050, 12, "uniform"),      # MP=512, R=16, n % 4 == 2
    (512, 1000, 32, "uniform"),      # MP=512, R=32
    (1, 999, 1, "uniform"),          # degenerate m = r = 1
]


def _run_gpu_mu(ntt, X, W0, H0, iters, obj=True, route="auto", engine=None):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Wd = torch.from_numpy(W0.astype(np.float32)).cuda()
    Hd = torch.from_numpy(H0.astype(np.float32)).cuda()
    od = torch.zeros(max(iters, 1), dtype=torch.float64, device="cuda") if obj else None
    ws = ntt.nmf_mu_step(Xd, Wd, Hd, iters, 1e-12, od, route=route, engine=engine)
    torch.cuda.synchronize()
    assert ntt.ntt_status_of_workspace(ws) == "NTT_OK"
    return Wd.cpu().numpy(), Hd.cpu().numpy(), (od.cpu().numpy() if obj else None)


@pytest.mark.parametrize("m,n,r,kind", SHAPES)
def test_mu_iterates_match_oracle(ntt, m, n, r, kind):
    X = _x_matrix(kind, m, n, seed=m * 7919 + n)
    W0 = synth.uniform_matrix((m, r), seed=11 + m)
    H0 = synth.uniform_matrix((r, n), seed=13 + n)
    iters = 10
    Wg, Hg, og = _run_gpu_mu(ntt, X, W0, H0, iters)
    Wo, Ho, tr = oracle.nmf_mu(X.astype(np.float64), W0, H0, iters)
    assert _fro_rel(Wg, Wo) <= REL_ITERATE
    assert _fro_rel(Hg, Ho) <= REL_ITERATE
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    # expanded Gram-form objective (FP64 combine) against the direct FP64 objective
    assert np.allclose(og, tr, rtol=2e-3, atol=1e-6 * float(np.sum(X.astype(np.float64) ** 2)))


def test_mu_single_iteration_every_entry(ntt):
    # one iteration: element-by-element comparison, every entry of W and H
    m, n, r = 32, 10000, 8
    X = _x_matrix("lowrank", m, n, 5)
    W0 = synth.uniform_matrix((m, r), 6)
    H0 = synth.uniform_matrix((r, n), 7)
    Wg, Hg, _ = _run_gpu_mu(ntt, X, W0, H0, 1)
    Wo, Ho, _ = oracle.nmf_mu(X.astype(np.float64), W0, H0, 1)
    assert np.allclose(Hg, Ho, rtol=1e-5, atol=1e-6 * Ho.max())
    assert np.allclose(Wg, Wo, rtol=1e-5, atol=1e-6 * Wo.max())


def test_mu_zero_iterations_and_zero_columns(ntt):
    m, n, r = 16, 1000, 4
    X = _x_matrix("uniform", m, n, 1)
    X[:, 100:200] = 0.0                       # columns of zeros -> H columns go to 0
    X[3, :] = 0.0                             # a row of zeros -> that W row goes to 0
    W0 = synth.uniform_matrix((m, r), 2)
    H0 = synth.uniform_matrix((r, n), 3)
    Wg, Hg, _ = _run_gpu_mu(ntt, X, W0, H0, 0, obj=False)
    assert np.array_equal(Wg, W0) and np.array_equal(Hg, H0)
    Wg, Hg, _ = _run_gpu_mu(ntt, X, W0, H0, 5)
    Wo, Ho, _ = oracle.nmf_mu(X.astype(np.float64), W0, H0, 5)
    assert np.all(Hg[:, 100:200] == 0.0) and np.all(Wg[3] == 0.0)
    assert _fro_rel(Wg, Wo) <= REL_ITERATE and _fro_rel(Hg, Ho) <= REL_ITERATE


def test_mu_deterministic(ntt):
    m, n, r = 32, 60000, 8
    X = _x_matrix("lowrank", m, n, 9)
    W0 = synth.uniform_matrix((m, r), 10)
    H0 = synth.uniform_matrix((r, n), 11)
    a = _run_gpu_mu(ntt, X, W0, H0, 7)
    b = _run_gpu_mu(ntt, X, W0, H0, 7)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# (256, 4096, 16), (128, 10000, 32), (200, 4104, 20), (130, 1032, 16) run on the
# BF16 tensor-core pass (128/256-row buckets, ranks 16/32, ragged last tiles,
# rows past m); the 16/32-row shapes on the FMA passes by default
@pytest.mark.parametrize("m,n,r", [(32, 40000, 8), (256, 4096, 16), (16, 8192, 16), (128, 10000, 32),
                                   (200, 4104, 20), (130, 1032, 16), (32, 20008, 32), (12, 4096, 12)])
def test_mu_bf16_x(ntt, m, n, r):
    X = _x_matrix("lowrank", m, n, 21)
    Xb = torch.from_numpy(X).to(torch.bfloat16)            # RN-even rounding of the input
    Xb64 = Xb.to(torch.float64).numpy()
    W0 = synth.uniform_matrix((m, r), 22)
    H0 = synth.uniform_matrix((r, n), 23)
    Wd = torch.from_numpy(W0).cuda()
    Hd = torch.from_numpy(H0).cuda()
    ws = ntt.nmf_mu_step(Xb.cuda(), Wd, Hd, 10)
    torch.cuda.synchronize()
    Wo, Ho, _ = oracle.nmf_mu(Xb64, W0, H0, 10)
    assert _fro_rel(Wd.cpu().numpy(), Wo) <= REL_ITERATE
    assert _fro_rel(Hd.cpu().numpy(), Ho) <= REL_ITERATE
    # stated error of the BF16-stored path against FP64 on the original FP32 X
    Wf, Hf, _ = oracle.nmf_mu(X.astype(np.float64), W0, H0, 10)
    e_w = _fro_rel(Wd.cpu().numpy(), Wf)
    e_h = _fro_rel(Hd.cpu().numpy(), Hf)
    print(f"bf16 X ({m}x{n}, r={r}): iterate error vs FP64 oracle W {e_w:.2e} H {e_h:.2e}")
    assert e_w <= REL_BF16_VS_FP64 and e_h <= REL_BF16_VS_FP64


# ------------------------------------------------------------------ whole nTT

def _decompose(ntt, A, ranks, iters, seed, x_dtype="f32", refine=0, tol=0.0, check_every=10, route="auto",
               eager=False):
    dims = A.shape
    plan = ntt.ntt_plan_create(dims, ranks, iters, 1e-12, x_dtype, refine, seed, tol, check_every, route, eager)
    ws = ntt.empty_workspace(plan.workspace_size())
    cores = [torch.empty(s, dtype=torch.float32, device="cuda") for s in plan.core_shapes()]
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    ntt.ntt_decompose(plan, Ad, cores, ws)
    stats = ntt.ntt_plan_get_stats(plan)
    return [c.cpu().numpy() for c in cores], stats, plan, Ad, ws


def test_ntt_c1_per_iterate(ntt):
    c = synth.CONFIGS["c1_8x4"]
    A, _ = synth.tt_tensor(c["dims"], c["ranks"], c["core_dist"], c["noise"], c["data_seed"])
    cores_g, stats, *_ = _decompose(ntt, A, c["ranks"], 10, c["init_seed"])
    cores_o, traces = oracle.ntt_decompose(A, c["ranks"], 10, seed=c["init_seed"])
    assert stats["status"] == "NTT_OK"
    for k, (g, o) in enumerate(zip(cores_g, cores_o)):
        assert _fro_rel(g, o) <= REL_ITERATE * (k + 1), f"core {k}"
    for s, st in enumerate(stats["stages"]):
        assert abs(st["resid"] - traces[s][-1]) <= 1e-3 * traces[s][-1]


def test_ntt_c1_full_config(ntt):
    c = synth.CONFIGS["c1_8x4"]
    A, _ = synth.tt_tensor(c["dims"], c["ranks"], c["core_dist"], c["noise"], c["data_seed"])
    cores_g, stats, plan, Ad, _ = _decompose(ntt, A, c["ranks"], c["iters"], c["init_seed"])
    cores_o, _ = oracle.ntt_decompose(A, c["ranks"], c["iters"], seed=c["init_seed"], record=False)
    eg = oracle.rel_error(A, cores_g)
    eo = oracle.rel_error(A, cores_o)
    assert abs(eg - eo) <= ABS_FINAL_EPS
    assert all(np.all(g >= 0) and np.all(np.isfinite(g)) for g in cores_g)
    # the device relative error (Eq. 3) agrees with the oracle's on the GPU cores
    err = torch.zeros(3, dtype=torch.float64, device="cuda")
    ntt.ntt_rel_error(c["dims"], c["ranks"], [torch.from_numpy(g).cuda() for g in cores_g], Ad, err)
    assert abs(err[0].item() - eg) <= 1e-6


def test_ntt_c2_recipe_16x6(ntt):
    # the 32^6 recipe scaled to 16^6 so the oracle finishes end to end
    c = synth.CONFIGS["c2_small_16x6"]
    A, _ = synth.tt_tensor(c["dims"], c["ranks"], c["core_dist"], c["noise"], c["data_seed"])
    cores_g, stats, *_ = _decompose(ntt, A, c["ranks"], c["iters"], c["init_seed"])
    cores_o, _ = oracle.ntt_decompose(A, c["ranks"], c["iters"], seed=c["init_seed"], record=False)
    eg, eo = oracle.rel_error(A, cores_g), oracle.rel_error(A, cores_o)
    print(f"16^6 rel error gpu {eg:.6f} oracle {eo:.6f}")
    assert abs(eg - eo) <= ABS_FINAL_EPS


def test_ntt_bf16_form_small(ntt):
    dims, ranks = (16, 16, 16, 16), (1, 8, 16, 8, 1)
    A, _ = synth.tt_tensor(dims, ranks, "exponential", 0.01, seed=3)
    cores_g, stats, *_ = _decompose(ntt, A, ranks, 100, 103, x_dtype="bf16", refine=5)
    cores_o, _ = oracle.ntt_decompose(A, ranks, 105, seed=103, record=False)
    eg, eo = oracle.rel_error(A, cores_g), oracle.rel_error(A, cores_o)
    print(f"bf16 form rel error gpu {eg:.6f} fp64 oracle (105 FP32 iterations) {eo:.6f}")
    assert abs(eg - eo) <= REL_BF16_VS_FP64
    assert stats["status"] == "NTT_OK"


def _clear_stops(traces, tol, K, iters, margin=1.1):
    """True when every stage's stopping decision under the oracle's trace is
    clear by `margin` on both sides of tol (so FP32 rounding cannot flip it)."""
    for tr in traces:
        u = len(tr)
        for v in range(2 * K, u + 1, K):
            dec = (tr[v - K - 1] - tr[v - 1]) / abs(tr[v - K - 1])
            if v < u and not dec > margin * tol:
                return False
            if v == u and u < iters and not dec < tol / margin:
                return False
    return any(len(t) < iters for t in traces)


@pytest.mark.parametrize("x_dtype,refine", [("f32", 0), ("bf16", 4)])
def test_ntt_stopping_test_matches_oracle(ntt, x_dtype, refine):
    """With tol > 0 each stage's main loop stops at the check where the
    objective's relative decrease over K iterations first falls below tol:
    the same iteration as the oracle's rule on its FP64 trace (tol chosen so
    that every decision is clear of rounding), refinement iterations run in
    full, and the result's Eq. (3) error matches the oracle's within 1e-3.
    Uniform (not low-rank) data keeps the objective a sizeable fraction of
    ||X||^2, where the FP64 Gram-form objective resolves small decreases."""
    dims, ranks = (12, 10, 48), (1, 3, 2, 1)
    A = synth.uniform_matrix((1, int(np.prod(dims))), 71).reshape(dims)
    K, iters = 10, 400
    chosen = None
    for tol in np.geomspace(1e-4, 3e-3, 40):
        cores_o, traces = oracle.ntt_decompose(A, ranks, iters, seed=4, tol=tol, check_every=K,
                                               x_precision=x_dtype, refine=refine)
        main = [t[:len(t) - refine] for t in traces]
        if _clear_stops(main, tol, K, iters):
            chosen = tol
            break
    assert chosen is not None, "no tol with clear stopping decisions"
    cores_g, stats, plan, Ad, ws = _decompose(ntt, A, ranks, iters, 4, x_dtype=x_dtype, refine=refine,
                                              tol=chosen, check_every=K)
    assert stats["status"] == "NTT_OK"
    assert [st["iters"] for st in stats["stages"]] == [len(t) for t in traces]
    err = torch.zeros(3, dtype=torch.float64, device="cuda")
    cg = [torch.from_numpy(c).cuda() for c in cores_g]
    ntt.ntt_rel_error(dims, ranks, cg, Ad, err)
    e_o = oracle.rel_error(A.astype(np.float64), cores_o)
    assert abs(err[0].item() - e_o) <= ABS_FINAL_EPS
    # tol = 0: every stage runs the fixed count
    _, stats0, *_ = _decompose(ntt, A, ranks, iters, 4, x_dtype=x_dtype, refine=refine)
    assert [st["iters"] for st in stats0["stages"]] == [iters + refine] * 2


HOST_CASES = [
    # (dims, ranks, x_dtype, refine): small ranks (single-problem passes only);
    # a first stage routed to the grouped engine (16 rows, rank 16); the
    # precision form with a BF16 tensor-core stage and grouped stages
    ((8, 9, 10, 7), (1, 4, 5, 3, 1), "f32", 0),
    ((16, 16, 16, 16), (1, 16, 16, 16, 1), "f32", 0),
    ((16, 8, 16, 16), (1, 16, 16, 16, 1), "bf16", 2),
]


@pytest.mark.parametrize("dims,ranks,x_dtype,refine", HOST_CASES)
def test_ntt_host_variant_equals_device(ntt, dims, ranks, x_dtype, refine):
    """Host-buffer calls issued back to back (A1, A2, A1, no sync between them:
    the input copies alternate between two slots and overlap the previous
    call's compute; each slot has its own cached graph and table upload) each
    give exactly the device-buffer result of their input."""
    A1, _ = synth.tt_tensor(dims, ranks, "uniform", 0.01, seed=8)
    A2, _ = synth.tt_tensor(dims, ranks, "uniform", 0.01, seed=9)
    ref = [_decompose(ntt, A, ranks, 30, 5, x_dtype=x_dtype, refine=refine)[0] for A in (A1, A2)]
    plan = ntt.ntt_plan_create(dims, ranks, 30, 1e-12, x_dtype, refine, 5)
    ws = ntt.empty_workspace(plan.workspace_size_host())
    Ah = [torch.from_numpy(A).pin_memory() for A in (A1, A2)]
    outs = []
    for which in (0, 1, 0):
        ch = [torch.empty(s, dtype=torch.float32).pin_memory() for s in plan.core_shapes()]
        ntt.ntt_decompose_host(plan, Ah[which], ch, ws)
        outs.append((which, ch))
    torch.cuda.synchronize()
    for which, ch in outs:
        for a, b in zip(ref[which], ch):
            assert np.array_equal(a, b.numpy())


@pytest.mark.parametrize("dims,ranks,x_dtype,refine", HOST_CASES[1:])
def test_ntt_alternating_workspaces_and_recapture(ntt, dims, ranks, x_dtype, refine):
    """Device-buffer calls of one plan on three (A, workspace) pairs issued back
    to back without a sync (the third capture replaces a cached graph whose
    launch may still be queued), then the first pair again: every call gives
    bitwise the result of a fresh plan on its input."""
    As = [synth.tt_tensor(dims, ranks, "uniform", 0.01, seed=s)[0] for s in (21, 22, 23)]
    ref = [_decompose(ntt, A, ranks, 20, 6, x_dtype=x_dtype, refine=refine)[0] for A in As]
    plan = ntt.ntt_plan_create(dims, ranks, 20, 1e-12, x_dtype, refine, 6)
    wss = [ntt.empty_workspace(plan.workspace_size()) for _ in range(3)]
    Ads = [torch.from_numpy(A).cuda() for A in As]
    outs = []
    for which in (0, 1, 2, 0, 1):
        cores = [torch.empty(s, dtype=torch.float32, device="cuda") for s in plan.core_shapes()]
        ntt.ntt_decompose(plan, Ads[which], cores, wss[which])
        outs.append((which, cores))
    torch.cuda.synchronize()
    for which, cores in outs:
        for a, b in zip(ref[which], cores):
            assert np.array_equal(a, b.cpu().numpy())


def test_ntt_eager_equals_graph(ntt):
    """A plan with NTT_PLAN_EAGER (every launch enqueued per call) gives bitwise
    the cached-graph result, on a plan with a grouped-engine stage."""
    dims, ranks = (16, 16, 16, 16), (1, 16, 16, 16, 1)
    A, _ = synth.tt_tensor(dims, ranks, "uniform", 0.01, seed=24)
    a = _decompose(ntt, A, ranks, 15, 3)[0]
    b = _decompose(ntt, A, ranks, 15, 3, eager=True)[0]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_ntt_repeat_is_bitwise_identical(ntt):
    dims, ranks = (12, 10, 14, 9), (1, 5, 6, 4, 1)
    A, _ = synth.tt_tensor(dims, ranks, "uniform", 0.01, seed=31)
    plan = ntt.ntt_plan_create(dims, ranks, 40, 1e-12, "f32", 0, 7)
    ws = ntt.empty_workspace(plan.workspace_size())
    Ad = torch.from_numpy(A).cuda()
    outs = []
    for _ in range(2):
        cores = [torch.empty(s, dtype=torch.float32, device="cuda") for s in plan.core_shapes()]
        ntt.ntt_decompose(plan, Ad, cores, ws)
        torch.cuda.synchronize()
        outs.append([c.cpu().numpy() for c in cores])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


# ------------------------------------------------------------------ Eq. (2), Eq. (3)

@pytest.mark.parametrize("dims,ranks", [((5, 7, 3, 6), (1, 2, 3, 2, 1)),
                                        ((8, 8, 8, 8), (1, 3, 3, 3, 1)),
                                        ((3, 250, 3), (1, 3, 2, 1)),
                                        ((17, 19), (1, 5, 1))])
def test_reconstruct_and_rel_error(ntt, dims, ranks):
    cores = [c.astype(np.float32) for c in synth.tt_cores(dims, ranks, "uniform", seed=41)]
    ref = oracle.tt_full([c.astype(np.float64) for c in cores])
    cd = [torch.from_numpy(c).cuda() for c in cores]
    out = torch.empty(math.prod(dims), dtype=torch.float32, device="cuda")
    ntt.ntt_reconstruct(dims, ranks, cd, out)
    got = out.cpu().numpy().reshape(dims)
    assert np.allclose(got, ref, rtol=1e-5, atol=0)
    A = (ref * (1.0 + 0.05 * synth.uniform_matrix(ref.shape, 3))).astype(np.float32)
    err = torch.zeros(3, dtype=torch.float64, device="cuda")
    ntt.ntt_rel_error(dims, ranks, cd, torch.from_numpy(A.ravel()).cuda(), err)
    eo = oracle.rel_error(A, cores)
    assert abs(err[0].item() - eo) <= 1e-5 * eo


# ------------------------------------------------------------------ full size, bench launch config

@pytest.fixture(scope="module")
def c2_full():
    c = synth.CONFIGS["c2_32x6"]
    A, info = synth.tt_tensor(c["dims"], c["ranks"], c["core_dist"], c["noise"], c["data_seed"])
    return c, A


def test_c2_full_size_first_iteration_sampled(ntt, c2_full):
    """Stage 1 of the 32^6 workload (32 x 33,554,432, r = 8), one MU iteration
    from the counter-RNG init in the launch configuration of the benchmark:
    H checked on sampled columns (each column of the H update is independent
    given W0), W against the oracle's full FP64 P = X H^T and Q = H H^T."""
    c, A = c2_full
    m, n, r = 32, 32 ** 5, 8
    seed = c["init_seed"]
    X = A.reshape(m, n)
    Xd = torch.from_numpy(X).cuda()
    Wd = torch.empty((m, r), dtype=torch.float32, device="cuda")
    Hd = torch.empty((r, n), dtype=torch.float32, device="cuda")
    ntt.ntt_uniform_init(seed, 0, 0, 0, Wd)
    ntt.ntt_uniform_init(seed, 0, 0, 1, Hd)
    ntt.nmf_mu_step(Xd, Wd, Hd, 1)
    torch.cuda.synchronize()
    W0 = oracle.uniform01(oracle.stream_key(seed, 0, 0, 0), np.arange(m * r, dtype=np.uint64)).reshape(m, r)
    G = W0.T @ W0
    # oracle H1 and P, Q in column chunks (FP64)
    P = np.zeros((m, r))
    Q = np.zeros((r, r))
    rng = np.random.Generator(np.random.PCG64(0))
    sample = np.sort(rng.choice(n, size=4096, replace=False))
    Hg = Hd.cpu().numpy()
    chunk = 1 << 21
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        Xc = X[:, c0:c1].astype(np.float64)
        H0c = oracle.init_columns_H(n, r, seed, 0, np.arange(c0, c1))
        H1c = np.maximum(0.0, H0c * (W0.T @ Xc) / (G @ H0c + 1e-12))
        P += Xc @ H1c.T
        Q += H1c @ H1c.T
        sel = sample[(sample >= c0) & (sample < c1)]
        if sel.size:
            assert np.allclose(Hg[:, sel], H1c[:, sel - c0], rtol=1e-5, atol=1e-7 * H1c.max())
    W1 = np.maximum(0.0, W0 * P / (W0 @ Q + 1e-12))
    assert _fro_rel(Wd.cpu().numpy(), W1) <= REL_ITERATE


def _golden_c2_rel_error():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_32x6_oracle.txt")
    with open(path) as f:
        for line in f:
            if line.startswith("rel_error "):
                return float(line.split()[1])
    raise AssertionError("no rel_error line in " + path)


def test_c2_full_size_decompose_properties(ntt, c2_full):
    """The whole 32^6 decomposition as the benchmark runs it: non-negative
    cores, non-increasing objective traces, Gram-form objective consistent
    with the direct FP64 residual, and its Eq. (3) relative error within
    ABS_FINAL_EPS of the FP64 oracle's whole decomposition of the same tensor
    from the same initial factors (tests/golden/c2_32x6_oracle.txt, written by
    tests/golden/make_c2_32x6_oracle.py, which calls only the oracle)."""
    c, A = c2_full
    plan = ntt.ntt_plan_create(c["dims"], c["ranks"], c["iters"], 1e-12, "f32", 0, c["init_seed"])
    ws = ntt.empty_workspace(plan.workspace_size())
    cores = [torch.empty(s, dtype=torch.float32, device="cuda") for s in plan.core_shapes()]
    Ad = torch.from_numpy(A.ravel()).cuda()
    ntt.ntt_decompose(plan, Ad, cores, ws)
    stats = ntt.ntt_plan_get_stats(plan)
    assert stats["status"] == "NTT_OK"
    for cc in cores:
        assert bool(torch.all(cc >= 0)) and bool(torch.all(torch.isfinite(cc)))
    for s, st in enumerate(stats["stages"]):
        # expanded Gram form at the last iteration vs direct residual (1% noise: f ~ 1e-4 ||X||^2)
        assert abs(st["obj_last"] - st["resid"]) <= 2e-2 * st["resid"] + 1e-7 * st["xnorm2"]
    err = torch.zeros(3, dtype=torch.float64, device="cuda")
    ntt.ntt_rel_error(c["dims"], c["ranks"], cores, Ad, err)
    e = err[0].item()
    eo = _golden_c2_rel_error()
    print(f"32^6 relative error {e:.6f} (oracle {eo:.6f}), total {stats['total_ms']:.1f} ms")
    assert 0.0 < e < 0.05
    assert abs(e - eo) <= ABS_FINAL_EPS


@pytest.mark.parametrize("m,n,r", [(32, 70000, 8), (16, 20000, 16), (24, 9000, 8), (32, 8192, 12),
                                   (32, 9000 * 128, 8)])
def test_tensor_core_and_fma_passes_agree(ntt, m, n, r):
    """The stacked split tensor-core form (m <= 32, r <= 16, route "tc") and
    the default FMA pass both match the oracle's iterates within the FP32
    tolerance."""
    X = _x_matrix("lowrank", m, n, 77 + m)
    W0 = synth.uniform_matrix((m, r), 78)
    H0 = synth.uniform_matrix((r, n), 79)
    eng = []
    Wt, Ht, _ = _run_gpu_mu(ntt, X, W0, H0, 10, route="tc", engine=eng)
    assert eng == ["tc_split"]
    Wf, Hf, _ = _run_gpu_mu(ntt, X, W0, H0, 10)
    Wo, Ho, _ = oracle.nmf_mu(X.astype(np.float64), W0, H0, 10)
    for Wg, Hg in ((Wt, Ht), (Wf, Hf)):
        assert _fro_rel(Wg, Wo) <= REL_ITERATE
        assert _fro_rel(Hg, Ho) <= REL_ITERATE


# (m, n, r): 32 and 16-row buckets, m and r below the bucket, a ragged last
# 32-column box, fewer boxes than warps, and many boxes per warp
@pytest.mark.parametrize("m,n,r", [(32, 40000, 8), (20, 36004, 5), (16, 8196, 8), (9, 100, 2),
                                   (32, 64, 8), (32, 2_000_000, 8), (1, 4096, 1)])
def test_narrow_and_wide_passes_agree(ntt, m, n, r):
    """The warp-streamed FMA pass (FP32 X, <= 32 rows, rank <= 8: route "fma")
    and the generic pass (route "generic") both match the oracle's iterates
    within the FP32 tolerance, and the narrow pass repeats bitwise."""
    X = _x_matrix("lowrank", m, n, 91 + m)
    W0 = synth.uniform_matrix((m, r), 92)
    H0 = synth.uniform_matrix((r, n), 93)
    eng = []
    Wn, Hn, on = _run_gpu_mu(ntt, X, W0, H0, 10, engine=eng, route="fma")
    Wn2, Hn2, _ = _run_gpu_mu(ntt, X, W0, H0, 10, route="fma")
    assert np.array_equal(Wn, Wn2) and np.array_equal(Hn, Hn2)
    Ww, Hw, _ = _run_gpu_mu(ntt, X, W0, H0, 10, route="generic", engine=eng)
    if n % 4 == 0:   # TMA-aligned rows: the narrow pass takes the FMA route
        assert eng == ["fma_narrow", "fma_pass"]
    Wo, Ho, tr = oracle.nmf_mu(X.astype(np.float64), W0, H0, 10)
    for Wg, Hg in ((Wn, Hn), (Ww, Hw)):
        assert _fro_rel(Wg, Wo) <= REL_ITERATE
        assert _fro_rel(Hg, Ho) <= REL_ITERATE
        assert np.all(Wg >= 0) and np.all(Hg >= 0)
    assert np.allclose(on, tr, rtol=2e-3, atol=1e-6 * float(np.sum(X.astype(np.float64) ** 2)))


def test_narrow_pass_reported_for_first_stage(ntt):
    """A 32-row, rank-8 first stage of a plan runs on the warp-level MMA form
    by default and on the narrow FMA pass with route "fma", and says so."""
    dims, ranks = (32, 16, 16, 8), (1, 8, 8, 4, 1)
    A, _ = synth.tt_tensor(dims, ranks, "uniform", 0.01, seed=5)
    cores, stats, *_ = _decompose(ntt, A, ranks, 5, 3)
    assert stats["status"] == "NTT_OK"
    assert stats["stages"][0]["engine"] == "tc_narrow"
    cores_f, stats_f, *_ = _decompose(ntt, A, ranks, 5, 3, route="fma")
    assert stats_f["stages"][0]["engine"] == "fma_narrow"
    cores_o, _ = oracle.ntt_decompose(A, ranks, 5, seed=3)
    for k, (g, f, o) in enumerate(zip(cores, cores_f, cores_o)):
        assert _fro_rel(g, o) <= REL_ITERATE * (k + 1), f"core {k}"
        assert _fro_rel(f, o) <= REL_ITERATE * (k + 1), f"core {k}"


# (m, n, r): 32 rows, rows below the bucket (17 .. 31), rank below the bucket,
# one 64-column stage, fewer stages than warps, many stages per warp
@pytest.mark.parametrize("m,n,r,kind", [(32, 40000, 8, "lowrank"), (32, 1 << 18, 8, "uniform"),
                                        (20, 64 * 500, 6, "lowrank"), (17, 64 * 70, 8, "uniform"),
                                        (32, 64, 8, "uniform"), (24, 1_999_936, 5, "lowrank"),
                                        (32, 64 * 1217, 1, "uniform")])
def test_mu_fp32_warp_mma_form(ntt, m, n, r, kind):
    """FP32 X of 17..32 rows at rank <= 8, n a multiple of 64: the default
    route runs the warp-level MMA form on X split once into bf16(X) and
    bf16(X - bf16(X)); iterates within the FP32 bound of the FP64 oracle on
    the unsplit X after 10 updates, the engine reported, a bitwise repeat."""
    X = _x_matrix(kind, m, n, 23 + m)
    W0 = synth.uniform_matrix((m, r), 24)
    H0 = synth.uniform_matrix((r, n), 25)
    eng = []
    Wg, Hg, og = _run_gpu_mu(ntt, X, W0, H0, 10, engine=eng)
    assert eng == ["tc_narrow"]
    Wg2, Hg2, _ = _run_gpu_mu(ntt, X, W0, H0, 10)
    assert np.array_equal(Wg, Wg2) and np.array_equal(Hg, Hg2)
    Wo, Ho, tr = oracle.nmf_mu(X.astype(np.float64), W0, H0, 10)
    assert _fro_rel(Wg, Wo) <= REL_ITERATE, _fro_rel(Wg, Wo)
    assert _fro_rel(Hg, Ho) <= REL_ITERATE, _fro_rel(Hg, Ho)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    assert np.allclose(og, tr, rtol=2e-3, atol=1e-6 * float(np.sum(X.astype(np.float64) ** 2)))


@pytest.mark.parametrize("m,n", [(32, 40008), (16, 4096), (33, 4096)])
def test_warp_mma_form_not_taken_outside_its_shapes(ntt, m, n):
    """n not a multiple of 64, 16 rows or fewer, more than 32 rows: another pass runs."""
    X = _x_matrix("uniform", m, n, 29)
    W0 = synth.uniform_matrix((m, 8), 30)
    H0 = synth.uniform_matrix((8, n), 31)
    eng = []
    _run_gpu_mu(ntt, X, W0, H0, 2, engine=eng)
    assert eng and eng[0] != "tc_narrow"


@pytest.mark.parametrize("x_dtype,refine", [("f32", 0), ("bf16", 3)])
def test_plan_engine_routes_agree(ntt, x_dtype, refine):
    """Stages with <= 256 rows and rank >= 16 run on the grouped engine by default;
    every route (single-problem passes only, grouped wherever it applies, FMA
    only, generic pass only, tensor cores wherever they apply) gives the same
    iterates within rounding (10 MU iterations per stage, per-core relative
    1e-4 x stage index), and each route reports the engines it allows."""
    dims, ranks = (16, 16, 16, 16, 16), (1, 8, 16, 16, 8, 1)
    A, _ = synth.tt_tensor(dims, ranks, "uniform", 0.01, seed=12)
    out = {}
    for route in ("auto", "pass", "grouped", "fma", "generic", "tc"):
        cores, stats, *_ = _decompose(ntt, A, ranks, 10, 7, x_dtype=x_dtype, refine=refine, route=route)
        assert stats["status"] == "NTT_OK"
        engines = [st["engine"] for st in stats["stages"]]
        if route in ("pass", "generic"):
            assert "grouped" not in engines
        if route == "generic":
            assert set(engines) == {"fma_pass"}
        if route == "fma":
            assert not {"tc_bf16", "tc_tf32"} & set(engines)
        out[route] = cores
    for route in out:
        for k, (a, b) in enumerate(zip(out[route], out["auto"])):
            assert _fro_rel(a, b) <= 1e-4 * (k + 1), f"{route} core {k}: {_fro_rel(a, b):.2e}"


def test_mu_bf16_tensor_core_pass_repeats_bitwise(ntt):
    m, n, r = 256, 8192, 32
    X = torch.from_numpy(_x_matrix("uniform", m, n, 5)).to(torch.bfloat16).cuda()
    out = []
    for _ in range(2):
        Wd = torch.from_numpy(synth.uniform_matrix((m, r), 6)).cuda()
        Hd = torch.from_numpy(synth.uniform_matrix((r, n), 7)).cuda()
        ntt.nmf_mu_step(X, Wd, Hd, 5)
        torch.cuda.synchronize()
        out.append((Wd.cpu().numpy(), Hd.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_mu_bf16_tensor_core_pass_long_accumulation(ntt):
    """One MU iteration on 128 x 2^20 BF16 X, rank 32: ~54 tiles per CTA, so the
    tensor-core pass's X H^T and H H^T accumulate over several TMEM runs.  H on
    sampled columns and W from the oracle's P and Q over all columns (FP64)."""
    m, n, r = 128, 1 << 20, 32
    rng = np.random.Generator(np.random.PCG64(41))
    X32 = rng.random((m, n), dtype=np.float32)
    Xb = torch.from_numpy(X32).to(torch.bfloat16)
    X = Xb.to(torch.float64).numpy()
    del X32
    W0 = synth.uniform_matrix((m, r), 42)
    H0 = synth.uniform_matrix((r, n), 43)
    Wd = torch.from_numpy(W0).cuda()
    Hd = torch.from_numpy(H0).cuda()
    ntt.nmf_mu_step(Xb.cuda(), Wd, Hd, 1)
    torch.cuda.synchronize()
    Hg = Hd.cpu().numpy()
    G = W0.astype(np.float64).T @ W0.astype(np.float64)
    P = np.zeros((m, r))
    Q = np.zeros((r, r))
    sample = np.sort(rng.choice(n, size=2048, replace=False))
    chunk = 1 << 17
    for c0 in range(0, n, chunk):
        Xc = X[:, c0:c0 + chunk]
        H0c = H0[:, c0:c0 + chunk].astype(np.float64)
        H1c = np.maximum(0.0, H0c * (W0.T @ Xc) / (G @ H0c + 1e-12))
        P += Xc @ H1c.T
        Q += H1c @ H1c.T
        sel = sample[(sample >= c0) & (sample < c0 + chunk)]
        assert np.allclose(Hg[:, sel], H1c[:, sel - c0], rtol=1e-5, atol=1e-7 * H1c.max())
    W1 = np.maximum(0.0, W0 * P / (W0 @ Q + 1e-12))
    assert _fro_rel(Wd.cpu().numpy(), W1) <= REL_ITERATE


@pytest.mark.parametrize("m,n,r", [(16, 8192, 16), (32, 20008, 32), (12, 4096, 12), (24, 40960, 20)])
def test_mu_bf16_stacked_tensor_core_form(ntt, m, n, r):
    """The stacked form of the BF16 tensor-core pass (16/32 rows; route "tc")
    against the oracle on the BF16-rounded X, 10 iterations."""
    X = _x_matrix("lowrank", m, n, 31)
    Xb = torch.from_numpy(X).to(torch.bfloat16)
    W0 = synth.uniform_matrix((m, r), 32)
    H0 = synth.uniform_matrix((r, n), 33)
    Wd = torch.from_numpy(W0).cuda()
    Hd = torch.from_numpy(H0).cuda()
    eng = []
    ntt.nmf_mu_step(Xb.cuda(), Wd, Hd, 10, route="tc", engine=eng)
    torch.cuda.synchronize()
    assert eng == ["tc_bf16"]
    Wo, Ho, _ = oracle.nmf_mu(Xb.to(torch.float64).numpy(), W0, H0, 10)
    assert _fro_rel(Wd.cpu().numpy(), Wo) <= REL_ITERATE
    assert _fro_rel(Hd.cpu().numpy(), Ho) <= REL_ITERATE


# ------------------------------------------------------------------ FP32 X on the tensor cores (split form)

@pytest.mark.parametrize("m,n,r,kind", [(256, 40000, 16, "lowrank"), (128, 20008, 32, "uniform"),
                                        (200, 9000, 20, "lowrank"), (256, 64, 16, "uniform"),
                                        (130, 777 * 8, 12, "lowrank"), (256, 1 << 18, 16, "uniform"),
                                        (512, 1 << 15, 16, "lowrank"), (300, 1000 * 8, 14, "uniform"),
                                        (512, 1 << 10, 16, "uniform"), (32, 1 << 18, 8, "uniform"),
                                        (32, 40008, 8, "lowrank"), (20, 9000, 6, "lowrank"),
                                        (16, 4096, 12, "uniform"), (32, 5000 * 8, 16, "lowrank"),
                                        (32, 8, 8, "uniform")])
def test_mu_fp32_split_tensor_core_form(ntt, m, n, r, kind):
    """FP32 X split once into bf16(X) + bf16(X - bf16(X)) on the BF16 tensor-core
    pass (route "tc"): iterates within the FP32 bound of the FP64 oracle on the
    unsplit X after 10 updates, the engine reported, and a bitwise repeat."""
    X = _x_matrix(kind, m, n, 17 + m)
    W0 = synth.uniform_matrix((m, r), 18)
    H0 = synth.uniform_matrix((r, n), 19)
    eng = []
    Wg, Hg, og = _run_gpu_mu(ntt, X, W0, H0, 10, route="tc", engine=eng)
    assert eng == ["tc_split"]
    Wg2, Hg2, _ = _run_gpu_mu(ntt, X, W0, H0, 10, route="tc")
    assert np.array_equal(Wg, Wg2) and np.array_equal(Hg, Hg2)
    Wo, Ho, tr = oracle.nmf_mu(X.astype(np.float64), W0, H0, 10)
    assert _fro_rel(Wg, Wo) <= REL_ITERATE, _fro_rel(Wg, Wo)
    assert _fro_rel(Hg, Ho) <= REL_ITERATE, _fro_rel(Hg, Ho)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    assert np.allclose(og, tr, rtol=2e-3, atol=1e-6 * float(np.sum(X.astype(np.float64) ** 2)))


def test_mu_fp32_split_form_full_stage2_shape_sampled(ntt):
    """The 32^6 job's stage-2 shape (256 x 1,048,576, r = 16) on the split
    tensor-core form, one iteration: H on sampled columns, W from the oracle's
    FP64 P = X H^T and Q = H H^T over all columns."""
    m, n, r = 256, 1 << 20, 16
    rng = np.random.Generator(np.random.PCG64(51))
    X = rng.random((m, n), dtype=np.float32)
    W0 = synth.uniform_matrix((m, r), 52)
    H0 = synth.uniform_matrix((r, n), 53)
    Wd = torch.from_numpy(W0).cuda()
    Hd = torch.from_numpy(H0).cuda()
    eng = []
    ntt.nmf_mu_step(torch.from_numpy(X).cuda(), Wd, Hd, 1, route="tc", engine=eng)
    torch.cuda.synchronize()
    assert eng == ["tc_split"]
    Hg = Hd.cpu().numpy()
    G = W0.astype(np.float64).T @ W0.astype(np.float64)
    P = np.zeros((m, r))
    Q = np.zeros((r, r))
    sample = np.sort(rng.choice(n, size=2048, replace=False))
    chunk = 1 << 17
    for c0 in range(0, n, chunk):
        Xc = X[:, c0:c0 + chunk].astype(np.float64)
        H0c = H0[:, c0:c0 + chunk].astype(np.float64)
        H1c = np.maximum(0.0, H0c * (W0.T @ Xc) / (G @ H0c + 1e-12))
        P += Xc @ H1c.T
        Q += H1c @ H1c.T
        sel = sample[(sample >= c0) & (sample < c0 + chunk)]
        assert np.allclose(Hg[:, sel], H1c[:, sel - c0], rtol=2e-5, atol=1e-7 * H1c.max())
    W1 = np.maximum(0.0, W0 * P / (W0 @ Q + 1e-12))
    assert _fro_rel(Wd.cpu().numpy(), W1) <= REL_ITERATE


def test_plan_stage2_runs_on_split_form(ntt):
    """The 32^6 recipe at 16^6: its 128-row, rank-16 second stage runs on the
    split tensor-core form by default and the cores match the FMA-only route."""
    c = synth.CONFIGS["c2_32x6"]
    dims = (16,) * 6
    A, _ = synth.tt_tensor(dims, c["ranks"], c["core_dist"], c["noise"], c["data_seed"])
    cores_a, stats_a, *_ = _decompose(ntt, A, c["ranks"], 10, c["init_seed"])
    assert stats_a["stages"][1]["engine"] == "tc_split"
    cores_f, stats_f, *_ = _decompose(ntt, A, c["ranks"], 10, c["init_seed"], route="fma")
    assert stats_f["stages"][1]["engine"] != "tc_split"
    for k, (a, b) in enumerate(zip(cores_a, cores_f)):
        assert _fro_rel(a, b) <= 1e-4 * (k + 1), f"core {k}: {_fro_rel(a, b):.2e}"

"""nmf_mu_many (many NMFs through the grouped engine) against the oracle's
multiplicative-update NMF, problem by problem, plus the property the serving
form rests on: a problem's iterates are bitwise the same alone or in a mix.

Tolerance: relative Frobenius difference of W and H after 10 iterations
<= 1e-4 against the FP64 oracle (FP32 arithmetic, FP64-combined reductions),
as for nmf_mu_step."""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_ITERATE = 1e-4

SHAPES = [
    (700, 900, 8),      # tall: two row blocks (512 + 188)
    (1300, 257, 5),     # tall: three row blocks, odd n (4-byte copies)
    (513, 1000, 32),    # tall: the second row block has one row
    (2048, 64, 32),     # tall: four full row blocks, one column tile
    (64, 10000, 20),    # fused, 32-rank bucket
    (300, 2050, 12),    # fused, 512-row bucket, n % 4 == 2
    (40, 5000, 17),     # fused, odd rank
    (16, 3, 2),         # fewer columns than one tile
    (1, 999, 1),        # m = r = 1
]


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


def _problem(m, n, r, seed):
    X = synth.uniform_matrix((m, n), seed)
    W0 = synth.uniform_matrix((m, r), seed + 1)
    H0 = synth.uniform_matrix((r, n), seed + 2)
    return X, W0, H0


def _run(ntt, probs, iters):
    Xs = [torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda() for X, _, _ in probs]
    Ws = [torch.from_numpy(W0.astype(np.float32)).cuda() for _, W0, _ in probs]
    Hs = [torch.from_numpy(H0.astype(np.float32)).cuda() for _, _, H0 in probs]
    ntt.nmf_mu_many(Xs, Ws, Hs, iters)
    torch.cuda.synchronize()
    return [W.cpu().numpy() for W in Ws], [H.cpu().numpy() for H in Hs]


def test_many_matches_oracle_per_problem(ntt):
    probs = [_problem(m, n, r, 100 + 7 * i) for i, (m, n, r) in enumerate(SHAPES)]
    iters = 10
    Wg, Hg = _run(ntt, probs, iters)
    for i, (X, W0, H0) in enumerate(probs):
        Wo, Ho, _ = oracle.nmf_mu(X.astype(np.float64), W0, H0, iters, record=False)
        assert _fro_rel(Wg[i], Wo) <= REL_ITERATE, f"{SHAPES[i]} W {_fro_rel(Wg[i], Wo):.2e}"
        assert _fro_rel(Hg[i], Ho) <= REL_ITERATE, f"{SHAPES[i]} H {_fro_rel(Hg[i], Ho):.2e}"
        assert np.all(Wg[i] >= 0) and np.all(Hg[i] >= 0)


def test_many_alone_equals_in_mix_bitwise(ntt):
    probs = [_problem(m, n, r, 500 + 3 * i) for i, (m, n, r) in enumerate(SHAPES)]
    Wm, Hm = _run(ntt, probs, 7)
    for i in (0, 1, 4, 7):
        Wa, Ha = _run(ntt, [probs[i]], 7)
        assert np.array_equal(Wa[0], Wm[i]) and np.array_equal(Ha[0], Hm[i]), SHAPES[i]


def test_many_zero_iterations_leave_factors(ntt):
    probs = [_problem(700, 50, 3, 9)]
    Wg, Hg = _run(ntt, probs, 0)
    assert np.array_equal(Wg[0], probs[0][1].astype(np.float32))
    assert np.array_equal(Hg[0], probs[0][2].astype(np.float32))

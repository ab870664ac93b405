"""Out-of-core multiplicative updates: X in (pinned) host memory streamed to
the device in column chunks every iteration.  Iterates match the in-HBM
nmf_mu_step and the FP64 oracle within the FP32 bound after 10 updates, for
several chunkings (a ragged last chunk, unaligned rows on the copy-loop's
cooperative loads, a single resident chunk) and pageable host memory."""

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


@pytest.mark.parametrize("m,n,r,chunk,pinned", [(32, 100000, 8, 30000, True), (256, 50000, 16, 16384, True),
                                                (24, 777, 3, 256, True), (100, 6000, 5, 8192, True),
                                                (64, 20000, 12, 4096, False)])
def test_streamed_iterates_match(ntt, m, n, r, chunk, pinned):
    rng = np.random.Generator(np.random.PCG64(m + n))
    X = (rng.random((m, 5)) @ rng.random((5, n)) + 0.01 * rng.random((m, n))).astype(np.float32)
    W0 = synth.uniform_matrix((m, r), 11)
    H0 = synth.uniform_matrix((r, n), 12)
    iters = 10
    Xh = torch.from_numpy(X)
    if pinned:
        Xh = Xh.pin_memory()
    W = torch.from_numpy(W0.copy()).cuda()
    H = torch.from_numpy(H0.copy()).cuda()
    obj = torch.zeros(iters, dtype=torch.float64, device="cuda")
    ntt.nmf_mu_step_host(Xh, W, H, iters, chunk, obj=obj)
    torch.cuda.synchronize()
    Wd = torch.from_numpy(W0.copy()).cuda()
    Hd = torch.from_numpy(H0.copy()).cuda()
    ntt.nmf_mu_step(torch.from_numpy(X).cuda(), Wd, Hd, iters)
    torch.cuda.synchronize()
    assert _rel(W.cpu(), Wd.cpu()) <= 1e-5 and _rel(H.cpu(), Hd.cpu()) <= 1e-5
    Wo, Ho, tr = oracle.nmf_mu(X.astype(np.float64), W0, H0, iters)
    assert _rel(W.cpu(), Wo) <= 1e-4 and _rel(H.cpu(), Ho) <= 1e-4
    xn = float(np.sum(X.astype(np.float64) ** 2))
    assert np.allclose(obj.cpu().numpy(), tr, rtol=2e-3, atol=1e-6 * xn)


def test_streamed_repeat_is_bitwise(ntt):
    m, n, r = 48, 70000, 10
    X = torch.from_numpy(synth.uniform_matrix((m, n), 3)).pin_memory()
    out = []
    for _ in range(2):
        W = torch.from_numpy(synth.uniform_matrix((m, r), 4)).cuda()
        H = torch.from_numpy(synth.uniform_matrix((r, n), 5)).cuda()
        ntt.nmf_mu_step_host(X, W, H, 5, 16384)
        torch.cuda.synchronize()
        out.append((W.cpu(), H.cpu()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])

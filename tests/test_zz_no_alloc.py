"""nmf_mu_step_noalloc: the entry point for callers that cannot allocate
device memory (its scratch is the library's own device array).  Checked
against nmf_mu_step with a caller workspace on the same inputs, bitwise (the
same kernels run in the same reduction order), on two calls in a row (the
second call finds the first call's scratch contents).  Kept in
a file of its own that pytest collects last."""

import numpy as np
import pytest

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


@pytest.mark.parametrize("m,n,r", [(32, 50000, 8), (256, 3000, 16), (24, 777, 3)])
def test_noalloc_matches_workspace_entry_point(ntt, m, n, r):
    X = torch.from_numpy(synth.uniform_matrix((m, n), 501)).cuda()
    W0 = synth.uniform_matrix((m, r), 502)
    H0 = synth.uniform_matrix((r, n), 503)
    Wr = torch.from_numpy(W0.copy()).cuda()
    Hr = torch.from_numpy(H0.copy()).cuda()
    objr = torch.zeros(6, dtype=torch.float64, device="cuda")
    ntt.nmf_mu_step(X, Wr, Hr, 6, 1e-12, objr)
    torch.cuda.synchronize()
    for call in range(2):
        W = torch.from_numpy(W0.copy()).cuda()
        H = torch.from_numpy(H0.copy()).cuda()
        obj = torch.zeros(6, dtype=torch.float64, device="cuda")
        ntt.nmf_mu_step_noalloc(X, W, H, 6, 1e-12, obj)
        torch.cuda.synchronize()
        # same kernels, same launch shapes, same fixed reduction order: bitwise equal
        assert torch.equal(W, Wr), f"call {call}: W differs (rel {_rel(W.cpu(), Wr.cpu()):.2e})"
        assert torch.equal(H, Hr), f"call {call}: H differs (rel {_rel(H.cpu(), Hr.cpu()):.2e})"
        assert torch.equal(obj, objr), f"call {call}: objective trace differs"


def test_noalloc_rejects_shapes_beyond_its_scratch(ntt):
    # m = 512, r = 32 needs more than the 8 MiB scratch array: clear error, no launch
    X = torch.zeros((512, 4096), dtype=torch.float32, device="cuda")
    W = torch.zeros((512, 32), dtype=torch.float32, device="cuda")
    H = torch.zeros((32, 4096), dtype=torch.float32, device="cuda")
    with pytest.raises(ntt.NTTError) as e:
        ntt.nmf_mu_step_noalloc(X, W, H, 1)
    assert e.value.code == 3

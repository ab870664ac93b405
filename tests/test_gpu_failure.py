"""Failure detection on the GPU without a fault: a bounded device wait that
runs out ends its kernel with a status word the host reads, and the context
and the workspace stay usable.

The probe kernel waits, with a limit the test chooses, on an mbarrier phase
that nothing completes, while a real bulk copy it started is in flight; it
then drains that copy (bounded) and records NTT_ERR_TIMEOUT -- the same path
every pass kernel takes when one of its waits gives up.  No fault, trap or
unbounded spin is involved."""

import time

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


@pytest.mark.parametrize("limit_ns", [0, 1_000_000, 20_000_000])
def test_wait_that_runs_out_reports_timeout_then_recovers(ntt, limit_ns):
    m, n, r = 32, 4096, 8
    ws = ntt.empty_workspace(ntt.nmf_mu_workspace_size(m, n, r))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ntt.ntt_wait_probe(ws, limit_ns)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert ntt.ntt_status_of_workspace(ws) == "NTT_ERR_TIMEOUT"
    # the wait lasted at least its limit and ended long before the 2 s default
    assert dt >= limit_ns * 1e-9 and dt < 1.0
    # the same workspace serves a normal call afterwards
    X = torch.from_numpy(synth.uniform_matrix((m, n), 1)).cuda()
    W = torch.from_numpy(synth.uniform_matrix((m, r), 2)).cuda()
    H = torch.from_numpy(synth.uniform_matrix((r, n), 3)).cuda()
    ntt.nmf_mu_step(X, W, H, 3, workspace=ws)
    torch.cuda.synchronize()
    assert ntt.ntt_status_of_workspace(ws) == "NTT_OK"
    assert bool(torch.all(torch.isfinite(W))) and bool(torch.all(H >= 0))


def test_wait_probe_rejects_bad_arguments(ntt):
    ws = ntt.empty_workspace(4096)
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_wait_probe(ws, -1)
    assert e.value.code == 1
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_wait_probe(ws[16:], 1000)
    assert e.value.code == 1

"""Serving form against the oracle's Algorithm 2 (one initialisation per
stage, the job's own seed), and the serving properties: bitwise the same
result alone or in a mix, BF16 jobs equal to FP32 jobs of the rounded values,
admission bounded by the HBM budget in arrival order.

Tolerance: per-core relative Frobenius difference <= 1e-4 times the stage
index after 10 iterations per stage (as for the plan and batched forms)."""

import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

JOBS = [
    ((12, 10, 8, 6), (1, 6, 9, 4, 1)),
    ((40, 30, 20, 10), (1, 20, 25, 8, 1)),     # stage 2 is 600 rows tall: row-block path
    ((9, 9, 9), (1, 3, 5, 1)),
    ((64, 48), (1, 32, 1)),                    # d = 2, rank 32
]


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


def _tensor(dims, ranks, seed):
    T, _ = synth.tt_tensor(dims, ranks, "uniform", 0.01, seed=seed)
    return torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32).ravel())


def _serve(ntt, jobs, stage_iters=10, tick=5, budget=1 << 30, max_jobs=64):
    srv = ntt.Server(budget, max_jobs=max_jobs, tick_iters=tick, stage_iters=stage_iters)
    try:
        handles = [srv.submit(A, dims, ranks, seed=seed) for A, dims, ranks, seed in jobs]
        infos = [srv.wait(h, timeout=120) for h in handles]
        stats = srv.stats()
    finally:
        srv.close()
    return handles, infos, stats


def test_served_jobs_match_oracle(ntt):
    jobs = [(_tensor(d, r, 50 + i), d, r, 900 + i) for i, (d, r) in enumerate(JOBS)]
    handles, infos, stats = _serve(ntt, jobs)
    assert stats["completed"] == len(JOBS) and stats["failed"] == 0
    for (A, dims, ranks, seed), h, info in zip(jobs, handles, infos):
        assert info["state"] == "done" and info["t_done"] >= info["t_admit"] >= info["t_submit"]
        ref, _ = oracle.ntt_decompose(A.numpy().reshape(dims).astype(np.float64), ranks, 10, seed=seed,
                                      record=False)
        for k, (g, o) in enumerate(zip(h.core_views(), ref)):
            assert _rel(g.numpy(), o) <= 1e-4 * (k + 1), f"{dims} core {k}: {_rel(g.numpy(), o):.2e}"
            assert np.all(g.numpy() >= 0)


def test_job_alone_equals_job_in_mix_bitwise(ntt):
    target = (_tensor(*JOBS[1], 77), JOBS[1][0], JOBS[1][1], 4242)
    others = [(_tensor(d, r, 60 + i), d, r, 10 + i) for i, (d, r) in enumerate(JOBS * 2)]
    alone, _, _ = _serve(ntt, [target])
    mixed, _, _ = _serve(ntt, others[:3] + [target] + others[3:], tick=10, stage_iters=10)
    assert torch.equal(alone[0].cores, mixed[3].cores)


def test_bf16_job_equals_f32_job_of_rounded_values(ntt):
    dims, ranks = JOBS[0]
    A = _tensor(dims, ranks, 5)
    Ab = A.to(torch.bfloat16)
    h, _, _ = _serve(ntt, [(Ab, dims, ranks, 1), (Ab.float().contiguous(), dims, ranks, 1)])
    assert torch.equal(h[0].cores, h[1].cores)


def test_admission_respects_budget_and_arrival_order(ntt):
    dims, ranks = (48, 40, 30, 20), (1, 16, 16, 8, 1)
    fp = ntt.ntt_server_job_footprint(dims, ranks)
    budget = 2 * fp + fp // 2           # two jobs fit, a third does not
    jobs = [(_tensor(dims, ranks, 30 + i), dims, ranks, i) for i in range(6)]
    handles, infos, stats = _serve(ntt, jobs, budget=budget)
    assert stats["completed"] == 6 and stats["peak_bytes"] <= budget
    admits = [i["t_admit"] for i in infos]
    assert admits == sorted(admits)                                   # FIFO admission
    for i, inf in enumerate(infos):                                   # never more than two resident
        overlap = sum(1 for o in infos if o["t_admit"] < inf["t_done"] and o["t_done"] > inf["t_admit"])
        assert overlap <= 2, (i, overlap)


def test_oversized_job_is_refused(ntt):
    dims, ranks = (64, 64, 64), (1, 16, 16, 1)
    srv = ntt.Server(1 << 20, max_jobs=4, tick_iters=5, stage_iters=10)
    try:
        with pytest.raises(ntt.NTTError) as e:
            srv.submit(_tensor(dims, ranks, 1), dims, ranks)
        assert e.value.code == 3    # NTT_ERR_OOM
    finally:
        srv.close()


def test_wait_timeout_then_result(ntt):
    dims, ranks = (32, 32, 32, 32), (1, 16, 16, 16, 1)
    srv = ntt.Server(1 << 30, max_jobs=4, tick_iters=10, stage_iters=200)
    try:
        h = srv.submit(_tensor(dims, ranks, 3), dims, ranks)
        with pytest.raises(ntt.NTTError) as e:
            srv.wait(h, timeout=1e-4)
        assert e.value.code == 5    # NTT_ERR_TIMEOUT: the job stays known
        info = srv.wait(h, timeout=120)
        assert info["state"] == "done"
    finally:
        srv.close()

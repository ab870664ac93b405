"""Stage-level checkpoint and resume (ntt_decompose_stages, include/ntt.h):
a decomposition run in pieces, with the unfolding between them saved to a
host file and read back into a fresh workspace, gives bitwise the cores of
one ntt_decompose call (the paper keeps its intermediate factors in a store
between the stages of Algorithm 2, Section III-B)."""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ntt():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2008_01340_gb300 as m
    m.lib()
    return m


def _setup(ntt, dims, ranks, iters, seed):
    A, _ = synth.tt_tensor(dims, ranks, "uniform", 0.01, 3)
    plan = ntt.ntt_plan_create(dims, ranks, iters, 1e-12, "f32", 0, seed)
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    return plan, Ad


def _cores(ntt, plan):
    return [torch.zeros(s, dtype=torch.float32, device="cuda") for s in plan.core_shapes()]


@pytest.mark.parametrize("dims,ranks,split", [((16,) * 6, (1, 8, 16, 16, 16, 8, 1), 2),
                                              ((8, 12, 10, 9, 7), (1, 4, 9, 6, 3, 1), 1),
                                              ((8, 12, 10, 9, 7), (1, 4, 9, 6, 3, 1), 3)])
def test_resume_from_saved_unfolding_is_bitwise(ntt, tmp_path, dims, ranks, split):
    plan, Ad = _setup(ntt, dims, ranks, 12, 5)
    ws = ntt.empty_workspace(plan.workspace_size())
    full = _cores(ntt, plan)
    ntt.ntt_decompose(plan, Ad, full, ws)
    torch.cuda.synchronize()
    # first piece: stages 0 .. split-1, then the checkpoint to a host file
    part = _cores(ntt, plan)
    H = torch.empty(ntt.ntt_unfolding_size(plan, split), dtype=torch.float32, device="cuda")
    ntt.ntt_decompose_stages(plan, 0, split, Ad, part, H, ws)
    torch.cuda.synchronize()
    path = tmp_path / "ckpt.npz"
    ntt.save_checkpoint(path, plan, split, part, H)
    # resume in a new plan with a new workspace, from the file alone
    plan2 = ntt.ntt_plan_create(dims, ranks, 12, 1e-12, "f32", 0, 5)
    ws2 = ntt.empty_workspace(plan2.workspace_size())
    s, saved, Hs = ntt.load_checkpoint(path, plan2)
    assert s == split
    res = _cores(ntt, plan2)
    for k in range(s):
        res[k].copy_(torch.from_numpy(saved[k]))
    ntt.ntt_decompose_stages(plan2, s, len(dims) - 1, torch.from_numpy(Hs).cuda(), res, None, ws2)
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(zip(full, res)):
        assert torch.equal(a, b), f"core {k}"


def test_every_stage_separately_is_bitwise(ntt):
    dims, ranks = (8, 12, 10, 9, 7), (1, 4, 9, 6, 3, 1)
    plan, Ad = _setup(ntt, dims, ranks, 8, 9)
    ws = ntt.empty_workspace(plan.workspace_size())
    full = _cores(ntt, plan)
    ntt.ntt_decompose(plan, Ad, full, ws)
    cores = _cores(ntt, plan)
    X = Ad
    for s in range(len(dims) - 1):
        last = s == len(dims) - 2
        H = None if last else torch.empty(ntt.ntt_unfolding_size(plan, s + 1), dtype=torch.float32, device="cuda")
        ntt.ntt_decompose_stages(plan, s, s + 1, X, cores, H, ws)
        X = H
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(zip(full, cores)):
        assert torch.equal(a, b), f"core {k}"


def test_checkpoint_of_another_plan_is_refused(ntt, tmp_path):
    dims, ranks = (8, 12, 10, 9, 7), (1, 4, 9, 6, 3, 1)
    plan, Ad = _setup(ntt, dims, ranks, 4, 1)
    ws = ntt.empty_workspace(plan.workspace_size())
    cores = _cores(ntt, plan)
    H = torch.empty(ntt.ntt_unfolding_size(plan, 2), dtype=torch.float32, device="cuda")
    ntt.ntt_decompose_stages(plan, 0, 2, Ad, cores, H, ws)
    torch.cuda.synchronize()
    path = tmp_path / "ckpt.npz"
    ntt.save_checkpoint(path, plan, 2, cores, H)
    other = ntt.ntt_plan_create(dims, ranks, 4, 1e-12, "f32", 0, 2)   # another seed
    with pytest.raises(ValueError):
        ntt.load_checkpoint(path, other)

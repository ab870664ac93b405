"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/ntt.h declares, and validates plans on the host."""

import ctypes
import os
import re

import pytest

import oracle
import paper_2008_01340_gb300 as ntt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", hdr)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                             txt, flags=re.M):
            names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(ntt.LIB_PATH):
        ntt.build()
    return ntt.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "ntt_decompose" in names and "nmf_mu_step" in names and "ntt_rel_error" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(ntt.EXPORTS) <= set(names)


def test_status_strings(lib):
    for code, name in ntt.STATUS.items():
        assert lib.ntt_status_string(code).decode() == name


def test_compression_ratio_matches_eq4(lib):
    for dims, ranks in [((5, 4, 5, 6), (1, 4, 3, 2, 1)), ((32,) * 6, (1, 8, 16, 16, 16, 8, 1)),
                        ((8, 8, 8, 8), (1, 3, 3, 3, 1))]:
        assert abs(ntt.ntt_compression_ratio(dims, ranks) - oracle.compression_ratio(dims, ranks)) < 1e-12


def test_plan_validation(lib):
    # r_1 > min(m, n) (Algorithm 2: N = min(m, n))
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan_create((4, 4), (1, 5, 1), 10)
    assert e.value.code == 2
    # r_0 != 1
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan_create((4, 4), (2, 2, 1), 10)
    assert e.value.code == 1
    # rank above the built maximum
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan_create((64, 64, 64), (1, 33, 33, 1), 10)
    assert e.value.code == 6
    # unfolding taller than the built maximum (r_1 n_2 = 32 * 32 = 1024 > 512)
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan_create((32, 32, 32), (1, 32, 16, 1), 10)
    assert e.value.code == 6
    # iters < 1
    with pytest.raises(ntt.NTTError):
        ntt.ntt_plan_create((8, 8), (1, 2, 1), 0)
    # no ranks: Algorithm 2's rank rule needs eps_rank > 0
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan_create((8, 8), None, 10)
    assert e.value.code == 1
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan_create((8, 8), None, 10, eps_rank=0.1, rank_cap=-1)
    assert e.value.code == 1
    # rank-rule plans are sized for the largest ranks the rule may choose:
    # min(m, n), the built maximum 32, the cap, and next height r_l n_{l+1} <= 512
    p = ntt.ntt_plan_create((8, 8, 8, 8), None, 10, eps_rank=0.1)
    assert p.current_ranks() == (1, 8, 32, 8, 1) and p.core_shapes()[1] == (8, 8, 32)
    p = ntt.ntt_plan_create((8, 8, 8, 8), None, 10, eps_rank=0.1, rank_cap=5)
    assert p.current_ranks() == (1, 5, 5, 5, 1)
    p = ntt.ntt_plan_create((4, 200, 3), None, 10, eps_rank=0.1)
    assert p.current_ranks() == (1, 2, 3, 1)     # 4 * 200 and 2 * 200 <= 512 needs r_1 <= 2
    with pytest.raises(ntt.NTTError) as e:        # first unfolding taller than 512
        ntt.ntt_plan_create((600, 4), None, 10, eps_rank=0.1)
    assert e.value.code == 6
    assert p.workspace_size() > 0
    # stopping test: tol >= 0 (not NaN), check_every >= 1 when tol > 0
    for tol, k in ((-1e-3, 10), (float("nan"), 10), (1e-3, 0)):
        with pytest.raises(ntt.NTTError) as e:
            ntt.ntt_plan_create((8, 8), (1, 2, 1), 10, tol=tol, check_every=k)
        assert e.value.code == 1
    ntt.ntt_plan_create((8, 8), (1, 2, 1), 10, tol=1e-3, check_every=5).destroy()
    ntt.ntt_plan_create((8, 8), (1, 2, 1), 10, tol=0.0, check_every=0).destroy()
    # kernel routes and flags are plan fields validated on the host
    for route in ntt.ROUTES:
        ntt.ntt_plan_create((8, 8), (1, 2, 1), 10, route=route, eager=True).destroy()
    with pytest.raises(ValueError):
        ntt.ntt_plan_create((8, 8), (1, 2, 1), 10, route="fastest")
    for route, flags in ((6, 0), (-1, 0), (0, 2)):
        d_arr, r_arr = ntt._i64arr((8, 8)), ntt._i64arr((1, 2, 1))
        desc = ntt._PlanDesc(d=2, dims=ctypes.cast(d_arr, ctypes.POINTER(ctypes.c_int64)),
                             ranks=ctypes.cast(r_arr, ctypes.POINTER(ctypes.c_int64)), iters=10,
                             eps_mu=1e-12, route=route, flags=flags)
        h = ctypes.c_void_p()
        assert lib.ntt_plan_create(ctypes.byref(desc), ctypes.byref(h)) == 1


def test_workspace_sizes(lib):
    p = ntt.ntt_plan_create((32,) * 6, (1, 8, 16, 16, 16, 8, 1), 200)
    ws = p.workspace_size()
    # H_1 (8 x 32^5 FP32, 1.07 GB) and H_2 (16 x 32^4) live in the workspace, and
    # the two BF16 terms of the largest split unfolding: stage 1's 32 x 32^5 for
    # the warp-level MMA form (stage 2's 256 x 32^4 for the split form is smaller)
    assert ws >= 4 * (8 * 32 ** 5 + 16 * 32 ** 4) + 4 * 32 ** 6
    assert ws < 6.0e9
    assert p.workspace_size_host() >= ws + 4 * 32 ** 6
    pb = ntt.ntt_plan_create((16,) * 8, (1, 16, 32, 32, 32, 32, 32, 16, 1), 200, x_dtype="bf16",
                             refine_iters=5)
    assert pb.workspace_size() >= 2 * 16 ** 8        # BF16 copy of X_1
    assert ntt.nmf_mu_workspace_size(32, 1000, 8) > 0
    with pytest.raises(ntt.NTTError):
        ntt.nmf_mu_workspace_size(600, 1000, 8)
    assert ntt.ntt_reconstruct_workspace_size((32,) * 6, (1, 8, 16, 16, 16, 8, 1)) > 0


def test_null_arguments_rejected_without_launch(lib):
    p = ntt.ntt_plan_create((8, 8), (1, 2, 1), 5)
    vp = ctypes.c_void_p
    assert lib.ntt_decompose(p.handle, None, None, None, None) == 1
    assert lib.nmf_mu_step(8, 8, 2, None, 0, None, None, 1, ctypes.c_float(1e-12), None, None, None) == 1
    assert lib.ntt_plan_workspace_size(None, None) == 1
    assert lib.ntt_uniform_init(1, 0, 0, 2, 10, vp(16), None) == 1   # bad matrix id
    assert lib.ntt_wait_probe(None, 1000, None) == 1
    assert lib.ntt_wait_probe(vp(256), -5, None) == 1
    assert lib.nmf_mu_step_route(8, 8, 2, vp(256), 0, vp(256), vp(256), 1, ctypes.c_float(1e-12), None,
                                 vp(256), None, 9, None) == 1                              # bad route


def test_stage_range_validation_and_unfolding_sizes(lib):
    """ntt_decompose_stages rejects empty or out-of-range stage ranges and
    missing buffers before any launch; ntt_unfolding_size is r_s prod_{j>=s} n_j."""
    dims, ranks = (8, 12, 10, 9, 7), (1, 4, 9, 6, 3, 1)
    p = ntt.ntt_plan_create(dims, ranks, 5)
    assert [ntt.ntt_unfolding_size(p, s) for s in (1, 2, 3)] == [4 * 12 * 10 * 9 * 7, 9 * 10 * 9 * 7, 6 * 9 * 7]
    for s in (0, 4, -1):
        with pytest.raises(ntt.NTTError):
            ntt.ntt_unfolding_size(p, s)
    vp = ctypes.c_void_p
    cores = (vp * 5)(*[vp(256)] * 5)
    for s0, s1 in ((0, 0), (2, 1), (-1, 2), (0, 5)):
        assert lib.ntt_decompose_stages(p.handle, s0, s1, vp(256), cores, vp(256), vp(256), None) == 1
    assert lib.ntt_decompose_stages(p.handle, 0, 2, vp(256), cores, None, vp(256), None) == 1   # H_out needed
    assert lib.ntt_decompose_stages(p.handle, 0, 2, None, cores, vp(256), vp(256), None) == 1   # X_in needed
    pr = ntt.ntt_plan_create(dims, None, 5, eps_rank=0.1)
    assert lib.ntt_decompose_stages(pr.handle, 0, 2, vp(256), cores, vp(256), vp(256), None) == 6   # rank rule


def test_batch_validation(lib):
    """Batched form: argument checks run on the host before any device call."""
    def code(instances, iters=10, restarts=4):
        with pytest.raises(ntt.NTTError) as e:
            ntt.ntt_batch_create(instances, iters, restarts)
        return e.value.code
    assert code([((8, 8, 8), (1, 9, 3, 1))]) == 2          # r_1 > min(m, n)
    assert code([((8, 8, 8), (2, 3, 3, 1))]) == 1          # r_0 != 1
    assert code([((8,), (1, 1))]) == 1                     # d < 2
    assert code([((64, 64, 64), (1, 33, 33, 1))]) == 6     # rank above the built maximum
    assert code([((8, 8), (1, 2, 1))], restarts=17) == 1   # more restarts than the built maximum
    assert code([((8, 8), (1, 2, 1))], iters=0) == 1
    assert lib.ntt_batch_destroy(None) == 1
    assert lib.ntt_decompose_batched(None, None, None, None, None) == 1


def test_many_validation(lib):
    """nmf_mu_many: argument checks on the host, before any device call."""
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64 * 1
    i32 = ctypes.c_int * 1
    b = ctypes.c_size_t()
    assert lib.nmf_mu_many_workspace_size(0, i64(8), i64(8), i32(2), ctypes.byref(b)) == 1      # count < 1
    assert lib.nmf_mu_many_workspace_size(1, i64(8), i64(8), i32(33), ctypes.byref(b)) == 6     # rank above 32
    assert lib.nmf_mu_many_workspace_size(1, i64(16385), i64(8), i32(2), ctypes.byref(b)) == 6  # taller than 16384
    assert lib.nmf_mu_many_workspace_size(1, i64(0), i64(8), i32(2), ctypes.byref(b)) == 1
    ptrs = (vp * 1)(None)
    assert lib.nmf_mu_many(1, i64(8), i64(8), i32(2), ptrs, ptrs, ptrs, 1, ctypes.c_float(1e-12),
                           vp(256), None) == 1                                                  # null factors


def test_split_scratch_in_single_nmf_workspaces(lib):
    """The tensor-core forms that read a split X get its scratch in the
    nmf_mu_step_route workspace, and only where their route lets them run:
    4 m n bytes for the warp-level MMA form (17..32 rows, rank <= 8, n a
    multiple of 64) on the default route, the tile-major image (whole 64-column
    tiles of the padded rows) for the split form with route "tc", nothing for
    BF16 X (an exact operand) or on the CUDA-core routes."""
    m, n = 32, 64 * 100
    auto = ntt.nmf_mu_workspace_size(m, n, 8, "f32", "auto")
    fma = ntt.nmf_mu_workspace_size(m, n, 8, "f32", "fma")
    assert auto - fma >= 4 * m * n
    # n % 64 != 0: the narrow FMA pass, no split scratch
    assert ntt.nmf_mu_workspace_size(m, n + 8, 8, "f32", "auto") == ntt.nmf_mu_workspace_size(m, n + 8, 8, "f32", "fma")
    m2, n2 = 200, 64 * 50 + 8                        # 256-row bucket, ragged last tile
    tc = ntt.nmf_mu_workspace_size(m2, n2, 16, "f32", "tc")
    plain = ntt.nmf_mu_workspace_size(m2, n2, 16, "f32", "fma")
    assert tc - plain >= ((n2 + 63) // 64) * 256 * 256
    assert (ntt.nmf_mu_workspace_size(16, 64 * 100, 16, "bf16", "auto")
            == ntt.nmf_mu_workspace_size(16, 64 * 100, 16, "bf16", "fma"))

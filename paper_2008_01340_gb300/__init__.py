"""Python binding of libntt (the GB300 non-negative tensor-train library).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libntt.so (built in-tree from csrc/ by `build()`).  Tensors are
torch CUDA tensors (device pointers via data_ptr()); streams are torch CUDA
streams (default: the current stream).  There is no CPU fallback: a missing
library or a failing call raises.

Entry points mirror include/ntt.h:
  ntt_plan_create / Plan.workspace_size / ntt_decompose / ntt_decompose_host /
  ntt_plan_get_stats / nmf_mu_step / nmf_mu_workspace_size /
  ntt_reconstruct / ntt_rel_error / ntt_uniform_init / ntt_compression_ratio
"""

from __future__ import annotations

import ctypes

import numpy as np
import os
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libntt.so")

NTT_MAX_D = 16
NTT_MAX_RANK = 32
NTT_MAX_ROWS = 512

STATUS = {
    0: "NTT_OK",
    1: "NTT_ERR_INVALID_ARG",
    2: "NTT_ERR_RANK_INFEASIBLE",
    3: "NTT_ERR_OOM",
    4: "NTT_ERR_CUDA",
    5: "NTT_ERR_TIMEOUT",
    6: "NTT_ERR_UNSUPPORTED",
}
NTT_F32, NTT_BF16 = 0, 1

# ntt_route: kernel routing of the MU loops (include/ntt.h)
ROUTES = {"auto": 0, "pass": 1, "grouped": 2, "fma": 3, "generic": 4, "tc": 5}
NTT_PLAN_EAGER = 1


def _route(route):
    if route not in ROUTES:
        raise ValueError(f"route must be one of {sorted(ROUTES)}")
    return ROUTES[route]

# Every symbol include/ntt.h declares.
EXPORTS = (
    "ntt_status_string", "ntt_version", "ntt_plan_create", "ntt_plan_workspace_size",
    "ntt_plan_workspace_size_host", "ntt_decompose", "ntt_decompose_host", "ntt_decompose_stages",
    "ntt_unfolding_size",
    "ntt_plan_get_stats", "ntt_plan_destroy", "nmf_mu_workspace_size", "nmf_mu_step",
    "nmf_mu_step_route", "nmf_mu_workspace_size_route", "ntt_wait_probe", "ntt_plan_get_ranks", "ntt_rank_workspace_size",
    "ntt_singular_values", "ntt_select_rank", "nmf_bcd_workspace_size", "nmf_bcd_step",
    "nmf_mu_shard_sizes", "nmf_mu_shard_norm", "nmf_mu_shard_pass", "nmf_mu_shard_update",
    "nmf_mu_host_workspace_size", "nmf_mu_step_host",
    "ntt_status_of_workspace", "ntt_uniform_init", "ntt_reconstruct_workspace_size",
    "ntt_reconstruct", "ntt_rel_error", "ntt_compression_ratio", "nmf_mu_step_noalloc",
    "ntt_batch_create", "ntt_batch_sizes", "ntt_batch_offsets", "ntt_decompose_batched",
    "ntt_batch_destroy", "ntt_batch_tune", "ntt_batch_get_tuning", "nmf_mu_many_workspace_size", "nmf_mu_many",
    "ntt_server_create", "ntt_server_job_footprint", "ntt_server_submit", "ntt_server_poll",
    "ntt_server_wait", "ntt_server_get_stats", "ntt_server_destroy",
)


class NTTError(RuntimeError):
    def __init__(self, code, where):
        self.code = int(code)
        super().__init__(f"{where}: {STATUS.get(self.code, self.code)}")


class _PlanDesc(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("dims", ctypes.POINTER(ctypes.c_int64)),
        ("ranks", ctypes.POINTER(ctypes.c_int64)),
        ("iters", ctypes.c_int),
        ("eps_mu", ctypes.c_float),
        ("x_dtype", ctypes.c_int),
        ("refine_iters", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("tol", ctypes.c_double),
        ("check_every", ctypes.c_int),
        ("route", ctypes.c_int),
        ("flags", ctypes.c_uint),
        ("eps_rank", ctypes.c_double),
        ("rank_cap", ctypes.c_int),
        ("solver", ctypes.c_int),
    ]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_jobs", ctypes.c_int),
                ("tick_iters", ctypes.c_int), ("stage_iters", ctypes.c_int), ("eps_mu", ctypes.c_float)]


class _JobInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("stage", ctypes.c_int),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("footprint_bytes", ctypes.c_size_t)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("ticks", ctypes.c_int64), ("resident", ctypes.c_int), ("queued", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("capacity_bytes", ctypes.c_size_t), ("busy_s", ctypes.c_double)]


JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}


class _Stats(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("status", ctypes.c_int),
        ("iters", ctypes.c_int * NTT_MAX_D),
        ("m", ctypes.c_int64 * NTT_MAX_D),
        ("n", ctypes.c_int64 * NTT_MAX_D),
        ("r", ctypes.c_int64 * NTT_MAX_D),
        ("xnorm2", ctypes.c_double * NTT_MAX_D),
        ("obj_first", ctypes.c_double * NTT_MAX_D),
        ("obj_last", ctypes.c_double * NTT_MAX_D),
        ("resid", ctypes.c_double * NTT_MAX_D),
        ("stage_ms", ctypes.c_float * NTT_MAX_D),
        ("iter_ms", ctypes.c_float * NTT_MAX_D),
        ("total_ms", ctypes.c_float),
        ("alg_bytes", ctypes.c_double * NTT_MAX_D),
        ("launches", ctypes.c_int64),
        ("engine", ctypes.c_int * NTT_MAX_D),
    ]


ENGINES = {0: "fma_pass", 1: "grouped", 2: "tc_bf16", 3: "tc_tf32", 4: "fma_narrow", 5: "bcd_pass",
           6: "tc_split", 7: "tc_narrow"}
SOLVERS = {"mu": 0, "bcd": 1}


_lib_handle = None


def lib():
    """Load libntt.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    p64 = ctypes.POINTER(ctypes.c_int64)
    psz = ctypes.POINTER(ctypes.c_size_t)
    L.ntt_status_string.restype = ctypes.c_char_p
    L.ntt_status_string.argtypes = [i32]
    L.ntt_version.restype = ctypes.c_char_p
    L.ntt_version.argtypes = []
    L.ntt_plan_create.argtypes = [ctypes.POINTER(_PlanDesc), ctypes.POINTER(vp)]
    L.ntt_plan_workspace_size.argtypes = [vp, psz]
    L.ntt_plan_workspace_size_host.argtypes = [vp, psz]
    L.ntt_decompose.argtypes = [vp, vp, ctypes.POINTER(vp), vp, vp]
    L.ntt_decompose_host.argtypes = [vp, vp, ctypes.POINTER(vp), vp, vp, vp]
    L.ntt_decompose_stages.argtypes = [vp, i32, i32, vp, ctypes.POINTER(vp), vp, vp, vp]
    L.ntt_unfolding_size.argtypes = [vp, i32, p64]
    L.ntt_plan_get_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
    L.ntt_plan_destroy.argtypes = [vp]
    L.nmf_mu_workspace_size.argtypes = [i64, i64, i32, i32, psz]
    L.nmf_mu_step.argtypes = [i64, i64, i32, vp, i32, vp, vp, i32, ctypes.c_float, vp, vp, vp]
    L.nmf_mu_workspace_size_route.argtypes = [i64, i64, i32, i32, i32, psz]
    L.nmf_mu_step_route.argtypes = [i64, i64, i32, vp, i32, vp, vp, i32, ctypes.c_float, vp, vp, vp, i32,
                                    ctypes.POINTER(ctypes.c_int)]
    L.nmf_mu_step_noalloc.argtypes = [i64, i64, i32, vp, i32, vp, vp, i32, ctypes.c_float, vp, vp]
    L.ntt_status_of_workspace.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.ntt_wait_probe.argtypes = [vp, i64, vp]
    L.ntt_plan_get_ranks.argtypes = [vp, p64]
    L.nmf_bcd_workspace_size.argtypes = [i64, i64, i32, psz]
    L.nmf_mu_shard_sizes.argtypes = [i64, i64, i32, psz, psz]
    L.nmf_mu_host_workspace_size.argtypes = [i64, i64, i32, i64, psz]
    L.nmf_mu_step_host.argtypes = [i64, i64, i32, vp, vp, vp, i32, ctypes.c_float, vp, i64, vp, vp]
    L.nmf_mu_shard_norm.argtypes = [i64, i64, vp, vp, vp, vp]
    L.nmf_mu_shard_pass.argtypes = [i64, i64, i32, vp, vp, vp, ctypes.c_float, vp, vp, vp]
    L.nmf_mu_shard_update.argtypes = [i64, i32, vp, vp, ctypes.c_float, ctypes.c_double, vp, vp, vp]
    L.nmf_bcd_step.argtypes = [i64, i64, i32, vp, vp, vp, i32, vp, vp, vp]
    L.ntt_rank_workspace_size.argtypes = [i64, i64, psz]
    L.ntt_singular_values.argtypes = [i64, i64, vp, vp, vp, vp]
    L.ntt_select_rank.argtypes = [i64, i64, vp, ctypes.c_double, i32, vp, vp, vp, vp]
    L.ntt_uniform_init.argtypes = [ctypes.c_uint64, i32, i32, i32, i64, vp, vp]
    L.ntt_reconstruct_workspace_size.argtypes = [i32, p64, p64, psz]
    L.ntt_reconstruct.argtypes = [i32, p64, p64, ctypes.POINTER(vp), vp, vp, vp]
    L.ntt_rel_error.argtypes = [i32, p64, p64, ctypes.POINTER(vp), vp, vp, vp, vp]
    psz_ = ctypes.POINTER(ctypes.c_size_t)
    L.ntt_batch_create.argtypes = [i32, ctypes.POINTER(ctypes.c_int), p64, p64, i32, i32,
                                   ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(vp)]
    L.ntt_batch_sizes.argtypes = [vp, psz_, psz_, psz_]
    L.ntt_batch_offsets.argtypes = [vp, p64, p64]
    L.ntt_decompose_batched.argtypes = [vp, vp, vp, vp, vp]
    L.ntt_batch_destroy.argtypes = [vp]
    L.ntt_batch_tune.argtypes = [vp, vp, vp, vp, vp, i32, ctypes.c_char_p]
    L.ntt_batch_get_tuning.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]
    L.ntt_compression_ratio.restype = ctypes.c_double
    L.ntt_compression_ratio.argtypes = [i32, p64, p64]
    for name in EXPORTS:
        if name not in ("ntt_status_string", "ntt_version", "ntt_compression_ratio"):
            getattr(L, name).restype = ctypes.c_int
    _lib_handle = L
    return L


def _check(code, where):
    if code != 0:
        raise NTTError(code, where)


def _i64arr(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_int64 * len(vals))(*vals)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _dev_ptr(t, dtype=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def empty_workspace(nbytes, device=None):
    """Device workspace buffer (uint8, 256-byte aligned by the caching allocator)."""
    import torch
    t = torch.empty(max(int(nbytes), 256), dtype=torch.uint8,
                    device=device or torch.device("cuda", torch.cuda.current_device()))
    if t.data_ptr() % 256:
        raise RuntimeError("workspace is not 256-byte aligned")
    return t


@dataclass
class Plan:
    handle: ctypes.c_void_p
    dims: tuple
    ranks: tuple
    iters: int
    x_dtype: str
    refine_iters: int
    max_ranks: tuple = None
    seed: int = 0

    def workspace_size(self):
        n = ctypes.c_size_t(0)
        _check(lib().ntt_plan_workspace_size(self.handle, ctypes.byref(n)), "ntt_plan_workspace_size")
        return n.value

    def workspace_size_host(self):
        n = ctypes.c_size_t(0)
        _check(lib().ntt_plan_workspace_size_host(self.handle, ctypes.byref(n)),
               "ntt_plan_workspace_size_host")
        return n.value

    def current_ranks(self):
        """The plan's ranks (include/ntt.h ntt_plan_get_ranks): the given ones, or
        with the rank rule the last call's choice (the bounds before any call)."""
        out = (ctypes.c_int64 * (len(self.dims) + 1))()
        _check(lib().ntt_plan_get_ranks(self.handle, out), "ntt_plan_get_ranks")
        return tuple(int(v) for v in out)

    def core_shapes(self):
        """Shapes of the core buffers to allocate (with the rank rule: the bounds)."""
        ranks = self.ranks if self.ranks is not None else self.max_ranks
        return [(ranks[k], self.dims[k], ranks[k + 1]) for k in range(len(self.dims))]

    def core_views(self, cores):
        """The cores at the plan's current ranks, as views of buffers of core_shapes()."""
        ranks = self.current_ranks()
        return [c.reshape(-1)[:ranks[k] * self.dims[k] * ranks[k + 1]].view(ranks[k], self.dims[k], ranks[k + 1])
                for k, c in enumerate(cores)]

    def destroy(self):
        if self.handle:
            lib().ntt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def ntt_plan_create(dims, ranks, iters, eps_mu=1e-12, x_dtype="f32", refine_iters=0, seed=0, tol=0.0,
                    check_every=10, route="auto", eager=False, eps_rank=0.0, rank_cap=0, solver="mu"):
    """route: one of ROUTES (ntt_route); eager: enqueue every call instead of a cached graph;
    ranks=None: Algorithm 2's rank rule with eps_rank (> 0) and optional rank_cap;
    solver: "mu" (multiplicative updates) or "bcd" (Algorithm 3)."""
    dims = tuple(int(n) for n in dims)
    ranks = tuple(int(r) for r in ranks) if ranks is not None else None
    d_arr = _i64arr(dims)
    r_arr = _i64arr(ranks) if ranks is not None else None
    desc = _PlanDesc()
    desc.d = len(dims)
    desc.dims = ctypes.cast(d_arr, ctypes.POINTER(ctypes.c_int64))
    desc.ranks = ctypes.cast(r_arr, ctypes.POINTER(ctypes.c_int64)) if r_arr is not None else None
    desc.iters = int(iters)
    desc.eps_mu = float(eps_mu)
    desc.x_dtype = NTT_BF16 if x_dtype == "bf16" else NTT_F32
    desc.refine_iters = int(refine_iters)
    desc.seed = int(seed)
    desc.tol = float(tol)
    desc.check_every = int(check_every)
    desc.route = _route(route)
    desc.flags = NTT_PLAN_EAGER if eager else 0
    desc.eps_rank = float(eps_rank)
    desc.rank_cap = int(rank_cap)
    if solver not in SOLVERS:
        raise ValueError(f"solver must be one of {sorted(SOLVERS)}")
    desc.solver = SOLVERS[solver]
    h = ctypes.c_void_p()
    _check(lib().ntt_plan_create(ctypes.byref(desc), ctypes.byref(h)), "ntt_plan_create")
    plan = Plan(h, dims, ranks, int(iters), x_dtype, int(refine_iters))
    plan.max_ranks = plan.current_ranks()
    plan.seed = int(seed)
    return plan


def _ptr_array(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*[p.value if isinstance(p, ctypes.c_void_p) else p
                                           for p in ptrs])


def ntt_decompose(plan, A, cores, workspace, stream=None):
    import torch
    a = _dev_ptr(A, torch.float32, "A")
    cps = _ptr_array([_dev_ptr(c, torch.float32, "core") for c in cores])
    w = _dev_ptr(workspace, None, "workspace")
    _check(lib().ntt_decompose(plan.handle, a, cps, w, _stream_ptr(stream)), "ntt_decompose")


def ntt_unfolding_size(plan, s):
    """Floats of the unfolding H_s that stage s reads (1 <= s <= d - 2)."""
    v = ctypes.c_int64()
    _check(lib().ntt_unfolding_size(plan.handle, int(s), ctypes.byref(v)), "ntt_unfolding_size")
    return v.value


def ntt_decompose_stages(plan, s0, s1, X_in, cores, H_out, workspace, stream=None):
    """Stages s0 .. s1-1 of the plan (checkpoint / resume at stage granularity):
    X_in is A (s0 == 0) or the unfolding H_{s0} an earlier call returned in
    H_out; cores s0 .. s1-1 are written (and the last core when s1 == d - 1);
    H_out (CUDA float32 of ntt_unfolding_size(plan, s1) floats, or None when
    s1 == d - 1) receives H_{s1}."""
    import torch
    x = _dev_ptr(X_in, torch.float32, "X_in")
    cps = _ptr_array([_dev_ptr(c, torch.float32, "core") for c in cores])
    h = None if H_out is None else _dev_ptr(H_out, torch.float32, "H_out")
    w = _dev_ptr(workspace, None, "workspace")
    _check(lib().ntt_decompose_stages(plan.handle, int(s0), int(s1), x, cps, h, w, _stream_ptr(stream)),
           "ntt_decompose_stages")


def save_checkpoint(path, plan, s, cores, H):
    """Write a stage checkpoint to `path` (numpy .npz, host): the cores
    0 .. s-1, the unfolding H_s that stage s reads, and the plan's dims, ranks
    and seed (the initial factors of stage k come from (seed, k))."""
    import numpy as np
    np.savez(path, stage=np.int64(s), dims=np.asarray(plan.dims, np.int64), ranks=np.asarray(plan.ranks, np.int64),
             seed=np.uint64(plan.seed), H=H.detach().cpu().numpy(),
             **{f"core{k}": cores[k].detach().cpu().numpy() for k in range(s)})


def load_checkpoint(path, plan):
    """Read a checkpoint written by save_checkpoint for the same plan: returns
    (stage, [host cores 0 .. stage-1], host H_stage)."""
    import numpy as np
    z = np.load(path)
    if (tuple(z["dims"]) != tuple(plan.dims) or tuple(z["ranks"]) != tuple(plan.ranks)
            or int(z["seed"]) != int(plan.seed)):
        raise ValueError("checkpoint belongs to a different plan (dims, ranks or seed)")
    s = int(z["stage"])
    return s, [z[f"core{k}"] for k in range(s)], z["H"]


def ntt_decompose_host(plan, A_host, cores_host, workspace, err_host=None, stream=None):
    """A_host, cores_host: CPU float32 tensors (pinned for asynchrony); err_host:
    optional CPU float64 tensor of 3 entries receiving Eq. (3) of the result."""
    import torch
    for t in [A_host, *cores_host]:
        if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError("host tensors must be contiguous CPU float32")
    eptr = None
    if err_host is not None:
        if err_host.is_cuda or err_host.dtype != torch.float64 or err_host.numel() < 3:
            raise TypeError("err_host must be a CPU float64 tensor of >= 3 entries")
        eptr = ctypes.c_void_p(err_host.data_ptr())
    cps = _ptr_array([c.data_ptr() for c in cores_host])
    w = _dev_ptr(workspace, None, "workspace")
    _check(lib().ntt_decompose_host(plan.handle, ctypes.c_void_p(A_host.data_ptr()), cps, eptr, w,
                                    _stream_ptr(stream)), "ntt_decompose_host")


def ntt_plan_get_stats(plan):
    st = _Stats()
    code = lib().ntt_plan_get_stats(plan.handle, ctypes.byref(st))
    d = st.d
    out = dict(status=STATUS.get(st.status, st.status), total_ms=st.total_ms,
               launches=st.launches, stages=[])
    for s in range(d - 1):
        out["stages"].append(dict(
            m=st.m[s], n=st.n[s], r=st.r[s], iters=st.iters[s], xnorm2=st.xnorm2[s],
            obj_first=st.obj_first[s], obj_last=st.obj_last[s], resid=st.resid[s],
            stage_ms=st.stage_ms[s], iter_ms=st.iter_ms[s], alg_bytes=st.alg_bytes[s],
            engine=ENGINES.get(st.engine[s], st.engine[s])))
    _check(code, "ntt_plan_get_stats")
    return out


def nmf_mu_workspace_size(m, n, r, x_dtype="f32", route="auto"):
    b = ctypes.c_size_t(0)
    _check(lib().nmf_mu_workspace_size_route(int(m), int(n), int(r), NTT_BF16 if x_dtype == "bf16" else NTT_F32,
                                             _route(route), ctypes.byref(b)), "nmf_mu_workspace_size_route")
    return b.value


def nmf_mu_step(X, W, H, iters, eps_mu=1e-12, obj=None, workspace=None, stream=None, route="auto",
                engine=None):
    """`iters` MU iterations on W (m x r) and H (r x n) in place; X is float32 or bfloat16.
    route: one of ROUTES (nmf_mu_step_route); engine: optional list that receives
    the name of the pass that ran."""
    import torch
    if X.dim() != 2 or W.dim() != 2 or H.dim() != 2:
        raise ValueError("X, W, H must be matrices")
    m, n = X.shape
    r = W.shape[1]
    if W.shape[0] != m or H.shape != (r, n):
        raise ValueError("shape mismatch")
    xd = "bf16" if X.dtype == torch.bfloat16 else "f32"
    if workspace is None:
        workspace = empty_workspace(nmf_mu_workspace_size(m, n, r, xd, route), X.device)
    optr = _dev_ptr(obj, torch.float64, "obj") if obj is not None else None
    eng = ctypes.c_int(-1)
    _check(lib().nmf_mu_step_route(m, n, r, _dev_ptr(X, None, "X"),
                                   NTT_BF16 if xd == "bf16" else NTT_F32,
                                   _dev_ptr(W, torch.float32, "W"), _dev_ptr(H, torch.float32, "H"),
                                   int(iters), float(eps_mu), optr, _dev_ptr(workspace, None, "ws"),
                                   _stream_ptr(stream), _route(route), ctypes.byref(eng)), "nmf_mu_step")
    if engine is not None:
        engine.append(ENGINES.get(eng.value, eng.value))
    return workspace


def nmf_mu_step_noalloc(X, W, H, iters, eps_mu=1e-12, obj=None, stream=None):
    """nmf_mu_step for callers that cannot allocate device memory: the scratch is
    the library's own 8 MiB device array (see include/ntt.h); shapes that need
    more raise NTTError (NTT_ERR_OOM).  Calls on one device must not overlap."""
    import torch
    if X.dim() != 2 or W.dim() != 2 or H.dim() != 2:
        raise ValueError("X, W, H must be matrices")
    m, n = X.shape
    r = W.shape[1]
    if W.shape[0] != m or H.shape != (r, n):
        raise ValueError("shape mismatch")
    xd = NTT_BF16 if X.dtype == torch.bfloat16 else NTT_F32
    optr = _dev_ptr(obj, torch.float64, "obj") if obj is not None else None
    _check(lib().nmf_mu_step_noalloc(m, n, r, _dev_ptr(X, None, "X"), xd,
                                     _dev_ptr(W, torch.float32, "W"),
                                     _dev_ptr(H, torch.float32, "H"), int(iters), float(eps_mu),
                                     optr, _stream_ptr(stream)), "nmf_mu_step_noalloc")


def nmf_bcd_workspace_size(m, n, r):
    b = ctypes.c_size_t(0)
    _check(lib().nmf_bcd_workspace_size(int(m), int(n), int(r), ctypes.byref(b)), "nmf_bcd_workspace_size")
    return b.value


def nmf_bcd_step(X, W, H, iters, obj=None, workspace=None, stream=None):
    """`iters` BCD iterations (Algorithm 3) on float32 CUDA X, W (m x r), H (r x n):
    initial factors in, the last accepted iterate out; obj: optional float64 CUDA
    tensor of `iters` entries receiving the accepted objective after each iteration."""
    import torch
    m, n = X.shape
    r = W.shape[1]
    if W.shape[0] != m or H.shape != (r, n):
        raise ValueError("shape mismatch")
    if workspace is None:
        workspace = empty_workspace(nmf_bcd_workspace_size(m, n, r), X.device)
    optr = _dev_ptr(obj, torch.float64, "obj") if obj is not None else None
    _check(lib().nmf_bcd_step(m, n, r, _dev_ptr(X, torch.float32, "X"), _dev_ptr(W, torch.float32, "W"),
                              _dev_ptr(H, torch.float32, "H"), int(iters), optr, _dev_ptr(workspace, None, "ws"),
                              _stream_ptr(stream)), "nmf_bcd_step")
    return workspace


def nmf_mu_step_host(X_host, W, H, iters, chunk_cols, eps_mu=1e-12, obj=None, workspace=None, stream=None):
    """Out-of-core MU: X_host is a CPU float32 tensor (pin it for asynchronous
    copies), streamed in column chunks every iteration; W, H CUDA float32 in place."""
    import torch
    if X_host.is_cuda or X_host.dtype != torch.float32 or not X_host.is_contiguous():
        raise TypeError("X_host must be a contiguous CPU float32 tensor")
    m, n = X_host.shape
    r = W.shape[1]
    if W.shape[0] != m or H.shape != (r, n):
        raise ValueError("shape mismatch")
    if workspace is None:
        b = ctypes.c_size_t()
        _check(lib().nmf_mu_host_workspace_size(m, n, r, int(chunk_cols), ctypes.byref(b)),
               "nmf_mu_host_workspace_size")
        workspace = empty_workspace(b.value, W.device)
    optr = _dev_ptr(obj, torch.float64, "obj") if obj is not None else None
    _check(lib().nmf_mu_step_host(m, n, r, ctypes.c_void_p(X_host.data_ptr()), _dev_ptr(W, torch.float32, "W"),
                                  _dev_ptr(H, torch.float32, "H"), int(iters), ctypes.c_float(eps_mu), optr,
                                  int(chunk_cols), _dev_ptr(workspace, None, "ws"), _stream_ptr(stream)),
           "nmf_mu_step_host")
    return workspace


class ShardOps:
    """The device halves of one rank's column-sharded MU iteration (include/ntt.h
    nmf_mu_shard_*): X_shard m x n_shard, H_shard r x n_shard, W m x r (CUDA float32)."""

    def __init__(self, m, n_shard, r, eps_mu=1e-12, device=None, stream=None):
        import torch
        wsb, pqn = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().nmf_mu_shard_sizes(int(m), int(n_shard), int(r), ctypes.byref(wsb), ctypes.byref(pqn)),
               "nmf_mu_shard_sizes")
        self.m, self.n, self.r, self.eps, self.stream = int(m), int(n_shard), int(r), float(eps_mu), stream
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.ws = empty_workspace(wsb.value, dev)
        self.pq = torch.zeros(pqn.value, dtype=torch.float64, device=dev)
        self.xn = torch.zeros(1, dtype=torch.float64, device=dev)

    def norm2(self, X):
        import torch
        _check(lib().nmf_mu_shard_norm(self.m, self.n, _dev_ptr(X, torch.float32, "X"),
                                       _dev_ptr(self.xn, torch.float64, "out"), _dev_ptr(self.ws, None, "ws"),
                                       _stream_ptr(self.stream)), "nmf_mu_shard_norm")
        return self.xn

    def local_pass(self, X, W, H):
        import torch
        _check(lib().nmf_mu_shard_pass(self.m, self.n, self.r, _dev_ptr(X, torch.float32, "X"),
                                       _dev_ptr(W, torch.float32, "W"), _dev_ptr(H, torch.float32, "H"),
                                       ctypes.c_float(self.eps), _dev_ptr(self.pq, torch.float64, "pq"),
                                       _dev_ptr(self.ws, None, "ws"), _stream_ptr(self.stream)), "nmf_mu_shard_pass")
        return self.pq

    def update(self, pq, W, xnorm2, obj=None):
        import torch
        optr = _dev_ptr(obj, torch.float64, "obj") if obj is not None else None
        _check(lib().nmf_mu_shard_update(self.m, self.r, _dev_ptr(pq, torch.float64, "pq"),
                                         _dev_ptr(W, torch.float32, "W"), ctypes.c_float(self.eps),
                                         ctypes.c_double(float(xnorm2)), optr, _dev_ptr(self.ws, None, "ws"),
                                         _stream_ptr(self.stream)), "nmf_mu_shard_update")


def sharded_nmf_mu(X_shard, W, H_shard, iters, ops, all_reduce=None):
    """Column-sharded multiplicative updates (Section III-B's 1-D column
    distribution): this rank updates its H columns and W (replicated) in place.
    ops: ShardOps of this rank (or any object with norm2 / local_pass / update);
    all_reduce: in-place sum of a tensor over the ranks (e.g.
    torch.distributed.all_reduce), None on one rank.  Per iteration the only
    exchange is the all-reduce of [P ; Q].  Returns the objective after each
    iteration (a list of floats)."""
    reduce = all_reduce or (lambda t: None)
    xn = ops.norm2(X_shard)
    reduce(xn)
    xnorm2 = float(xn[0])
    trace = []
    for _ in range(int(iters)):
        pq = ops.local_pass(X_shard, W, H_shard)
        reduce(pq)
        obj = pq.new_zeros(1)
        ops.update(pq, W, xnorm2, obj)
        trace.append(float(obj[0]))
    return trace


def shard_bounds(n, world):
    """Contiguous column blocks of n columns over `world` ranks: rank p owns
    columns bounds[p] .. bounds[p + 1] - 1 (block sizes differ by at most one)."""
    return [int(n) * p // int(world) for p in range(int(world) + 1)]


def handoff_plan(r, n, n_next_dim, world):
    """The exchange that turns a column-sharded H (r x n, blocks shard_bounds(n,
    world)) into the column-sharded next unfolding X' = reshape(H, r n_next_dim,
    n / n_next_dim) (C order: X'[i n_next_dim + j, c] = H[i, j n' + c], n' =
    n / n_next_dim).  Returns (n', sends) with sends[q][p] = the H columns, in
    increasing order, that rank q sends to rank p: those j n' + c owned by q
    with c in p's block of X'.  Every column of H goes to exactly one rank."""
    if n % n_next_dim:
        raise ValueError("n must be a multiple of the next mode size")
    n2 = n // n_next_dim
    hb, xb = shard_bounds(n, world), shard_bounds(n2, world)
    sends = [[[] for _ in range(world)] for _ in range(world)]
    for q in range(world):
        for k in range(hb[q], hb[q + 1]):
            c = k % n2
            p = next(i for i in range(world) if xb[i] <= c < xb[i + 1])
            sends[q][p].append(k)
    return n2, sends


def sharded_ntt_decompose(X_shard, dims, ranks, iters, rank, world, ops_factory, init, all_reduce=None,
                          exchange=None):
    """Algorithm 2 on column-sharded unfoldings (Section III-B's 1-D column
    distribution), every stage's NMF by sharded_nmf_mu.  This rank holds the
    columns shard_bounds(n, world)[rank] .. of the first unfolding (dims[0] x
    prod(dims[1:])).  Per stage: the sharded MU iterations (all-reduce of
    [P ; Q]), the column-L1 hand-off of W (replicated) folded into this rank's H
    rows, the core from W, then the exchange of H columns that lays out the next
    unfolding in the same column blocks (handoff_plan: an all-to-all; the last
    core, H of the last stage, is gathered on every rank).
      ops_factory(m, n_shard, r): ShardOps (or any object with its interface)
      init(m, n, r, stage, c0, c1): (W0 m x r, H0 columns c0 .. c1 - 1), the
        unsharded initial factors' values (the counter RNG is column-indexable)
      all_reduce(t): in-place sum over the ranks (None on one rank)
      exchange(sends): sends[p] = tensor (rows x k_p) for rank p; returns the
        list of tensors received from every rank (None on one rank).
    Returns (cores, traces): cores as tensors on every rank."""
    import torch
    d = len(dims)
    if len(ranks) != d + 1 or ranks[0] != 1 or ranks[-1] != 1:
        raise ValueError("ranks must have d + 1 entries with r_0 = r_d = 1")
    xchg = exchange or (lambda sends: sends)
    cores, traces = [], []
    X = X_shard
    for s in range(d - 1):
        m, r = ranks[s] * dims[s], ranks[s + 1]
        n = 1
        for v in dims[s + 1:]:
            n *= v
        b = shard_bounds(n, world)
        c0, c1 = b[rank], b[rank + 1]
        if X.shape != (m, c1 - c0):
            raise ValueError(f"stage {s}: this rank's unfolding block must be {m} x {c1 - c0}")
        W0, H0 = init(m, n, r, s, c0, c1)
        W = W0.clone()
        H = H0.clone()
        traces.append(sharded_nmf_mu(X, W, H, iters, ops_factory(m, c1 - c0, r), all_reduce))
        # column-L1 hand-off: W's column sums are the same on every rank
        norms = W.sum(dim=0)
        scale = torch.where(norms > 0, norms, torch.ones_like(norms))
        W = W / scale
        H = H * scale[:, None]
        cores.append(W.reshape(ranks[s], dims[s], r))
        last = s == d - 2
        if last:
            # the last core: every rank's H columns to every rank
            got = xchg([H for _ in range(world)])
            cores.append(torch.cat(list(got), dim=1).reshape(r, dims[d - 1], 1))
            break
        n2, plan = handoff_plan(r, n, dims[s + 1], world)
        sends = []
        for p in range(world):
            cols = torch.tensor(plan[rank][p], dtype=torch.long) - c0
            sends.append(H[:, cols.to(H.device)].contiguous() if cols.numel() else H[:, :0].contiguous())
        got = xchg(sends)
        xb = shard_bounds(n2, world)
        e0, e1 = xb[rank], xb[rank + 1]
        Xn = H.new_zeros((r * dims[s + 1], e1 - e0))
        for q in range(world):
            ks = torch.tensor(plan[q][rank], dtype=torch.long)
            if ks.numel() == 0:
                continue
            j, c = ks // n2, ks % n2 - e0
            blk = got[q]                                  # r x len(ks), columns in increasing k
            for i in range(r):
                Xn[i * dims[s + 1] + j.to(Xn.device), c.to(Xn.device)] = blk[i]
        X = Xn
    return cores, traces


def _many_args(Xs, Ws, Hs):
    import torch
    count = len(Xs)
    if count < 1 or len(Ws) != count or len(Hs) != count:
        raise ValueError("Xs, Ws, Hs: same non-zero length")
    m, n, r = [], [], []
    for X, W, H in zip(Xs, Ws, Hs):
        if X.dim() != 2 or W.dim() != 2 or H.dim() != 2:
            raise ValueError("X, W, H must be matrices")
        if W.shape[0] != X.shape[0] or H.shape != (W.shape[1], X.shape[1]):
            raise ValueError("shape mismatch")
        m.append(X.shape[0]); n.append(X.shape[1]); r.append(W.shape[1])
    return count, _i64arr(m), _i64arr(n), (ctypes.c_int * count)(*r)


def nmf_mu_many_workspace_size(shapes):
    """shapes: list of (m, n, r)."""
    count = len(shapes)
    b = ctypes.c_size_t()
    _check(lib().nmf_mu_many_workspace_size(count, _i64arr([s[0] for s in shapes]),
                                            _i64arr([s[1] for s in shapes]),
                                            (ctypes.c_int * count)(*[s[2] for s in shapes]),
                                            ctypes.byref(b)), "nmf_mu_many_workspace_size")
    return b.value


def nmf_mu_many(Xs, Ws, Hs, iters, eps_mu=1e-12, workspace=None, stream=None):
    """`iters` MU iterations of every (X_i, W_i, H_i), in place on W_i, H_i (FP32 CUDA tensors)."""
    import torch
    count, m, n, r = _many_args(Xs, Ws, Hs)
    if workspace is None:
        workspace = empty_workspace(nmf_mu_many_workspace_size(
            [(X.shape[0], X.shape[1], W.shape[1]) for X, W in zip(Xs, Ws)]), Xs[0].device)
    vp = ctypes.c_void_p
    xa = (vp * count)(*[_dev_ptr(X, torch.float32, "X") for X in Xs])
    wa = (vp * count)(*[_dev_ptr(W, torch.float32, "W") for W in Ws])
    ha = (vp * count)(*[_dev_ptr(H, torch.float32, "H") for H in Hs])
    _check(lib().nmf_mu_many(count, m, n, r, xa, wa, ha, int(iters), ctypes.c_float(eps_mu),
                             _dev_ptr(workspace, None, "ws"), _stream_ptr(stream)), "nmf_mu_many")
    return workspace


def ntt_status_of_workspace(workspace):
    v = ctypes.c_int(0)
    _check(lib().ntt_status_of_workspace(_dev_ptr(workspace, None, "ws"), ctypes.byref(v)),
           "ntt_status_of_workspace")
    return STATUS.get(v.value, v.value)


def ntt_wait_probe(workspace, limit_ns, stream=None):
    """Enqueue the bounded-wait probe on an nmf_mu_step workspace: its status
    word reads NTT_ERR_TIMEOUT once the stream has run it (include/ntt.h)."""
    _check(lib().ntt_wait_probe(_dev_ptr(workspace, None, "ws"), int(limit_ns), _stream_ptr(stream)),
           "ntt_wait_probe")


def ntt_rank_workspace_size(m, n):
    b = ctypes.c_size_t(0)
    _check(lib().ntt_rank_workspace_size(int(m), int(n), ctypes.byref(b)), "ntt_rank_workspace_size")
    return b.value


def ntt_singular_values(X, sigma=None, workspace=None, stream=None):
    """Singular values of a CUDA float32 matrix X (non-increasing, float64 CUDA tensor)."""
    import torch
    m, n = X.shape
    if sigma is None:
        sigma = torch.empty(min(m, n), dtype=torch.float64, device=X.device)
    if workspace is None:
        workspace = empty_workspace(ntt_rank_workspace_size(m, n), X.device)
    _check(lib().ntt_singular_values(m, n, _dev_ptr(X, torch.float32, "X"), _dev_ptr(sigma, torch.float64, "sigma"),
                                     _dev_ptr(workspace, None, "ws"), _stream_ptr(stream)), "ntt_singular_values")
    return sigma


def ntt_select_rank(X, eps_rank, rank_cap=0, rank=None, sigma=None, workspace=None, stream=None):
    """Algorithm 2's rank of a CUDA float32 matrix X into `rank` (int32 CUDA tensor, 1 entry)."""
    import torch
    m, n = X.shape
    if rank is None:
        rank = torch.zeros(1, dtype=torch.int32, device=X.device)
    if workspace is None:
        workspace = empty_workspace(ntt_rank_workspace_size(m, n), X.device)
    sp = _dev_ptr(sigma, torch.float64, "sigma") if sigma is not None else None
    _check(lib().ntt_select_rank(m, n, _dev_ptr(X, torch.float32, "X"), float(eps_rank), int(rank_cap),
                                 _dev_ptr(rank, torch.int32, "rank"), sp, _dev_ptr(workspace, None, "ws"),
                                 _stream_ptr(stream)), "ntt_select_rank")
    return rank


def ntt_uniform_init(seed, stage, restart, matrix, out, stream=None):
    import torch
    _check(lib().ntt_uniform_init(int(seed), int(stage), int(restart), int(matrix), out.numel(),
                                  _dev_ptr(out, torch.float32, "out"), _stream_ptr(stream)),
           "ntt_uniform_init")


def ntt_reconstruct_workspace_size(dims, ranks):
    b = ctypes.c_size_t(0)
    _check(lib().ntt_reconstruct_workspace_size(len(dims), _i64arr(dims), _i64arr(ranks),
                                                ctypes.byref(b)), "ntt_reconstruct_workspace_size")
    return b.value


def ntt_reconstruct(dims, ranks, cores, out, workspace=None, stream=None):
    import torch
    if workspace is None:
        workspace = empty_workspace(ntt_reconstruct_workspace_size(dims, ranks), out.device)
    cps = _ptr_array([_dev_ptr(c, torch.float32, "core") for c in cores])
    _check(lib().ntt_reconstruct(len(dims), _i64arr(dims), _i64arr(ranks), cps,
                                 _dev_ptr(out, torch.float32, "out"),
                                 _dev_ptr(workspace, None, "ws"), _stream_ptr(stream)),
           "ntt_reconstruct")
    return workspace


def ntt_rel_error(dims, ranks, cores, A, err, workspace=None, stream=None):
    """err: CUDA float64 tensor of >= 3 entries (rel error, ||A - A~||^2, ||A||^2)."""
    import torch
    if workspace is None:
        workspace = empty_workspace(ntt_reconstruct_workspace_size(dims, ranks), A.device)
    cps = _ptr_array([_dev_ptr(c, torch.float32, "core") for c in cores])
    _check(lib().ntt_rel_error(len(dims), _i64arr(dims), _i64arr(ranks), cps,
                               _dev_ptr(A, torch.float32, "A"), _dev_ptr(err, torch.float64, "err"),
                               _dev_ptr(workspace, None, "ws"), _stream_ptr(stream)),
           "ntt_rel_error")
    return workspace


class Batch:
    """Plan of the batched form: B instances (dims, ranks), restarts per stage."""

    def __init__(self, instances, iters, restarts, eps_mu=1e-12, seed=0):
        self.instances = [(tuple(int(x) for x in d), tuple(int(x) for x in r)) for d, r in instances]
        B = len(self.instances)
        d_arr = (ctypes.c_int * B)(*[len(d) for d, _ in self.instances])
        dims = _i64arr([x for d, _ in self.instances for x in d])
        ranks = _i64arr([x for _, r in self.instances for x in r])
        h = ctypes.c_void_p()
        _check(lib().ntt_batch_create(B, d_arr, dims, ranks, int(iters), int(restarts),
                                      float(eps_mu), int(seed), ctypes.byref(h)), "ntt_batch_create")
        self.handle = h
        a, c, w = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().ntt_batch_sizes(h, ctypes.byref(a), ctypes.byref(c), ctypes.byref(w)),
               "ntt_batch_sizes")
        self.input_floats, self.core_floats, self.workspace_bytes = a.value, c.value, w.value
        io = (ctypes.c_int64 * B)()
        co = (ctypes.c_int64 * sum(len(d) for d, _ in self.instances))()
        _check(lib().ntt_batch_offsets(h, io, co), "ntt_batch_offsets")
        self.input_off = list(io)
        self.core_off = list(co)

    def core_views(self, cores_packed):
        """Per instance, the list of its cores as views of the packed buffer."""
        out, c = [], 0
        for dims, ranks in self.instances:
            lst = []
            for k, n in enumerate(dims):
                size = ranks[k] * n * ranks[k + 1]
                lst.append(cores_packed[self.core_off[c]:self.core_off[c] + size]
                           .view(ranks[k], n, ranks[k + 1]))
                c += 1
            out.append(lst)
        return out

    def destroy(self):
        if getattr(self, "handle", None):
            lib().ntt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def ntt_batch_create(instances, iters, restarts, eps_mu=1e-12, seed=0):
    return Batch(instances, iters, restarts, eps_mu, seed)


def ntt_batch_tune(batch, A_packed, cores_packed, workspace, probe_iters=10, cache_path=None, stream=None):
    """Autotune the grouped engine's CTA split per stage (include/ntt.h); returns
    dict(split=[per stage], from_cache=..., timed=...)."""
    import torch
    path = cache_path.encode() if cache_path else None
    _check(lib().ntt_batch_tune(batch.handle, _dev_ptr(A_packed, torch.float32, "A"),
                                _dev_ptr(cores_packed, torch.float32, "cores"),
                                _dev_ptr(workspace, None, "workspace"), _stream_ptr(stream), int(probe_iters), path),
           "ntt_batch_tune")
    return ntt_batch_get_tuning(batch)


def ntt_batch_get_tuning(batch):
    nst = max(len(d) for d, _ in batch.instances) - 1
    split = (ctypes.c_int * max(1, nst))()
    fc, tm = ctypes.c_int(), ctypes.c_int()
    _check(lib().ntt_batch_get_tuning(batch.handle, nst, split, ctypes.byref(fc), ctypes.byref(tm)),
           "ntt_batch_get_tuning")
    return {"split": list(split)[:nst], "from_cache": fc.value, "timed": tm.value}


def ntt_decompose_batched(batch, A_packed, cores_packed, workspace, stream=None):
    """A_packed / cores_packed: CUDA float32 tensors laid out by batch.input_off / core_off.
    Asynchronous (one cached CUDA graph); the status word is ntt_status_of_workspace(workspace)."""
    import torch
    _check(lib().ntt_decompose_batched(batch.handle, _dev_ptr(A_packed, torch.float32, "A"),
                                       _dev_ptr(cores_packed, torch.float32, "cores"),
                                       _dev_ptr(workspace, None, "workspace"), _stream_ptr(stream)),
           "ntt_decompose_batched")


def _info_dict(info):
    return {"state": JOB_STATES.get(info.state, info.state), "status": STATUS.get(info.status, info.status),
            "stage": info.stage, "t_submit": info.t_submit, "t_admit": info.t_admit, "t_done": info.t_done,
            "footprint_bytes": info.footprint_bytes}


def ntt_server_job_footprint(dims, ranks, x_dtype="f32"):
    b = ctypes.c_size_t()
    _check(lib().ntt_server_job_footprint(len(dims), _i64arr(dims), _i64arr(ranks),
                                          NTT_BF16 if x_dtype == "bf16" else NTT_F32, ctypes.byref(b)),
           "ntt_server_job_footprint")
    return b.value


class ServerJob:
    """A submitted job: `cores` (host float32, filled when done) and the input it keeps alive."""

    def __init__(self, job_id, dims, ranks, A, cores):
        self.id, self.dims, self.ranks, self._A, self.cores = job_id, dims, ranks, A, cores

    def core_views(self):
        out, off = [], 0
        for k, n in enumerate(self.dims):
            size = self.ranks[k] * n * self.ranks[k + 1]
            out.append(self.cores[off:off + size].view(self.ranks[k], n, self.ranks[k + 1]))
            off += size
        return out


class Server:
    """Serving form (include/ntt.h): continuous batching of nTT jobs on the current device."""

    def __init__(self, hbm_budget_bytes, max_jobs=256, tick_iters=10, stage_iters=100, eps_mu=1e-12):
        cfg = _ServerConfig(int(hbm_budget_bytes), int(max_jobs), int(tick_iters), int(stage_iters),
                            float(eps_mu))
        h = ctypes.c_void_p()
        _check(lib().ntt_server_create(ctypes.byref(cfg), ctypes.byref(h)), "ntt_server_create")
        self.handle = h

    def submit(self, A, dims, ranks, seed=0, pin_output=True):
        """A: host torch tensor (float32 or bfloat16, contiguous, prod(dims) entries)."""
        import torch
        if A.is_cuda or not A.is_contiguous() or A.numel() != int(np.prod(dims)):
            raise ValueError("A must be a contiguous host tensor of prod(dims) entries")
        if A.dtype not in (torch.float32, torch.bfloat16):
            raise TypeError("A must be float32 or bfloat16")
        dims = tuple(int(x) for x in dims)
        ranks = tuple(int(x) for x in ranks)
        ncore = sum(ranks[k] * n * ranks[k + 1] for k, n in enumerate(dims))
        cores = torch.zeros(ncore, dtype=torch.float32, pin_memory=pin_output)
        jid = ctypes.c_int64()
        _check(lib().ntt_server_submit(self.handle, len(dims), _i64arr(dims), _i64arr(ranks),
                                       ctypes.c_void_p(A.data_ptr()),
                                       NTT_BF16 if A.dtype == torch.bfloat16 else NTT_F32,
                                       ctypes.c_uint64(int(seed)), ctypes.c_void_p(cores.data_ptr()),
                                       ctypes.byref(jid)), "ntt_server_submit")
        return ServerJob(jid.value, dims, ranks, A, cores)

    def poll(self, job):
        info = _JobInfo()
        _check(lib().ntt_server_poll(self.handle, ctypes.c_int64(job.id), ctypes.byref(info)), "ntt_server_poll")
        return _info_dict(info)

    def wait(self, job, timeout=-1.0):
        """Block until `job` is done; returns its info dict (raises NTTError if it failed)."""
        info = _JobInfo()
        code = lib().ntt_server_wait(self.handle, ctypes.c_int64(job.id), ctypes.c_double(timeout),
                                     ctypes.byref(info))
        _check(code, "ntt_server_wait")
        return _info_dict(info)

    def stats(self):
        st = _ServerStats()
        _check(lib().ntt_server_get_stats(self.handle, ctypes.byref(st)), "ntt_server_get_stats")
        return {f: getattr(st, f) for f, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().ntt_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ntt_compression_ratio(dims, ranks):
    return lib().ntt_compression_ratio(len(dims), _i64arr(dims), _i64arr(ranks))


def decompose(A, ranks, iters, eps_mu=1e-12, x_dtype="f32", refine_iters=0, seed=0, stream=None, tol=0.0,
              check_every=10, route="auto", eps_rank=0.0, rank_cap=0):
    """Convenience wrapper: returns (cores, stats) for a CUDA float32 tensor A
    (ranks=None: Algorithm 2's rank rule with eps_rank)."""
    import torch
    plan = ntt_plan_create(tuple(A.shape), ranks, iters, eps_mu, x_dtype, refine_iters, seed, tol, check_every,
                           route, eps_rank=eps_rank, rank_cap=rank_cap)
    ws = empty_workspace(plan.workspace_size(), A.device)
    cores = [torch.empty(s, dtype=torch.float32, device=A.device) for s in plan.core_shapes()]
    ntt_decompose(plan, A.contiguous(), cores, ws, stream)
    stats = ntt_plan_get_stats(plan)
    cores = [c.clone() for c in plan.core_views(cores)]
    plan.destroy()
    return cores, stats


def build(**kw):
    from ._build import build as _b
    return _b(**kw)

"""Seeded synthetic inputs for the non-negative tensor-train (nTT) hot path.

Shared by the tests, the benchmark and the oracle checks.  This module only
draws random numbers and assembles input tensors following the paper's data
recipe (Section IV-A "Data Generation": every TT core entry is drawn at random,
and the tensor is the product of the cores, formed by reshaping the cores into
matrices and multiplying them).  It holds none of the multiplicative-update,
objective or error arithmetic of the method.

Everything is deterministic in the seed, independent of the number of threads
used to build a large tensor (each row block draws its noise from its own
spawned seed sequence).
"""

from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

__all__ = [
    "CONFIGS",
    "tt_cores",
    "tt_tensor",
    "uniform_matrix",
    "stage_shapes",
    "batched_instances",
    "serving_requests",
]

# Workload recipes.  Sizes, rank patterns, core distributions, noise level and
# iteration counts of the five workloads; seeds are fixed per workload.
CONFIGS = {
    # 4-way 8x8x8x8, ranks (1,3,3,3,1), U[0,1) cores, |N(0, (0.01 mean)^2)| noise
    "c1_8x4": dict(dims=(8, 8, 8, 8), ranks=(1, 3, 3, 3, 1), core_dist="uniform",
                   noise=0.01, iters=500, data_seed=1, init_seed=101, x_dtype="f32"),
    # 6-way 32^6 (1.07e9 entries, 4.3 GB FP32), ranks (1,8,16,16,16,8,1)
    "c2_32x6": dict(dims=(32,) * 6, ranks=(1, 8, 16, 16, 16, 8, 1), core_dist="uniform",
                    noise=0.01, iters=200, data_seed=2, init_seed=102, x_dtype="f32"),
    # 8-way 16^8 (4.3e9 entries), exponential(1) cores, BF16-stored X + FP32 refinement
    "c3_16x8": dict(dims=(16,) * 8, ranks=(1, 16, 32, 32, 32, 32, 32, 16, 1),
                    core_dist="exponential", noise=0.01, iters=200, refine_iters=5,
                    data_seed=3, init_seed=103, x_dtype="bf16"),
    # Same recipe as c2 at 16^6: a shape the oracle can finish end to end.
    "c2_small_16x6": dict(dims=(16,) * 6, ranks=(1, 8, 16, 16, 16, 8, 1), core_dist="uniform",
                          noise=0.01, iters=200, data_seed=2, init_seed=102, x_dtype="f32"),
}


def tt_cores(dims, ranks, dist="uniform", seed=0):
    """Random non-negative TT cores G_k of shape (r_{k-1}, n_k, r_k), float64.

    dist: "uniform" -> U[0,1) entries (Section IV-A); "exponential" -> Exp(1).
    """
    dims = tuple(int(n) for n in dims)
    ranks = tuple(int(r) for r in ranks)
    if len(ranks) != len(dims) + 1 or ranks[0] != 1 or ranks[-1] != 1:
        raise ValueError("ranks must have d+1 entries with r_0 = r_d = 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    cores = []
    for k, n in enumerate(dims):
        shape = (ranks[k], n, ranks[k + 1])
        if dist == "uniform":
            g = rng.random(shape)
        elif dist == "exponential":
            g = rng.standard_exponential(shape)
        else:
            raise ValueError(f"unknown core distribution {dist!r}")
        cores.append(g)
    return cores


def _left_matrix(cores):
    """Cores G_1..G_s multiplied into a (n_1...n_s) x r_s matrix (data recipe)."""
    g = cores[0]
    L = g.reshape(g.shape[1], g.shape[2])
    for g in cores[1:]:
        r0, n, r1 = g.shape
        L = (L @ g.reshape(r0, n * r1)).reshape(-1, r1)
    return L


def _right_matrix(cores):
    """Cores G_{s+1}..G_d multiplied into an r_s x (n_{s+1}...n_d) matrix."""
    g = cores[-1]
    R = g.reshape(g.shape[0], g.shape[1] * g.shape[2])
    for g in reversed(cores[:-1]):
        r0, n, r1 = g.shape
        R = (g.reshape(r0 * n, r1) @ R).reshape(r0, -1)
    return R


def _split_point(dims):
    total = math.prod(dims)
    best, best_s = None, 1
    for s in range(1, len(dims)):
        left = math.prod(dims[:s])
        score = abs(math.log(left) - 0.5 * math.log(total))
        if best is None or score < best:
            best, best_s = score, s
    return best_s


def tt_tensor(dims, ranks, dist="uniform", noise=0.01, seed=0, out=None, threads=None,
              return_cores=False):
    """Dense non-negative FP32 tensor = product of random TT cores + |Gaussian| noise.

    The clean tensor is the product of the cores (Section IV-A); the noise is
    |N(0, sigma^2)| with sigma = noise * mean(clean tensor), added entrywise,
    and the sum is rounded once to FP32.  `out` may be a preallocated float32
    array (e.g. a pinned host buffer) of prod(dims) entries.
    """
    dims = tuple(int(n) for n in dims)
    cores = tt_cores(dims, ranks, dist, seed)
    s = _split_point(dims)
    L = _left_matrix(cores[:s])          # rows x r_s
    R = _right_matrix(cores[s:])         # r_s x cols
    rows, cols = L.shape[0], R.shape[1]
    total = rows * cols
    mean = float(L.sum(axis=0) @ R.sum(axis=1)) / total
    sigma = noise * mean
    if out is None:
        out = np.empty(total, dtype=np.float32)
    flat = out.reshape(-1)
    if flat.size != total or flat.dtype != np.float32:
        raise ValueError("out must be a float32 array of prod(dims) entries")
    mat = flat.reshape(rows, cols)
    rows_per_block = max(1, min(rows, (1 << 22) // max(cols, 1)))
    nblocks = (rows + rows_per_block - 1) // rows_per_block
    child = np.random.SeedSequence([seed, 0x7E11]).spawn(nblocks)

    def work(b):
        r0 = b * rows_per_block
        r1 = min(rows, r0 + rows_per_block)
        blk = L[r0:r1] @ R
        if sigma > 0.0:
            rng = np.random.Generator(np.random.PCG64(child[b]))
            blk += np.abs(rng.standard_normal(blk.shape)) * sigma
        mat[r0:r1] = blk.astype(np.float32)

    nthreads = threads or min(32, os.cpu_count() or 1)
    if nblocks == 1 or nthreads == 1:
        for b in range(nblocks):
            work(b)
    else:
        with ThreadPoolExecutor(max_workers=nthreads) as ex:
            list(ex.map(work, range(nblocks)))
    A = flat.reshape(dims)
    info = dict(mean=mean, sigma=sigma, split=s)
    if return_cores:
        return A, info, cores
    return A, info


def uniform_matrix(shape, seed):
    """U[0,1) FP32 matrix (multiples of 2^-24, exact in FP32 and FP64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random(shape, dtype=np.float32)


def stage_shapes(dims, ranks):
    """(m, n, r) of every unfolding X_k = (r_{k-1} n_k) x prod_{j>k} n_j (Algorithm 2)."""
    d = len(dims)
    out = []
    for k in range(d - 1):
        m = ranks[k] * dims[k]
        n = math.prod(dims[k + 1:])
        out.append((m, n, ranks[k + 1]))
    return out


def _clamp_ranks(dims, ranks):
    """Clamp r_k to min(r_{k-1} n_k, prod_{j>k} n_j) left to right (N = min(m, n))."""
    ranks = list(ranks)
    d = len(dims)
    for k in range(1, d):
        m = ranks[k - 1] * dims[k - 1]
        n = math.prod(dims[k:])
        ranks[k] = max(1, min(ranks[k], m, n))
    ranks[d] = 1
    return tuple(ranks)


def batched_instances(count=512, seed=4, d_range=(3, 6), n_range=(8, 24), r_range=(2, 12)):
    """Shapes of the batched workload: d ~ U{3..6}, n_k ~ U{8..24}, r_k ~ U{2..12} clamped."""
    rng = np.random.Generator(np.random.PCG64(seed))
    inst = []
    for i in range(count):
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        dims = tuple(int(x) for x in rng.integers(n_range[0], n_range[1] + 1, size=d))
        inner = [int(x) for x in rng.integers(r_range[0], r_range[1] + 1, size=d - 1)]
        ranks = _clamp_ranks(dims, (1, *inner, 1))
        inst.append(dict(dims=dims, ranks=ranks, data_seed=int(seed) * 100003 + i))
    return inst


def serving_requests(count=1000, seed=5, d_range=(4, 7), size_range=(1e4, 1e8),
                     r_range=(4, 32), rate=1.0):
    """Poisson stream of nTT requests: d ~ U{4..7}, size ~ logU[1e4, 1e8],
    n_k = max(2, round(S^(1/d) 2^u)), u ~ U[-1/2, 1/2]; r_k ~ U{4..32} clamped;
    dtype FP32 or BF16 with probability 1/2; exponential inter-arrival times."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    t = 0.0
    for i in range(count):
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        S = math.exp(rng.uniform(math.log(size_range[0]), math.log(size_range[1])))
        u = rng.uniform(-0.5, 0.5, size=d)
        dims = tuple(max(2, int(round(S ** (1.0 / d) * 2.0 ** uk))) for uk in u)
        inner = [int(x) for x in rng.integers(r_range[0], r_range[1] + 1, size=d - 1)]
        ranks = _clamp_ranks(dims, (1, *inner, 1))
        dtype = "bf16" if rng.random() < 0.5 else "f32"
        t += rng.exponential(1.0 / rate)
        reqs.append(dict(dims=dims, ranks=ranks, x_dtype=dtype, arrival=t,
                         data_seed=int(seed) * 1000003 + i))
    return reqs

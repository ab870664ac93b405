"""FP64 CPU oracle for the non-negative tensor-train (nTT) hot path.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline / reference legs; the CUDA product path never imports,
links or calls anything here, and nothing here imports the CUDA path.

Plain, slow, obviously-correct numpy in float64.  Every function cites the part
of the paper it restates:

* Eq. (2)  tensor-train element formula            -> tt_entry, tt_full
* Eq. (3)  relative reconstruction error           -> rel_error
* Eq. (4)  compression ratio                       -> compression_ratio
* Algorithm 2 (distnTT) with fixed TT ranks        -> ntt_decompose
* Algorithm 1 (distReshape) as a C-order reshape   -> unfold
* Multiplicative-update NMF (Lee-Seung), which the paper times against BCD in
  Section IV (strong scaling, Fig. 7c); update order H then W, epsilon added to
  both denominators                                -> mu_update_H, mu_update_W, nmf_mu
* objective 1/2 ||X - WH||_F^2 (Algorithm 3's objective)   -> objective
* optional relative-change stopping test on that objective (tol = 0: the
  fixed iteration count of Algorithm 3's loop)     -> stop_reached
* counter-based SplitMix64 initialisation (the paper only says "rand") -> uniform01
* precision form (not in the paper, whose experiments are FP32: each unfolding
  rounded to bfloat16, the MU iterations on it, then refinement iterations on
  the unrounded unfolding)                          -> bf16_round, ntt_decompose(x_precision=)
* Algorithm 2's rank rule: r_l = the smallest k with
  sqrt(sigma_{k+1}^2 + ... + sigma_N^2) / sqrt(sigma_1^2 + ... + sigma_N^2) <= eps,
  sigma_i the singular values of X_l, N = min(m, n)
                                                   -> singular_values, select_rank,
                                                      ntt_decompose(ranks=None, eps_rank=)
* Algorithm 3 (distBCDnmf): block coordinate descent with prox-linear
  (projected gradient) block updates, extrapolation and the restart test,
  read through the method it cites (Xu & Yin 2013)  -> bcd_nmf, ntt_decompose(solver="bcd")

Readings where the paper is silent or garbled (the list is repeated in the
design notes):
* initial factors are plain U[0,1) (Algorithm 3's normalised init is for BCD);
* after each stage every column of W is divided by its L1 norm and the norm is
  folded into the matching row of H (the product W H is unchanged); a zero
  column is left as it is;
* the unfolding X_l is (r_{l-1} n_l) x prod_{j>l} n_j (Algorithm 2's comment on
  S is inconsistent; this is the shape its reshape produces);
* best restart = lowest final objective, ties to the lowest restart index;
* rank rule: k >= 1 (a rank-0 factor is no NMF); an all-zero X gets rank 1;
  an optional cap min(k, rank_cap) is this library's (the built kernels go to
  rank 32), not the paper's;
* Algorithm 3 (its listing is garbled in places) as APG-BCD: the W step is
  max(0, W_m - (W_m HH^T - XH^T) / ||HH^T||_2) (the printed line drops the
  gradient), the H step max(0, H_m - (W^TW H_m - W^TX) / ||W^TW||_2) (the
  printed square root is read as the same spectral norm), the initial
  objective is 1/2 ||X||_F^2 (printed without the square); an iteration whose
  objective is >= the last accepted one is rejected and the next one starts
  from the last accepted iterate without extrapolation (the "correction");
  otherwise t <- (1 + sqrt(1 + 4 t^2)) / 2, w = (t_old - 1) / t and each block
  is extrapolated by min(w, delta sqrt(L_prev / L)) with L its Lipschitz
  constant of this iteration and L_prev that of the previous accepted one.
  The listing's in-loop W /= ||W||_1 is not applied inside the loop (it would
  rescale W between the two block steps of one iteration without rescaling
  H); the column-L1 normalisation happens once per stage in the hand-off.

Parity pins for every function live in tests/test_oracle_pins.py.  No function
here is "parity unpinned".
"""

from __future__ import annotations

import math

import numpy as np

EPS_MU = 1e-12

# --------------------------------------------------------------------------
# Counter-based SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
# number generators", OOPSLA 2014).  Generator state advances by the golden
# gamma; each output is the state passed through the 64-bit finaliser.  The
# i-th output (0-based) of a generator seeded with s is mix64(s + (i+1)*gamma).
# --------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_outputs(seed, index):
    """Outputs number `index` (array, 0-based) of SplitMix64 seeded with `seed`."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(seed) + (idx + np.uint64(1)) * _GAMMA)


def stream_key(seed, stage, restart, matrix):
    """Key of the random stream for (stage, restart, matrix); matrix 0 = W, 1 = H.

    key = output number (stage * 2^20 + restart * 2 + matrix) of SplitMix64(seed).
    """
    stream = (int(stage) << 20) + (int(restart) << 1) + int(matrix)
    return int(splitmix64_outputs(int(seed), stream))


def uniform01(key, index):
    """U[0,1) values (x >> 40) * 2^-24 of SplitMix64(key) outputs at `index`.

    24-bit values: exact in FP32 and FP64.
    """
    x = splitmix64_outputs(key, index) >> np.uint64(40)
    return x.astype(np.float64) * (1.0 / 16777216.0)


def init_factors(m, n, r, seed, stage, restart=0):
    """W0 (m x r) and H0 (r x n), row-major element order, from the counter RNG."""
    kw = stream_key(seed, stage, restart, 0)
    kh = stream_key(seed, stage, restart, 1)
    W0 = uniform01(kw, np.arange(m * r, dtype=np.uint64)).reshape(m, r)
    H0 = uniform01(kh, np.arange(r * n, dtype=np.uint64)).reshape(r, n)
    return W0, H0


def init_columns_H(n, r, seed, stage, cols, restart=0):
    """Columns `cols` of H0 (r x len(cols)) without forming all of H0."""
    kh = stream_key(seed, stage, restart, 1)
    cols = np.asarray(cols, dtype=np.uint64)
    idx = np.arange(r, dtype=np.uint64)[:, None] * np.uint64(n) + cols[None, :]
    return uniform01(kh, idx)


# --------------------------------------------------------------------------
# Multiplicative-update NMF.
# --------------------------------------------------------------------------

def mu_update_H(X, W, H, eps=EPS_MU):
    """H <- max(0, H * (W^T X) / (W^T W H + eps))."""
    num = W.T @ X
    den = (W.T @ W) @ H + eps
    return np.maximum(0.0, H * num / den)


def mu_update_W(X, W, H, eps=EPS_MU):
    """W <- max(0, W * (X H^T) / (W (H H^T) + eps))."""
    num = X @ H.T
    den = W @ (H @ H.T) + eps
    return np.maximum(0.0, W * num / den)


def objective(X, W, H):
    """1/2 ||X - W H||_F^2 computed directly (no expanded Gram form)."""
    R = X - W @ H
    return 0.5 * float(np.sum(R * R))


def stop_reached(trace, u, tol, check_every):
    """Relative-change stopping test on the objective trace (the objective
    1/2 ||X - WH||^2 that Algorithm 3 tracks; the paper iterates to a maximum
    count, so the test is optional and tol = 0 keeps the fixed count).  After
    iteration u (1-based), with u a multiple of K = check_every and u >= 2K,
    stop when f_{u-K} - f_u <= tol |f_{u-K}|, where f_v = trace[v - 1]."""
    K = int(check_every)
    if tol <= 0.0 or K <= 0 or u % K != 0 or u < 2 * K:
        return False
    f0, f1 = trace[u - K - 1], trace[u - 1]
    return f0 - f1 <= tol * abs(f0)


def nmf_mu(X, W0, H0, iters, eps=EPS_MU, record=True, tol=0.0, check_every=10):
    """Run up to `iters` full multiplicative-update iterations, H first then W
    (fewer when tol > 0 and stop_reached says so; that needs record=True).

    Returns (W, H, trace) where trace[t] = 1/2 ||X - W_{t+1} H_{t+1}||^2.
    """
    X = np.asarray(X, dtype=np.float64)
    W = np.array(W0, dtype=np.float64)
    H = np.array(H0, dtype=np.float64)
    trace = []
    for u in range(1, int(iters) + 1):
        H = mu_update_H(X, W, H, eps)
        W = mu_update_W(X, W, H, eps)
        if record or tol > 0.0:
            trace.append(objective(X, W, H))
        if stop_reached(trace, u, tol, check_every):
            break
    return W, H, np.array(trace)


def handoff_normalize(W, H):
    """Divide each column of W by its L1 norm and multiply the matching row of H by it."""
    W = np.array(W, dtype=np.float64)
    H = np.array(H, dtype=np.float64)
    s = W.sum(axis=0)
    for j in range(W.shape[1]):
        if s[j] > 0.0:
            W[:, j] /= s[j]
            H[j, :] *= s[j]
    return W, H


# --------------------------------------------------------------------------
# Algorithm 2's rank rule.
# --------------------------------------------------------------------------

def singular_values(X):
    """The min(m, n) singular values of X in non-increasing order (FP64 SVD,
    the distSVD step of Algorithm 2 on one node)."""
    return np.linalg.svd(np.asarray(X, dtype=np.float64), compute_uv=False)


def select_rank(sigma, eps_rank, rank_cap=None):
    """Algorithm 2: the smallest k (1 <= k <= N) whose tail ratio
    sqrt(sum_{i>k} sigma_i^2) / sqrt(sum_i sigma_i^2) is <= eps_rank; N =
    len(sigma).  All-zero sigma gives 1.  rank_cap (optional) caps the result."""
    sig2 = np.asarray(sigma, dtype=np.float64) ** 2
    N = len(sig2)
    total = float(np.sum(sig2))
    k_sel = N
    if total <= 0.0:
        k_sel = 1
    else:
        for k in range(1, N + 1):
            tail = float(np.sum(sig2[k:]))
            if math.sqrt(tail) / math.sqrt(total) <= eps_rank:
                k_sel = k
                break
    if rank_cap is not None:
        k_sel = min(k_sel, int(rank_cap))
    return max(1, k_sel)


# --------------------------------------------------------------------------
# Algorithm 3: BCD NMF with extrapolation and restarts.
# --------------------------------------------------------------------------
BCD_DELTA = 0.9999


def spectral_norm_sym(M):
    """||M||_2 of a symmetric positive semi-definite matrix (its largest eigenvalue)."""
    M = np.asarray(M, dtype=np.float64)
    if M.size == 0:
        return 0.0
    return float(np.max(np.linalg.eigvalsh(M)))


def bcd_nmf(X, W0, H0, iters, delta=BCD_DELTA, record=True, info=None):
    """Algorithm 3 on one node (see the readings in the module docstring).

    Initial factors W0, H0 are scaled to Frobenius norm sqrt(||X||_F) each
    (Algorithm 3's normalisation).  Iteration l: W step from the extrapolated
    W_m with the Gram terms of the current H, H step from the extrapolated H_m
    with the new W, objective f = 1/2 ||X - W H||^2; f >= the last accepted
    objective rejects the iteration (the factors return to the last accepted
    ones and the next steps start there without extrapolation), otherwise the
    iterate is accepted and both blocks are extrapolated.

    Returns (W, H, trace, accepted): the last accepted factors, trace[l] = the
    last accepted objective after iteration l+1, accepted[l] = whether
    iteration l+1 was accepted.  info (optional dict) receives "f": the
    objective of every iteration's new iterate, accepted or not.
    """
    X = np.asarray(X, dtype=np.float64)
    nx = float(np.linalg.norm(X))
    W = np.array(W0, dtype=np.float64)
    H = np.array(H0, dtype=np.float64)
    nw, nh = float(np.linalg.norm(W)), float(np.linalg.norm(H))
    if nw > 0.0:
        W = W / nw * math.sqrt(nx)
    if nh > 0.0:
        H = H / nh * math.sqrt(nx)
    W_acc, H_acc = W, H            # last accepted iterate
    W_m, H_m = W, H                # extrapolated points the next steps start from
    HHt, XHt = H_acc @ H_acc.T, X @ H_acc.T
    t = 1.0
    obj = 0.5 * nx * nx
    Lw_prev = Lh_prev = None
    trace, accepted = [], []
    for _ in range(int(iters)):
        Lw = spectral_norm_sym(HHt)
        W_new = np.maximum(0.0, W_m - (W_m @ HHt - XHt) / Lw) if Lw > 0.0 else W_m.copy()
        WtW = W_new.T @ W_new
        Lh = spectral_norm_sym(WtW)
        H_new = np.maximum(0.0, H_m - (WtW @ H_m - W_new.T @ X) / Lh) if Lh > 0.0 else H_m.copy()
        f = objective(X, W_new, H_new)
        if info is not None:
            info.setdefault("f", []).append(f)
        if f >= obj:
            # correction: back to the last accepted iterate, no extrapolation
            W_m, H_m = W_acc, H_acc
            HHt, XHt = H_acc @ H_acc.T, X @ H_acc.T
            accepted.append(False)
        else:
            t_new = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
            w = (t - 1.0) / t_new
            lw_prev = Lw if Lw_prev is None else Lw_prev
            lh_prev = Lh if Lh_prev is None else Lh_prev
            w_w = min(w, delta * math.sqrt(lw_prev / Lw)) if Lw > 0.0 else 0.0
            w_h = min(w, delta * math.sqrt(lh_prev / Lh)) if Lh > 0.0 else 0.0
            W_m = W_new + w_w * (W_new - W_acc)
            H_m = H_new + w_h * (H_new - H_acc)
            W_acc, H_acc = W_new, H_new
            HHt, XHt = H_acc @ H_acc.T, X @ H_acc.T
            t, obj = t_new, f
            Lw_prev, Lh_prev = Lw, Lh
            accepted.append(True)
        if record:
            trace.append(obj)
    return W_acc, H_acc, np.array(trace), np.array(accepted, dtype=bool)


# --------------------------------------------------------------------------
# Algorithm 2.
# --------------------------------------------------------------------------

# --------------------------------------------------------------------------
# Precision form.
# --------------------------------------------------------------------------

def bf16_round(x):
    """Round-to-nearest, ties-to-even of real values to bfloat16 (8 significand
    bits including the leading one, FP32's exponent range), returned as float64.
    Defined from the format: with e = floor(log2 |x|) the representable values
    near x are the multiples of 2^(e-7); x is rounded to the nearest multiple,
    halfway cases to the even multiple.  Zero stays zero; inputs are finite and
    inside the normal range."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x != 0.0
    ax = np.abs(x[nz])
    e = np.floor(np.log2(ax))
    # log2 can land one below/above at exact powers of two: correct e so that 2^e <= ax < 2^(e+1)
    e = np.where(np.exp2(e) > ax, e - 1, e)
    e = np.where(np.exp2(e + 1) <= ax, e + 1, e)
    ulp = np.exp2(e - 7)
    out[nz] = np.sign(x[nz]) * np.rint(ax / ulp) * ulp      # np.rint: halfway to even
    return out


def unfold(T, m):
    """Algorithm 1 on one device: the C-order reshape of T into m x (size/m)."""
    T = np.asarray(T)
    return T.reshape(m, T.size // m)


def ntt_decompose(A, ranks, iters, eps=EPS_MU, seed=0, restarts=1, record=True, x_precision="f32",
                  refine=0, tol=0.0, check_every=10, eps_rank=None, rank_cap=None, solver="mu", info=None):
    """Non-negative tensor train of A (Algorithm 2).

    Stage l (0-based s = l-1): X = reshape(current, r_{l-1} n_l, rest); NMF of
    rank r_l by multiplicative updates from the counter-RNG init; W becomes core
    G_l (r_{l-1} x n_l x r_l) after the column-L1 hand-off normalisation and H
    becomes the next `current`.  The last core is the final H.
    x_precision="bf16": the stage's `iters` iterations run on bf16_round(X),
    then `refine` more on X itself (the precision form); the objective that
    picks the restart is on X.
    tol > 0: each stage's main loop stops early under stop_reached (the
    refinement iterations always run).
    ranks=None: every r_l comes from Algorithm 2's rule on X_l (select_rank
    with eps_rank, optional rank_cap), chosen before the stage's NMF.
    solver="bcd": each NMF runs bcd_nmf (Algorithm 3) from the same counter-RNG
    init instead of the multiplicative updates (FP32 form, no restarts).
    Returns (cores, traces), traces[s] = objective trace of the kept restart
    (with record=False only the final objective of each stage).  The ranks
    used are the cores' shapes.  info (optional dict) receives "sigma": the
    singular values of every unfolding the rank rule saw.
    """
    A = np.asarray(A)
    dims = A.shape
    d = len(dims)
    if ranks is None:
        if eps_rank is None:
            raise ValueError("ranks=None needs eps_rank")
        ranks = [1] * (d + 1)
    else:
        ranks = tuple(int(r) for r in ranks)
        if len(ranks) != d + 1 or ranks[0] != 1 or ranks[-1] != 1:
            raise ValueError("ranks must have d+1 entries with r_0 = r_d = 1")
    ranks = list(ranks)
    select = eps_rank is not None
    cur = A.astype(np.float64)
    cores, traces = [], []
    for s in range(d - 1):
        m = ranks[s] * dims[s]
        n = math.prod(dims[s + 1:])
        if select:
            sig = singular_values(unfold(cur, m))
            if info is not None:
                info.setdefault("sigma", []).append(sig)
            ranks[s + 1] = select_rank(sig, eps_rank, rank_cap)
        r = ranks[s + 1]
        if r > min(m, n):
            raise ValueError(f"rank r_{s+1}={r} exceeds min(m, n)=min({m},{n})")
        X = unfold(cur, m)
        best = None
        Xi = bf16_round(X) if x_precision == "bf16" else X
        for rs in range(restarts):
            W0, H0 = init_factors(m, n, r, seed, s, rs)
            if solver == "bcd":
                W, H, tr, _ = bcd_nmf(Xi, W0, H0, iters, record=record)
            else:
                W, H, tr = nmf_mu(Xi, W0, H0, iters, eps, record=record, tol=tol, check_every=check_every)
            if refine:
                W, H, tr2 = nmf_mu(X, W, H, refine, eps, record=record)
                tr = np.concatenate([tr, tr2])
            final = objective(X, W, H)          # on the unrounded unfolding
            if not record:
                tr = np.array([final])
            if best is None or final < best[3]:
                best = (W, H, tr, final)
        W, H, tr, _ = best
        W, H = handoff_normalize(W, H)
        cores.append(W.reshape(ranks[s], dims[s], r))
        traces.append(tr)
        cur = H
    cores.append(cur.reshape(ranks[d - 1], dims[d - 1], 1))
    return cores, traces


# --------------------------------------------------------------------------
# Eq. (2)-(4).
# --------------------------------------------------------------------------

def tt_entry(cores, idx):
    """Eq. (2): A[i_1..i_d] = G1[:, i_1, :] G2[:, i_2, :] ... Gd[:, i_d, :] (a 1x1 product)."""
    v = np.ones((1, 1))
    for g, i in zip(cores, idx):
        v = v @ np.asarray(g, dtype=np.float64)[:, int(i), :]
    return float(v[0, 0])


def tt_full(cores):
    """Eq. (2) for every index: contract the cores left to right into the full tensor."""
    dims = [g.shape[1] for g in cores]
    acc = np.asarray(cores[0], dtype=np.float64).reshape(dims[0], cores[0].shape[2])
    for g in cores[1:]:
        g = np.asarray(g, dtype=np.float64)
        acc = np.tensordot(acc, g, axes=([acc.ndim - 1], [0]))
    return acc.reshape(dims)


def rel_error(A, cores):
    """Eq. (3): ||A - A~||_F / ||A||_F with A~ the tensor of `cores`."""
    A = np.asarray(A, dtype=np.float64)
    At = tt_full(cores)
    return float(np.linalg.norm((A - At).ravel()) / np.linalg.norm(A.ravel()))


def compression_ratio(dims, ranks):
    """Eq. (4): prod(n_i) / sum_i n_i r_{i-1} r_i."""
    return math.prod(dims) / sum(n * ranks[i] * ranks[i + 1] for i, n in enumerate(dims))

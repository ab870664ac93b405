"""Host-side model of the warp-level MMA pass's data movement (no GPU).

The pass (csrc/mu_pass_tcw.cu) keeps a 64-column stage of the interleaved
split X (line L = 2 i + term, 128 bytes, 16-byte chunks XOR L mod 8) and of H
(line 2 k + half), loads MMA fragments with ldmatrix (plain and transposed)
and runs m16n8k16 BF16 MMAs.  These tests restate, in numpy, the PTX fragment
layouts of ldmatrix .x4 and of mma.m16n8k16 (A row-major, B column-major,
FP32 C/D) and the kernel's per-lane addressing, and check that one stage
reproduces Y = W^T X, the H update, P = X H_new^T and Q = H_new H_new^T,
and that every ldmatrix phase touches eight distinct 16-byte bank groups.
"""

import numpy as np
import pytest

SEG = 64


def bf16(a):
    """Round float32 values to BF16 (nearest, ties to even), returned as float32."""
    a = np.asarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def stage_x(X1, X2):
    """The X part of a stage as a dict byte offset -> BF16 value (lines 2 i + term)."""
    mp = X1.shape[0]
    mem = {}
    for i in range(mp):
        for term, T in enumerate((X1, X2)):
            L = 2 * i + term
            for c in range(SEG):
                off = L * 128 + (((c >> 3) ^ (L & 7)) << 4) + (c & 7) * 2
                mem[off] = T[i, c]
    return mem


def h_off(rank, col):
    line = rank * 2 + (col >> 5)
    w = col & 31
    return line * 128 + (((w >> 2) ^ (line & 7)) << 4) + (w & 3) * 4


def ldmatrix_x4(mem, addrs, trans):
    """PTX ldmatrix.m8n8.x4(.trans).b16: lane 8 j + i gives the address of row i
    of matrix j; returns regs[lane][j] = (lo, hi)."""
    mats = []
    for j in range(4):
        rows = [[mem[addrs[8 * j + i] + 2 * c] for c in range(8)] for i in range(8)]
        mats.append(np.array(rows, dtype=np.float32))
    regs = []
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        rr = []
        for j in range(4):
            M = mats[j].T if trans else mats[j]
            rr.append((M[g, 2 * t], M[g, 2 * t + 1]))
        regs.append(rr)
    return regs


def mma(a_regs, b_regs, acc):
    """mma.m16n8k16.row.col: rebuild A (16 x 16), B (16 x 8) from the per-lane
    fragments, D = A B + C, scattered back to acc[lane][4]."""
    A = np.zeros((16, 16))
    B = np.zeros((16, 8))
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        a = a_regs[lane]
        A[g, 2 * t:2 * t + 2] = a[0]
        A[g + 8, 2 * t:2 * t + 2] = a[1]
        A[g, 2 * t + 8:2 * t + 10] = a[2]
        A[g + 8, 2 * t + 8:2 * t + 10] = a[3]
        b = b_regs[lane]
        B[2 * t:2 * t + 2, g] = b[0]
        B[2 * t + 8:2 * t + 10, g] = b[1]
    D = A @ B
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        acc[lane] += np.array([D[g, 2 * t], D[g, 2 * t + 1], D[g + 8, 2 * t], D[g + 8, 2 * t + 1]])


def split3(v):
    t1 = bf16(v)
    r1 = np.float32(v) - t1
    t2 = bf16(r1)
    t3 = bf16(np.float32(r1) - t2)
    return t1, t2, t3


def check_phases(addrs):
    """Each ldmatrix matrix (8 lanes, 16 bytes each) must hit 8 distinct bank groups."""
    for j in range(4):
        groups = {(a % 128) // 16 for a in addrs[8 * j:8 * j + 8]}
        assert len(groups) == 8, addrs[8 * j:8 * j + 8]


@pytest.mark.parametrize("mp", [32, 16])
def test_stage_model_reproduces_the_products(mp):
    rng = np.random.default_rng(3 + mp)
    r = 8
    X = rng.random((mp, SEG)).astype(np.float32)
    W = rng.random((mp, r)).astype(np.float32)
    H = rng.random((r, SEG)).astype(np.float32)
    G = (W.astype(np.float64).T @ W).astype(np.float32)
    eps = 1e-12
    X1 = bf16(X)
    X2 = bf16(X - X1)
    xmem = stage_x(X1, X2)
    hmem = {h_off(k, c): H[k, c] for k in range(r) for c in range(SEG)}
    W1 = bf16(W)
    W2 = bf16(W - W1)
    ks_n = 2 * mp // 16
    P = np.zeros((32, 4 * (2 * mp // 16)))      # per lane: accP[mt][4] flattened
    accP = [np.zeros((32, 4)) for _ in range(2 * mp // 16)]
    accQa = np.zeros((32, 4))
    accQb = np.zeros((32, 4))
    Hn_all = np.zeros((r, SEG))
    for ck in range(SEG // 16):
        c0 = ck * 16
        y1 = np.zeros((32, 4))
        y2 = np.zeros((32, 4))
        for ks in range(ks_n):
            addrs = []
            for lane in range(32):
                lj, li = lane >> 3, lane & 7
                line = 16 * ks + li + 8 * (lj >> 1)
                chunk = (c0 >> 3) + (lj & 1)
                addrs.append(line * 128 + ((chunk ^ (line & 7)) << 4))
            check_phases(addrs)
            a = ldmatrix_x4(xmem, addrs, trans=True)
            for Wt, y in ((W1, y1), (W2, y2)):
                b = []
                for lane in range(32):
                    g, t = lane >> 2, lane & 3
                    vals = []
                    for h in range(2):
                        row = 8 * ks + 4 * h + t
                        w = Wt[row, g] if row < mp else 0.0
                        vals.append((w, w))
                    b.append(vals)
                mma(a, b, y)
        Y = (W.astype(np.float64).T @ (X1.astype(np.float64) + X2))[:, c0:c0 + 16]
        for lane in range(32):
            g, t = lane >> 2, lane & 3
            yv = y1[lane] + y2[lane]
            # rows of the D fragment: column c0 + g / c0 + g + 8, ranks 2t, 2t + 1
            assert np.allclose(yv, [Y[2 * t, g], Y[2 * t + 1, g], Y[2 * t, g + 8], Y[2 * t + 1, g + 8]],
                               rtol=2e-5)
            for q, (col, k) in enumerate([(c0 + g, 2 * t), (c0 + g, 2 * t + 1), (c0 + g + 8, 2 * t),
                                          (c0 + g + 8, 2 * t + 1)]):
                gh = sum(G[k, i] * hmem[h_off(i, col)] for i in range(8))
                Hn_all[k, col] = max(0.0, hmem[h_off(k, col)] * yv[q] / (gh + eps))
        for lane in range(32):
            g, t = lane >> 2, lane & 3
            for q, (col, k) in enumerate([(c0 + g, 2 * t), (c0 + g, 2 * t + 1), (c0 + g + 8, 2 * t),
                                          (c0 + g + 8, 2 * t + 1)]):
                hmem[h_off(k, col)] = Hn_all[k, col]
        # B fragments of H_new^T split in three terms
        hb = []
        for lane in range(32):
            g, t = lane >> 2, lane & 3
            v0 = np.array([hmem[h_off(g, c0 + 2 * t)], hmem[h_off(g, c0 + 2 * t + 1)]], dtype=np.float32)
            v1 = np.array([hmem[h_off(g, c0 + 2 * t + 8)], hmem[h_off(g, c0 + 2 * t + 9)]], dtype=np.float32)
            hb.append((split3(v0), split3(v1)))
        for mt in range(2 * mp // 16):
            addrs = []
            for lane in range(32):
                lj, li = lane >> 3, lane & 7
                line = 16 * mt + li + 8 * (lj & 1)
                chunk = (c0 >> 3) + (lj >> 1)
                addrs.append(line * 128 + ((chunk ^ (line & 7)) << 4))
            check_phases(addrs)
            a = ldmatrix_x4(xmem, addrs, trans=False)
            for h in range(3):
                b = [[tuple(hb[lane][0][h]), tuple(hb[lane][1][h])] for lane in range(32)]
                mma(a, b, accP[mt])
        a12 = [[tuple(hb[l][0][0]), tuple(hb[l][0][1]), tuple(hb[l][1][0]), tuple(hb[l][1][1])] for l in range(32)]
        a13 = [[tuple(hb[l][0][0]), tuple(hb[l][0][2]), tuple(hb[l][1][0]), tuple(hb[l][1][2])] for l in range(32)]
        mma(a12, [[tuple(hb[l][0][0]), tuple(hb[l][1][0])] for l in range(32)], accQa)
        mma(a12, [[tuple(hb[l][0][1]), tuple(hb[l][1][1])] for l in range(32)], accQa)
        mma(a13, [[tuple(hb[l][0][2]), tuple(hb[l][1][2])] for l in range(32)], accQb)
    # the end-of-kernel assembly (one warp)
    Pw = np.zeros((mp, 8))
    Qw = np.zeros((8, 8))
    Qt = np.zeros((8, 8))
    for mt in range(2 * mp // 16):
        for lane in range(32):
            g, t = lane >> 2, lane & 3
            for q in range(4):
                v = accP[mt][lane][q] + accP[mt][lane ^ 4][q]
                if g % 2 == 0:
                    Pw[(16 * mt + g + 8 * (q >> 1)) >> 1, 2 * t + (q & 1)] = v
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        for q in range(2):
            Qw[g, 2 * t + q] = accQa[lane][q] + accQa[lane][2 + q] + accQb[lane][q]
            Qt[g, 2 * t + q] = accQb[lane][q]
    Q = Qw + Qt.T
    # reference: the H update of the oracle's form on X1 + X2
    Xs = X1.astype(np.float64) + X2
    Hn_ref = np.maximum(0.0, H * (W.astype(np.float64).T @ Xs) / (G.astype(np.float64) @ H + eps))
    assert np.allclose(Hn_all, Hn_ref, rtol=1e-4)
    assert np.allclose(Pw, Xs @ Hn_all.T, rtol=1e-5)
    assert np.allclose(Q, Hn_all @ Hn_all.T, rtol=1e-6)


def test_split_layout_is_interleaved_by_segment():
    """Row i of the split matrix: [X1 seg 0 | X2 seg 0 | X1 seg 1 | ...], the
    index arithmetic of split_x12_kernel (8 columns per thread)."""
    m, n = 3, 256
    rng = np.random.default_rng(5)
    X = rng.random((m, n)).astype(np.float32)
    out = np.zeros((m, 2 * n), dtype=np.float32)
    for q in range(m * (n // 8)):
        row, c8 = q // (n // 8), (q % (n // 8)) * 8
        v = X[row, c8:c8 + 8]
        t1 = bf16(v)
        t2 = bf16(v - t1)
        sg, c = c8 // SEG, c8 % SEG
        base = sg * 2 * SEG + c
        out[row, base:base + 8] = t1
        out[row, base + SEG:base + SEG + 8] = t2
    for sg in range(n // SEG):
        seg = X[:, sg * SEG:(sg + 1) * SEG]
        assert np.array_equal(out[:, sg * 2 * SEG:sg * 2 * SEG + SEG], bf16(seg))
        assert np.array_equal(out[:, sg * 2 * SEG + SEG:(sg + 1) * 2 * SEG], bf16(seg - bf16(seg)))


def test_precomputed_lane_offsets_match_the_layout():
    """The kernel's per-lane address parts: ldmatrix rows (a lane offset plus
    2048 per K step or line tile, chunk 2 ck ^ lane constant), H box reads
    (a compile-time part plus the lane's part for the 32-column half), and the
    H_new staging tile (word rank * 32 + (col ^ 8 pi(rank))), whose four stores
    and two 8-byte loads per lane each cover the 32 banks once."""
    def h_ct(i, c0, h):
        return (2 * i + (c0 >> 5)) * 128 + (((((c0 & 31) >> 2) + 2 * h) ^ ((2 * i) & 6)) << 4)

    def pi(k):
        return (k & 3) ^ (k >> 2)

    for ck in range(4):
        c0 = 16 * ck
        for lane in range(32):
            g, t, lj, li = lane >> 2, lane & 3, lane >> 3, lane & 7
            ly, lamy = (li + 8 * (lj >> 1)) * 128, li ^ (lj & 1)
            lp, lamp = (li + 8 * (lj & 1)) * 128, li ^ (lj >> 1)
            for x in range(4):
                line = 16 * x + li + 8 * (lj >> 1)
                chunk = (c0 >> 3) + (lj & 1)
                assert x * 2048 + ly + (((2 * ck) ^ lamy) << 4) == line * 128 + ((chunk ^ (line & 7)) << 4)
                line = 16 * x + li + 8 * (lj & 1)
                chunk = (c0 >> 3) + (lj >> 1)
                assert x * 2048 + lp + (((2 * ck) ^ lamp) << 4) == line * 128 + ((chunk ^ (line & 7)) << 4)
            hq = [((g >> 2) << 4) + (g & 3) * 4, (((g >> 2) ^ 1) << 4) + (g & 3) * 4]
            for i in range(8):
                for h in range(2):
                    assert h_ct(i, c0, h) + hq[c0 >> 5] == h_off(i, c0 + g + 8 * h)
    # staging tile
    for e in range(2):
        for h in range(2):
            words = [(2 * (l & 3) + e) * 32 + (((l >> 2) + 8 * h) ^ (8 * pi(2 * (l & 3) + e))) for l in range(32)]
            assert len({w % 32 for w in words}) == 32
            assert all(0 <= w < 256 for w in words)
    tile = {}
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        for e in range(2):
            for h in range(2):
                tile[(2 * t + e) * 32 + ((g + 8 * h) ^ (8 * pi(2 * t + e)))] = (2 * t + e, g + 8 * h)
    for h in range(2):
        for p0 in (0, 16):
            banks = []
            for lane in range(p0, p0 + 16):
                g, t = lane >> 2, lane & 3
                w = g * 32 + ((2 * t + 8 * h) ^ (8 * pi(g)))
                assert tile[w] == (g, 2 * t + 8 * h) and tile[w + 1] == (g, 2 * t + 8 * h + 1)
                banks += [w % 32, (w + 1) % 32]
            assert len(set(banks)) == 32


# ---------------------------------------------------------------------------
# The BF16-X form (mu_pass_tcwb.cu): 16 rows as X lines (row = line), rank 16
# in two n-tiles, G H on the MMAs from an H^T A fragment, Q = Qa + Qb + Qb^T.

def _h16_addr(t, g, c0, e, q, h):
    """The kernel's H box offset of (rank 2t + e + 8q, column c0 + g + 8h)."""
    hl = [4 * t * 128 + ((g >> 2) << 4) + (g & 3) * 4, 4 * t * 128 + 128 + (((g >> 2) ^ 1) << 4) + (g & 3) * 4]
    A = ((c0 & 31) >> 2) + 2 * h
    return hl[c0 >> 5] + (2 * e + 16 * q) * 128 + (((A ^ (2 * e)) ^ (4 * (t & 1))) << 4)


def test_bf16_form_stage_model_reproduces_the_products():
    rng = np.random.default_rng(9)
    m = r = 16
    X = bf16(rng.random((m, SEG)).astype(np.float32))          # exact BF16 operand
    W = rng.random((m, r)).astype(np.float32)
    H = rng.random((r, SEG)).astype(np.float32)
    G = (W.astype(np.float64).T @ W).astype(np.float32)
    eps = 1e-12
    xmem = {}
    for i in range(m):
        for c in range(SEG):
            xmem[i * 128 + (((c >> 3) ^ (i & 7)) << 4) + (c & 7) * 2] = X[i, c]
    hmem = {}
    for k in range(r):
        for c in range(SEG):
            hmem[h_off(k, c)] = H[k, c]
    # the kernel's H address formula equals the layout's
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        for ck in range(4):
            for e in range(2):
                for q in range(2):
                    for h in range(2):
                        assert _h16_addr(t, g, 16 * ck, e, q, h) == h_off(2 * t + e + 8 * q, 16 * ck + g + 8 * h)
    Wt3 = split3(W)
    Gt = split3(G)
    def pi(k):
        return (k & 7 & 3) ^ ((k & 7) >> 2)
    accP = [np.zeros((32, 4)) for _ in range(2)]
    Qa = [np.zeros((32, 4)) for _ in range(2)]
    Qb = [np.zeros((32, 4)) for _ in range(2)]
    Hn_all = np.zeros((r, SEG))
    for ck in range(4):
        c0 = 16 * ck
        # Y: one K step over the 16 rows
        addrs = []
        for lane in range(32):
            lj, li = lane >> 3, lane & 7
            ly, lamy = (li + 8 * (lj >> 1)) * 128, li ^ (lj & 1)
            addrs.append(ly + (((2 * ck) ^ lamy) << 4))
        check_phases(addrs)
        a = ldmatrix_x4(xmem, addrs, trans=True)
        y = [np.zeros((32, 4)) for _ in range(2)]
        for nt in range(2):
            for Wt in Wt3:
                b = []
                for lane in range(32):
                    g, t = lane >> 2, lane & 3
                    b.append([(Wt[2 * t, 8 * nt + g], Wt[2 * t + 1, 8 * nt + g]),
                              (Wt[2 * t + 8, 8 * nt + g], Wt[2 * t + 9, 8 * nt + g])])
                mma(a, b, y[nt])
        # G H from the H^T fragment (three terms) and G (three terms)
        hv = []
        for lane in range(32):
            g, t = lane >> 2, lane & 3
            v = {}
            for q in range(2):
                for h in range(2):
                    v[(q, h)] = np.array([hmem[_h16_addr(t, g, c0, 0, q, h)], hmem[_h16_addr(t, g, c0, 1, q, h)]],
                                         dtype=np.float32)
            hv.append(v)
        ht = [{key: split3(val) for key, val in hv[l].items()} for l in range(32)]
        def afr(term):
            return [[tuple(ht[l][(0, 0)][term]), tuple(ht[l][(0, 1)][term]), tuple(ht[l][(1, 0)][term]),
                     tuple(ht[l][(1, 1)][term])] for l in range(32)]
        gh = [np.zeros((32, 4)) for _ in range(2)]
        for nt in range(2):
            def bgf(term):
                return [[(Gt[term][2 * (l & 3), 8 * nt + (l >> 2)], Gt[term][2 * (l & 3) + 1, 8 * nt + (l >> 2)]),
                         (Gt[term][2 * (l & 3) + 8, 8 * nt + (l >> 2)], Gt[term][2 * (l & 3) + 9, 8 * nt + (l >> 2)])]
                        for l in range(32)]
            for ta, tb in ((0, 0), (0, 1), (1, 0), (0, 2), (2, 0), (1, 1)):
                mma(afr(ta), bgf(tb), gh[nt])
        Yref = W.astype(np.float64).T @ X.astype(np.float64)
        GHref = G.astype(np.float64) @ H.astype(np.float64)
        hn = [np.zeros((32, 4)) for _ in range(2)]
        for lane in range(32):
            g, t = lane >> 2, lane & 3
            for nt in range(2):
                for q in range(4):
                    col, k = c0 + g + 8 * (q >> 1), 8 * nt + 2 * t + (q & 1)
                    assert np.isclose(y[nt][lane][q], Yref[k, col], rtol=1e-6)
                    assert np.isclose(gh[nt][lane][q], GHref[k, col], rtol=1e-6)
                    h0 = hv[lane][(nt, q >> 1)][q & 1]
                    assert h0 == H[k, col]
                    hn[nt][lane][q] = max(0.0, h0 * y[nt][lane][q] / (gh[nt][lane][q] + eps))
                    Hn_all[k, col] = hn[nt][lane][q]
        # staging tile and the B fragments of H_new^T
        tile = {}
        for lane in range(32):
            g, t = lane >> 2, lane & 3
            for nt in range(2):
                for e in range(2):
                    k = 8 * nt + 2 * t + e
                    for h in range(2):
                        tile[k * 32 + ((g + 8 * h) ^ (8 * pi(k)))] = hn[nt][lane][2 * h + e]
        hb = []
        for lane in range(32):
            g, t = lane >> 2, lane & 3
            per = []
            for nt in range(2):
                k = 8 * nt + g
                w0 = k * 32 + ((2 * t) ^ (8 * pi(k)))
                w1 = k * 32 + ((2 * t + 8) ^ (8 * pi(k)))
                per.append((split3(np.array([tile[w0], tile[w0 + 1]], dtype=np.float32)),
                            split3(np.array([tile[w1], tile[w1 + 1]], dtype=np.float32))))
            hb.append(per)
        # P
        addrs = []
        for lane in range(32):
            lj, li = lane >> 3, lane & 7
            lp, lamp = (li + 8 * (lj & 1)) * 128, li ^ (lj >> 1)
            addrs.append(lp + (((2 * ck) ^ lamp) << 4))
        check_phases(addrs)
        a = ldmatrix_x4(xmem, addrs, trans=False)
        for nt in range(2):
            for term in range(3):
                mma(a, [[tuple(hb[l][nt][0][term]), tuple(hb[l][nt][1][term])] for l in range(32)], accP[nt])
        # Q
        def qa(term):
            return [[tuple(hb[l][0][0][term]), tuple(hb[l][1][0][term]), tuple(hb[l][0][1][term]),
                     tuple(hb[l][1][1][term])] for l in range(32)]
        for nt in range(2):
            def qb(term):
                return [[tuple(hb[l][nt][0][term]), tuple(hb[l][nt][1][term])] for l in range(32)]
            mma(qa(0), qb(0), Qa[nt])
            mma(qa(1), qb(1), Qa[nt])
            mma(qa(0), qb(1), Qb[nt])
            mma(qa(0), qb(2), Qb[nt])
    P = np.zeros((m, r))
    Qm = np.zeros((r, r))
    Qt = np.zeros((r, r))
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        for nt in range(2):
            for q in range(4):
                row, col = g + 8 * (q >> 1), 8 * nt + 2 * t + (q & 1)
                P[row, col] = accP[nt][lane][q]
                Qm[row, col] = Qa[nt][lane][q] + Qb[nt][lane][q]
                Qt[row, col] = Qb[nt][lane][q]
    Q = Qm + Qt.T
    Hn_ref = np.maximum(0.0, H * (W.astype(np.float64).T @ X) / (G.astype(np.float64) @ H + eps))
    assert np.allclose(Hn_all, Hn_ref, rtol=5e-5)
    assert np.allclose(P, X.astype(np.float64) @ Hn_all.T, rtol=1e-6)
    assert np.allclose(Q, Hn_all @ Hn_all.T, rtol=1e-6)


def test_bf16_form_staging_tile_is_conflict_free():
    """The 16-rank staging tile of the BF16-X form: the lane's eight stores
    (ranks 8 nt + 2t + e, columns g + 8h) and four 8-byte B-fragment loads
    (rank 8 nt + g, columns 2t + 8h, + 1) each cover the 32 banks once, and
    every (rank, column) of the 16 x 16 chunk has its own word."""
    def pi(k):
        return (k & 7 & 3) ^ ((k & 7) >> 2)

    seen = set()
    for nt in range(2):
        for e in range(2):
            for h in range(2):
                words = [(8 * nt + 2 * (l & 3) + e) * 32 + (((l >> 2) + 8 * h) ^ (8 * pi(8 * nt + 2 * (l & 3) + e)))
                         for l in range(32)]
                assert len({w % 32 for w in words}) == 32
                seen.update(words)
        for h in range(2):
            for p0 in (0, 16):
                banks = []
                for l in range(p0, p0 + 16):
                    g, t = l >> 2, l & 3
                    w = (8 * nt + g) * 32 + ((2 * t + 8 * h) ^ (8 * pi(8 * nt + g)))
                    banks += [w % 32, (w + 1) % 32]
                assert len(set(banks)) == 32
    assert len(seen) == 256 and max(seen) < 512

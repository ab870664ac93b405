"""Host-side checks of the narrow MU pass's index arithmetic (no GPU).

The narrow pass (csrc/mu_pass_narrow.cu) reads X and H boxes of 32 FP32
columns stored with the 128-byte swizzle (16-byte chunk index XOR row mod 8),
assigns lane = (row split sa = lane & 7, column group cq = lane >> 3), and
reduces Y over the eight row splits with shuffles in an XOR slot order
(slot i holds rank i ^ sa).  These tests restate that addressing and data
movement in Python and check:

* every shared-memory access of every (step, lane) lies inside its box;
* the lanes of one shared-memory phase (8 lanes for 16-byte loads, 16 for
  8-byte loads) touch distinct bank groups, or the same address;
* a lane-level model of the reduce-scatter, the H_new gather and the P, Q
  accumulation reproduces W^T X, X H_new^T and H_new H_new^T.
"""

import numpy as np
import pytest

BOX_COLS = 32
# (rows bucket MP, columns per lane CPL): the configurations the pass launches
CONFIGS = [(32, 4), (16, 2)]


def _x_addr(sa, ii, ch, cw):
    row = sa + 8 * ii
    return row * 128 + ((ch ^ (row & 7)) << 4) + cw


def _h_addr(row, ch, cw):
    return row * 128 + ((ch ^ row) << 4) + cw


def _lane_cols(step, cq, cpl):
    cb = (step * 4 + cq) * cpl * 4          # byte offset of the lane's columns in a row
    return cb >> 4, cb & 15, cb // 4        # chunk, byte within chunk, first column


@pytest.mark.parametrize("mp,cpl", CONFIGS)
def test_accesses_stay_inside_the_boxes(mp, cpl):
    rpl, nstep = mp // 8, BOX_COLS // (4 * cpl)
    xbox, hbox = mp * 128, 8 * 128
    seen = set()
    for step in range(nstep):
        for lane in range(32):
            sa, cq = lane & 7, lane >> 3
            ch, cw, c0 = _lane_cols(step, cq, cpl)
            assert 0 <= c0 and c0 + cpl <= BOX_COLS
            for ii in range(rpl):
                a = _x_addr(sa, ii, ch, cw)
                assert 0 <= a and a + 4 * cpl <= xbox
                assert a % (4 * cpl) == 0           # vector loads are naturally aligned
                seen.update((sa + 8 * ii, c0 + c) for c in range(cpl))
            for i in range(8):
                a = _h_addr(sa ^ i, ch, cw)
                assert 0 <= a and a + 4 * cpl <= hbox and a % (4 * cpl) == 0
    # the lanes of a warp cover every (row, column) of the X box exactly
    assert seen == {(r, c) for r in range(mp) for c in range(BOX_COLS)}


@pytest.mark.parametrize("mp,cpl", CONFIGS)
def test_shared_loads_are_conflict_free(mp, cpl):
    rpl, nstep = mp // 8, BOX_COLS // (4 * cpl)
    width = 4 * cpl                            # bytes per lane
    phase = 128 // width                       # lanes served by one 128-byte wavefront

    def check(addrs):
        for p0 in range(0, 32, phase):
            words = {}
            for a in addrs[p0:p0 + phase]:
                words.setdefault((a % 128) // width, set()).add(a)
            # one address per bank group (equal addresses are a broadcast)
            assert all(len(v) == 1 for v in words.values()), words

    for step in range(nstep):
        cols = [_lane_cols(step, lane >> 3, cpl) for lane in range(32)]
        for ii in range(rpl):
            check([_x_addr(lane & 7, ii, cols[lane][0], cols[lane][1]) for lane in range(32)])
        for i in range(8):
            check([_h_addr((lane & 7) ^ i, cols[lane][0], cols[lane][1]) for lane in range(32)])


def _shfl_xor(vals, mask):
    """vals[lane] -> value of lane ^ mask, for the 32 lanes of a warp."""
    return [vals[lane ^ mask] for lane in range(32)]


@pytest.mark.parametrize("mp,cpl", CONFIGS)
def test_lane_model_reproduces_the_products(mp, cpl):
    """One box through the lane-level model: W rows sa + 8 ii in slot order
    (slot i = rank i ^ sa), rank-pair accumulators, the three reduce-scatter
    steps, the H update, the H_new gather from lanes ^ 2j and ^ 2j + 1, and P,
    Q in the slot order the end-of-kernel reduction unscrambles."""
    rng = np.random.default_rng(7)
    r = 8
    rpl, nstep = mp // 8, BOX_COLS // (4 * cpl)
    X = rng.random((mp, BOX_COLS))
    W = rng.random((mp, r))
    H = rng.random((r, BOX_COLS))
    G = W.T @ W
    eps = 1e-12
    Y_ref = W.T @ X
    Hn_ref = np.maximum(0.0, H * Y_ref / (G @ H + eps))
    P = np.zeros((mp, r))
    Q = np.zeros((r, r))
    Hn = np.zeros((r, BOX_COLS))
    for step in range(nstep):
        c0s = [_lane_cols(step, lane >> 3, cpl)[2] for lane in range(32)]
        # rank-pair partials y2[lane][j][c] = (slot 2j, slot 2j + 1) at column c
        y2 = []
        for lane in range(32):
            sa, c0 = lane & 7, c0s[lane]
            acc = np.zeros((4, cpl, 2))
            for ii in range(rpl):
                row = sa + 8 * ii
                for j in range(4):
                    for c in range(cpl):
                        acc[j, c, 0] += W[row, (2 * j) ^ sa] * X[row, c0 + c]
                        acc[j, c, 1] += W[row, (2 * j + 1) ^ sa] * X[row, c0 + c]
            y2.append(acc)
        # lane xor 4: keep pairs 0, 1 and add the partner's pairs 2, 3
        up = _shfl_xor([a[2:4].copy() for a in y2], 4)
        y2 = [np.concatenate([a[0:2] + u, a[2:4]]) for a, u in zip(y2, up)]
        # lane xor 2: keep pair 0 and add the partner's pair 1
        up = _shfl_xor([a[1].copy() for a in y2], 2)
        y2 = [np.concatenate([(a[0] + u)[None], a[1:]]) for a, u in zip(y2, up)]
        # lane xor 1: slot 0 plus the partner's slot 1
        up = _shfl_xor([a[0, :, 1].copy() for a in y2], 1)
        yv = [a[0, :, 0] + u for a, u in zip(y2, up)]
        hn = []
        for lane in range(32):
            sa, c0 = lane & 7, c0s[lane]
            cols = slice(c0, c0 + cpl)
            assert np.allclose(yv[lane], Y_ref[sa, cols], rtol=1e-12)
            gh = sum(G[sa, sa ^ i] * H[sa ^ i, cols] for i in range(8))
            h = np.maximum(0.0, H[sa, cols] * yv[lane] / (gh + eps))
            hn.append(h)
            Hn[sa, cols] = h
        for lane in range(32):
            sa, c0 = lane & 7, c0s[lane]
            for j in range(4):
                a = hn[lane ^ (2 * j)]          # rank sa ^ 2j
                b = hn[lane ^ (2 * j + 1)]      # rank sa ^ (2j + 1)
                for ii in range(rpl):
                    row = sa + 8 * ii
                    x = X[row, c0:c0 + cpl]
                    P[row, (2 * j) ^ sa] += np.dot(x, a)
                    P[row, (2 * j + 1) ^ sa] += np.dot(x, b)
                Q[sa, (2 * j) ^ sa] += np.dot(hn[lane], a)
                Q[sa, (2 * j + 1) ^ sa] += np.dot(hn[lane], b)
    assert np.allclose(Hn, Hn_ref, rtol=1e-12)
    assert np.allclose(P, X @ Hn_ref.T, rtol=1e-12)
    assert np.allclose(Q, Hn_ref @ Hn_ref.T, rtol=1e-12)


# ---------------------------------------------------------------------------
# The 3-D-copy form for 32 rows (n a multiple of 32): a stage holds NB = 2
# adjacent 32-column segments of every X and H row as 128-byte lines ordered
# (row, segment), 16-byte chunks XOR line mod 8; four row splits x eight
# column groups (lane = sb + 4 cq), two columns per lane per step, lane sb
# holding X rows sb + 4 ii and W in slot order slot i -> rank i ^ 2 sb; H
# rows read in the order i ^ sb, the lane's own ranks 2 sb, 2 sb + 1 once more.

NB = 2


def _row4(sb, ii):
    return sb + 4 * ii


def _lane_cols4(step, cq):
    cb = (step * 8 + cq) * 8                # byte offset of the lane's two columns in a line
    return cb >> 4, cb & 15, cb // 4


def _line_addr(row, g, ch, cw):
    line = row * NB + g
    return line * 128 + ((ch ^ (line & 7)) << 4) + cw


def _four_split_h_rows(sb):
    return [i ^ sb for i in range(8)] + [2 * sb, 2 * sb + 1]


def test_four_split_accesses_stay_inside_the_boxes():
    mp, rpl = 32, 8
    xbox, hbox = mp * NB * 128, 8 * NB * 128
    seen, hseen = set(), set()
    for g in range(NB):
        for step in range(2):
            for lane in range(32):
                sb, cq = lane & 3, lane >> 2
                ch, cw, c0 = _lane_cols4(step, cq)
                assert 0 <= c0 and c0 + 2 <= BOX_COLS
                for ii in range(rpl):
                    a = _line_addr(_row4(sb, ii), g, ch, cw)
                    assert 0 <= a and a + 8 <= xbox and a % 8 == 0
                    seen.update((_row4(sb, ii), 32 * g + c0 + c) for c in range(2))
                for row in _four_split_h_rows(sb):
                    a = _line_addr(row, g, ch, cw)
                    assert 0 <= a and a + 8 <= hbox and a % 8 == 0
                    hseen.update((row, 32 * g + c0 + c) for c in range(2))
    assert seen == {(r, c) for r in range(mp) for c in range(NB * BOX_COLS)}
    assert hseen == {(r, c) for r in range(8) for c in range(NB * BOX_COLS)}


def test_four_split_shared_loads_are_conflict_free():
    """Every X load and the eight G H loads: the 16 lanes of each half-warp
    cover the 32 banks once.  The two loads of the lane's own ranks are
    allowed a two-way conflict (the only loads that have one)."""
    def ways(addrs):
        worst = 1
        for p0 in range(0, 32, 16):            # 8-byte loads: 16 lanes per wavefront
            words = {}
            for a in addrs[p0:p0 + 16]:
                words.setdefault((a % 128) // 8, set()).add(a)
            worst = max(worst, max(len(v) for v in words.values()))
        return worst

    for g in range(NB):
        for step in range(2):
            cols = [_lane_cols4(step, lane >> 2) for lane in range(32)]
            for ii in range(8):
                assert ways([_line_addr(_row4(lane & 3, ii), g, cols[lane][0], cols[lane][1])
                             for lane in range(32)]) == 1
            for i in range(8):
                assert ways([_line_addr(i ^ (lane & 3), g, cols[lane][0], cols[lane][1])
                             for lane in range(32)]) == 1
            for e in range(2):
                assert ways([_line_addr(2 * (lane & 3) + e, g, cols[lane][0], cols[lane][1])
                             for lane in range(32)]) <= 2


def test_four_split_lane_model_reproduces_the_products():
    """One stage through the lane-level model of the 3-D-copy form: rank-pair
    partials in slot order, the two reduce-scatter steps (lane xor 2, then
    xor 1), the H update of ranks 2 sb, 2 sb + 1 with G H summed in the read
    order i ^ sb, the H_new gather from lanes ^ d, and P, Q in the order the
    end-of-kernel reduction writes."""
    rng = np.random.default_rng(11)
    mp, r, rpl = 32, 8, 8
    ncol = NB * BOX_COLS
    X = rng.random((mp, ncol))
    W = rng.random((mp, r))
    H = rng.random((r, ncol))
    G = W.T @ W
    eps = 1e-12
    Y_ref = W.T @ X
    Hn_ref = np.maximum(0.0, H * Y_ref / (G @ H + eps))
    P = np.zeros((mp, r))
    Q = np.zeros((r, r))
    Hn = np.zeros((r, ncol))
    for g in range(NB):
        for step in range(2):
            c0s = [32 * g + _lane_cols4(step, lane >> 2)[2] for lane in range(32)]
            y2 = []   # y2[lane][j, c, e] = slot 2j + e at column c
            for lane in range(32):
                sb, c0 = lane & 3, c0s[lane]
                acc = np.zeros((4, 2, 2))
                for ii in range(rpl):
                    row = _row4(sb, ii)
                    for j in range(4):
                        for e in range(2):
                            acc[j, :, e] += W[row, (2 * j + e) ^ (2 * sb)] * X[row, c0:c0 + 2]
                y2.append(acc)
            # lane xor 2: pairs 0, 1 plus the partner's pairs 2, 3
            up = _shfl_xor([a[2:4].copy() for a in y2], 2)
            y2 = [np.concatenate([a[0:2] + u, a[2:4]]) for a, u in zip(y2, up)]
            # lane xor 1: pair 0 plus the partner's pair 1
            up = _shfl_xor([a[1].copy() for a in y2], 1)
            yv = [a[0] + u for a, u in zip(y2, up)]          # [c, e] = Y[2 sb + e] at column c
            hn = []
            for lane in range(32):
                sb, c0 = lane & 3, c0s[lane]
                cols = slice(c0, c0 + 2)
                h = np.zeros((2, 2))                           # [c, e]
                for e in range(2):
                    k = 2 * sb + e
                    assert np.allclose(yv[lane][:, e], Y_ref[k, cols], rtol=1e-12)
                    gh = sum(G[k, i ^ sb] * H[i ^ sb, cols] for i in range(8))
                    h[:, e] = np.maximum(0.0, H[k, cols] * yv[lane][:, e] / (gh + eps))
                    Hn[k, cols] = h[:, e]
                hn.append(h)
            for lane in range(32):
                sb, c0 = lane & 3, c0s[lane]
                for d in range(4):
                    hp = hn[lane ^ d]                          # ranks 2 (sb ^ d) + e
                    for e in range(2):
                        k = 2 * (sb ^ d) + e
                        for ii in range(rpl):
                            row = _row4(sb, ii)
                            P[row, k] += np.dot(X[row, c0:c0 + 2], hp[:, e])
                        for e2 in range(2):
                            Q[2 * sb + e2, k] += np.dot(hn[lane][:, e2], hp[:, e])
    assert np.allclose(Hn, Hn_ref, rtol=1e-12)
    assert np.allclose(P, X @ Hn_ref.T, rtol=1e-12)
    assert np.allclose(Q, Hn_ref @ Hn_ref.T, rtol=1e-12)

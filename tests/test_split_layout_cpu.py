"""Host-side model of the split tensor-core form's tile-major X image (no GPU).

split_blocked_kernel (csrc/mu_pass_tcs.cu) writes X1 = bf16(X) and
X2 = bf16(X - X1) tile by tile (64 columns) as the pass's shared-memory
stage: 8-row groups of X1 and X2 alternate in 1024-byte atoms, row r8 of a
group at r8 * 128, its 16-byte chunk c at (c ^ r8) * 16.  The pass's MMA
descriptors read that stage with the second term at XLBO = 1024 bytes and
8-row groups at XSBO = 2048.  These tests restate the kernel's thread-index
arithmetic and check that it writes every byte of the image once, in bounds,
and that the descriptor offsets find element (term, row, col) where the
kernel put it.
"""

import numpy as np
import pytest


def kernel_writes(m, n, mp):
    """(tile, row, chunk) per thread as the kernel decomposes q; returns the
    byte ranges each thread writes for X1 and X2 with their (term, row, col0)."""
    ntiles = (n + 63) // 64
    out = []
    for q in range(ntiles * mp * 8):
        c = q & 7
        rowt = q >> 3
        row = rowt % mp
        t = rowt // mp
        g, r8 = row >> 3, row & 7
        base = ((t * (mp // 8) + g) * 2) * 1024 + r8 * 128 + ((c ^ r8) << 4)
        out.append((base, 0, t, row, c * 8))
        out.append((base + 1024, 1, t, row, c * 8))
    return ntiles, out


@pytest.mark.parametrize("m,n,mp", [(256, 256, 256), (200, 192 + 8, 256), (512, 128, 512), (128, 64, 128)])
def test_blocked_image_is_written_once_and_matches_the_descriptors(m, n, mp):
    ntiles, writes = kernel_writes(m, n, mp)
    xst = mp * 128 * 2
    assert ntiles * xst == ((n + 63) // 64) * mp * 256           # split_blocked_bytes
    covered = np.zeros(ntiles * xst, dtype=np.int32)
    for base, term, t, row, col0 in writes:
        assert 0 <= base and base + 16 <= ntiles * xst
        covered[base:base + 16] += 1
        # the stage of tile t starts at t * XST; inside it the descriptors put
        # (term, row, col) at (row / 8) * XSBO + term * XLBO + (row % 8) * 128 + swizzled chunk
        off = base - t * xst
        assert 0 <= off < xst
        xlbo, xsbo = 1024, 2048
        expect = (row >> 3) * xsbo + term * xlbo + (row & 7) * 128 + ((((col0 >> 3) ^ (row & 7))) << 4)
        assert off == expect
    assert np.all(covered == 1)


def test_phase_b_row_blocks_and_k_steps():
    """Phase B reads 128-row blocks at mb * 16 * XSBO and the K steps past 64
    columns (the X2 term) at + XLBO: element (term, row, col) of the stage."""
    mp = 256
    for mb in range(mp // 128):
        for kk in range(8):
            term, k16 = kk >> 2, (kk & 3) * 16
            for row in range(mb * 128, mb * 128 + 128, 37):
                for col in (k16, k16 + 15):
                    # descriptor start + the row's place in 8-row groups (SBO) and the swizzle
                    start = mb * 16 * 2048 + term * 1024 + (kk & 3) * 32
                    r = row - mb * 128
                    addr_desc = start - (kk & 3) * 32 + (r >> 3) * 2048 + (r & 7) * 128 + \
                        ((((col >> 3) ^ (r & 7))) << 4) + (col & 7) * 2
                    addr_img = (row >> 3) * 2048 + term * 1024 + (row & 7) * 128 + \
                        ((((col >> 3) ^ (row & 7))) << 4) + (col & 7) * 2
                    assert addr_desc == addr_img

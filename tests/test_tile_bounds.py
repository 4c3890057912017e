"""CPU replica of the 2D CUDA-core tile's index arithmetic (sweep2d_tile.cuh,
k_sweep2d.cu): every shared-memory read and write of the direct sweeps and of
the counterpart form's vertical and horizontal folds stays inside its buffer
plus the 32-float slack on each side, for every blocking depth and folded
radius the library runs, full and ragged tiles alike.  Also checks that the
precomputed full-tile item split reproduces the generic one.

The formulas below restate the kernels' region, strip and row-group
arithmetic; a change there must be mirrored here.
"""

import itertools

import pytest

TX = 128        # output columns per tile
BUF_PAD = 32    # floats of slack before and after each shared-memory buffer
NTHR = 512


def rup(v, m):
    return (v + m - 1) // m * m


def items(nsx, nr, R, nthr=NTHR, window=True):
    """(k offset, ya, yb) of every thread's item; window: runs of >= 2R rows."""
    G = nthr // nsx
    G = max(1, min(G, nr // (2 * R) if window else nr))
    out = []
    for it in range(0, nsx * G):
        k, g = it % nsx, it // nsx
        out.append((k, (g * nr) // G, ((g + 1) * nr) // G))
    return out, G


def check_range(lo, hi, SP, ROWS, what):
    """Flat float offsets [lo, hi) relative to a buffer's first data float."""
    assert lo >= -BUF_PAD, (what, lo)
    assert hi <= SP * ROWS + BUF_PAD, (what, hi, SP * ROWS)


def direct_tile(R, b, TY, vx, vy):
    H = b * R
    HX = rup(H, 4)
    SP, ROWS = TX + 2 * HX, TY + 2 * H
    RP = rup(R, 4)
    for s in range(b):
        sh = (s + 1) * R
        final = s == b - 1
        r0, r1 = (H, H + vy) if final else (sh, 2 * H + vy - sh)
        c0, c1 = (HX, HX + vx) if final else (HX - H + sh, HX + vx + H - sh)
        k0, k1 = c0 // 4, (c1 + 3) // 4
        its, _ = items(k1 - k0, r1 - r0, R)
        for k, ya, yb in its:
            cx = 4 * (k0 + k)
            ya, yb = r0 + ya, r0 + yb
            # input rows ya-R .. yb+R-1, columns cx-RP .. cx+4+RP
            check_range((ya - R) * SP + cx - RP, (yb + R - 1) * SP + cx + 4 + RP, SP, ROWS,
                        "direct read")
            if not final:
                check_range(ya * SP + cx, (yb - 1) * SP + cx + 4, SP, ROWS, "direct write")


def counterpart_tile(R, b, TY, vx, vy):
    H = b * R
    HX = rup(H, 4)
    SP, ROWS = TX + 2 * HX, TY + 2 * H
    RP = rup(R, 4)
    CW = 2 if R >= 6 else 4
    for s in range(b):
        sh = (s + 1) * R
        r0, r1 = sh, 2 * H + vy - sh
        c0, c1 = HX - H + sh, HX + vx + H - sh
        # vertical fold over columns [x0, x1) in strips of CW
        x0, x1 = (c0 - R) // 4 * 4, (c1 + R + 3) // 4 * 4
        assert x0 >= 0 and x1 <= SP
        its, _ = items(x1 // CW - x0 // CW, r1 - r0, R)
        for k, ya, yb in its:
            col = CW * (x0 // CW + k)
            ya, yb = r0 + ya, r0 + yb
            check_range((ya - R) * SP + col, (yb + R - 1) * SP + col + CW, SP, ROWS, "vfold read")
            check_range(ya * SP + col, (yb - 1) * SP + col + CW, SP, ROWS, "vfold write")
        # horizontal fold: every output row on its own
        k0, k1 = c0 // 4, (c1 + 3) // 4
        its, _ = items(k1 - k0, r1 - r0, R, window=False)
        for k, ya, yb in its:
            cx = 4 * (k0 + k)
            ya, yb = r0 + ya, r0 + yb
            check_range(ya * SP + cx - RP, (yb - 1) * SP + cx + 4 + RP, SP, ROWS, "hfold read")
            if s < b - 1:
                check_range(ya * SP + cx, (yb - 1) * SP + cx + 4, SP, ROWS, "hfold write")


SHAPES = [(128, None), (1, 1), (3, 5), (77, 37), (124, 8)]


@pytest.mark.parametrize("R", [1, 2, 3, 4, 6, 8])
def test_direct_sweep_accesses_stay_in_buffers(R):
    for b in range(1, 17):
        if b * R > 16:
            break
        for TY in range(16, 193, 8):
            if TY + 2 * b * R > 256:
                continue
            for vx, vy in SHAPES:
                direct_tile(R, b, TY, vx, TY if vy is None else min(vy, TY))


@pytest.mark.parametrize("R", [1, 2, 3, 4, 6, 8])
def test_counterpart_accesses_stay_in_buffers(R):
    for b in range(1, 17):
        if b * R > 16:
            break
        for TY in range(16, 193, 8):
            if TY + 2 * b * R > 256:
                continue
            for vx, vy in SHAPES:
                counterpart_tile(R, b, TY, vx, TY if vy is None else min(vy, TY))


def test_full_tile_split_matches_generic():
    """The once-per-CTA split (multiply-high reciprocals) equals the divisions."""
    def magic(d):
        return (0x100000000 + d - 1) // d
    for R, b, TY, nthr in itertools.product([1, 2, 3, 4, 6, 8], range(1, 9),
                                            range(16, 193, 8), (256, 512)):
        if b * R > 16 or TY + 2 * b * R > 256:
            continue
        H = b * R
        HX = rup(H, 4)
        for s in range(b):
            if s < b - 1:
                sh = (s + 1) * R
                nr = 2 * H + TY - 2 * sh
                k0, k1 = (HX - H + sh) // 4, (HX + TX + H - sh + 3) // 4
            else:
                nr, k0, k1 = TY, HX // 4, (HX + TX + 3) // 4
            nsx = k1 - k0
            G = max(1, min(nthr // nsx, nr // (2 * R)))
            if nsx < 2 or G < 2:
                continue  # such sweeps keep the divisions
            mn, mg = magic(nsx), magic(G)
            for it in range(nsx * G):
                g = (it * mn) >> 32
                got = (it - g * nsx, g, (g * nr * mg) >> 32, ((g + 1) * nr * mg) >> 32)
                want = (it % nsx, it // nsx, (it // nsx) * nr // G, (it // nsx + 1) * nr // G)
                assert got == want, (R, b, TY, s, it)

"""Index models of the fused level passes (no GPU): the thread-to-tile mappings of
k_zero_residual_restrict and k_prolong_jacobi in kernels_mg.cu, replayed in Python for
square, non-square and both block shapes.  They check that every shared-memory index is
in range, that every tile entry a stencil or the restriction reads was filled by the
stage before, that every fine node's zero-start value is written by exactly one block,
and that the prolongation fills each needed entry once from the coarse cell that holds
it.  The kernels index exactly as modelled here (constants and formulas are the same)."""
import pytest

BX, BY = 32, 8                      # stencil blocks (level_by chooses BY or 2)
DBX, DBY = 16, 8                    # coarse block of the residual-restriction pass
DUW, DRW = 2 * DBX + 3, 2 * DBX + 1
SMS = 152


def level_by(mx, my):
    return 2 if mx * my < 2 * SMS * BX * BY else BY


def check_down(mx, my):
    mcx, mcy = (mx - 1) // 2, (my - 1) // 2
    cby = 2 if mcx * mcy < 2 * SMS * DBX * DBY else DBY
    nthr = DUW * (2 * cby + 3)
    assert nthr <= DUW * (2 * DBY + 3) <= 1024
    assert (nthr // DUW - 3) // 2 == cby                       # the kernel recovers cby
    written = {}
    for I0 in range(0, mcx, DBX):
        for J0 in range(0, mcy, cby):
            filled = set()
            for t in range(nthr):                                 # stage 1: u on the tile
                a, b = t % DUW, t // DUW
                assert b < 2 * DBY + 3
                i, j = 2 * I0 - 1 + a, 2 * J0 - 1 + b
                filled.add((a, b))
                if 0 <= i < mx and 0 <= j < my:
                    oi, oj = min(i >> 1, mcx - 1), min(j >> 1, mcy - 1)
                    if I0 <= oi < I0 + DBX and J0 <= oj < J0 + cby:
                        written[(i, j)] = written.get((i, j), 0) + 1
            rh = 2 * cby + 1
            res = set()
            for t in range(min(nthr, DRW * rh)):                  # stage 2: residuals
                a, b = t % DRW, t // DRW
                i, j = 2 * I0 + a, 2 * J0 + b
                if i >= mx or j >= my:
                    continue
                for q in ((a + 1, b + 1), (a, b + 1), (a + 2, b + 1), (a + 1, b), (a + 1, b + 2)):
                    assert q in filled
                assert b < 2 * DBY + 1
                res.add((a, b))
            for t in range(min(nthr, DBX * cby)):                 # stage 3: restriction
                I, J = I0 + t % DBX, J0 + t // DBX
                if I < mcx and J < mcy:
                    a, b = 2 * (t % DBX) + 1, 2 * (t // DBX) + 1
                    assert all((a + dx, b + dy) in res for dx in (-1, 0, 1) for dy in (-1, 0, 1))
    assert all(written.get((i, j), 0) == 1 for i in range(mx) for j in range(my))


def check_up(mx, my):
    mcx, mcy = (mx - 1) // 2, (my - 1) // 2
    by = level_by(mx, my)
    for i0 in range(0, mx, BX):
        for j0 in range(0, my, by):
            K0, K1 = (i0 - 1) >> 1, (i0 + BX) >> 1
            L0, L1 = (j0 - 1) >> 1, (j0 + by) >> 1
            nkx = K1 - K0 + 1
            ncell = nkx * (L1 - L0 + 1)
            assert ncell <= BX * by
            count = {}
            for q in range(ncell):
                K, L = K0 + q % nkx, L0 + q // nkx
                if K < 0 or L < 0 or K > mcx or L > mcy:
                    continue
                for n in range(4):
                    i, j = 2 * K + (n & 1), 2 * L + (n >> 1)
                    if i >= mx or j >= my or i < i0 - 1 or i > i0 + BX or j < j0 - 1 or j > j0 + by:
                        continue
                    ti, tj = i - i0 + 1, j - j0 + 1
                    assert 0 <= ti < BX + 2 and 0 <= tj < BY + 2
                    count[(ti, tj)] = count.get((ti, tj), 0) + 1
            for ty in range(by):
                for tx in range(BX):
                    i, j = i0 + tx, j0 + ty
                    if i >= mx or j >= my:
                        continue
                    for di, dj in ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)):
                        inside = 0 <= i + di < mx and 0 <= j + dj < my
                        assert count.get((tx + 1 + di, ty + 1 + dj), 0) == (1 if inside else 0)


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 16), (32, 32), (64, 64), (128, 128), (256, 256), (512, 512),
                                   (64, 32), (32, 128), (256, 64)])
def test_fused_pass_tilings(nx, ny):
    check_down(nx - 1, ny - 1)
    check_up(nx - 1, ny - 1)

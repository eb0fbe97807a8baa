"""Pin of the oracle's tile rectangle (the last step of the FP32 decision spec) against a
rectangle the test builds itself.

The 3DGS binning that the paper's rasterizer inherits (Supp. A.3) lists a Gaussian in every
screen tile its 3-sigma square [u - r, u + r] x [v - r, v + r] reaches, with r = ceil(3 sqrt
(lambda_max)) of the projected covariance and the half-open tile range
[floor((u - r) / TW), floor((u + r + TW - 1) / TW)) clamped to the grid. Stated per tile, that
range is every tile tx of the grid with u - r < TW (tx + 1) (the square starts left of the
tile's right edge) and u + r >= TW tx + 1 (it reaches at least one pixel into the tile); a
Gaussian with no such tile in x or in y is culled.

Here the screen mean (u, v) and the radius r come from the Gaussian's parameters by the
textbook EWA closed form in FP64 (an isotropic Gaussian at depth 1 in front of an identity
camera, J = [[fx, 0, -fx x], [0, fy, -fy y]], Sigma' = s^2 J J^T + 0.3 I), on inputs chosen so
that FP32 rounding cannot move either: power-of-two focal lengths, dyadic means, 3 sqrt(lambda)
half a pixel away from an integer. The tiles come from the per-tile membership test above,
iterated over the grid, so a floor/ceil, off-by-one or clamp slip in the oracle's arithmetic
fails one of the cases: left and right square edges exactly on, 1/256 px below and 1/256 px
above a tile edge, squares clamped at either image border, squares wholly outside, ragged image
sizes, and both tile shapes (16 x 16 and 8 x 32).
"""
import math

import numpy as np
import pytest

import oracle

FX = FY = 128.0          # power of two: fx * x is exact for dyadic x
DELTA = 2.0 ** -8        # a sub-pixel step that every value below represents exactly


def fparams(W, H):
    fp = np.zeros(20, np.float32)
    fp[0] = fp[5] = fp[10] = 1.0      # world-to-camera rotation = I
    fp[11] = 1.0                      # t = (0, 0, 1): the plane z = 0 sits at depth 1
    fp[12], fp[13] = FX, FY
    fp[14], fp[15] = W / 2.0, H / 2.0
    fp[16] = 0.2                      # near plane
    return fp


def lam_max(s, x, y):
    """Larger eigenvalue of Sigma' = s^2 J J^T + 0.3 I in the form the renderer uses
    (mid + sqrt(max(0.1, mid^2 - det)), whose 0.1 floor only matters for near-isotropic
    splats), for an isotropic Gaussian of scale s at (x, y, 0) seen from depth 1."""
    a = s * s * FX * FX * (1 + x * x) + 0.3
    c = s * s * FY * FY * (1 + y * y) + 0.3
    b = s * s * FX * FY * x * y
    mid = 0.5 * (a + c)
    det = a * c - b * b
    return mid + math.sqrt(max(0.1, mid * mid - det))


def scale_for_radius(r, x, y):
    """The scale s whose 3 sqrt(lambda) is r - 1/2 (bisection in FP64), returned as the
    FP32-rounded log-scale and the FP64 radius it gives, asserted half a pixel clear of the
    integers so that the FP32 spec rounds to the same ceiling."""
    lo, hi = 1e-6, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if 3 * math.sqrt(lam_max(mid, x, y)) < r - 0.5:
            lo = mid
        else:
            hi = mid
    ls = float(np.float32(math.log(lo)))
    q = 3 * math.sqrt(lam_max(math.exp(ls), x, y))
    assert abs(q - round(q)) > 0.4, q
    return ls, math.ceil(q)


def expected_range(c, r, tile, n_tiles):
    """Tiles whose span [tile t, tile (t + 1)) the square [c - r, c + r] reaches, per the
    membership test of the module docstring; None when there are none."""
    ts = [t for t in range(n_tiles) if c - r < tile * (t + 1) and c + r >= tile * t + 1]
    return (ts[0], ts[-1] + 1) if ts else None


def build_case(W, H, tile, cases):
    """cases: (u, v, r) targets. Returns the model arrays and the expected rectangles."""
    TW, TH = tile
    n = len(cases)
    n_pad = (n + 3) // 4 * 4
    g0 = np.zeros((14, n_pad), np.float32)
    cx, cy = W / 2.0, H / 2.0
    want = []
    for i, (u, v, r) in enumerate(cases):
        x, y = (u - cx) / FX, (v - cy) / FY
        assert np.float32(x) == x and np.float32(y) == y   # dyadic, exact in FP32
        assert abs(x) < 1.3 * cx / FX and abs(y) < 1.3 * cy / FY  # the Jacobian clamp is off
        ls, r_got = scale_for_radius(r, x, y)
        assert r_got == r
        g0[0, i], g0[1, i], g0[2, i] = x, y, 0.0
        g0[3, i] = 1.0                                 # identity rotation
        g0[7:10, i] = ls
        g0[10, i] = 2.0
        g0[11:14, i] = 0.5
        ex = expected_range(u, r, TW, (W + TW - 1) // TW)
        ey = expected_range(v, r, TH, (H + TH - 1) // TH)
        want.append((0, 0, 0, 0) if ex is None or ey is None else (ex[0], ey[0], ex[1], ey[1]))
    return g0, np.zeros((1, 9, n_pad), np.float32), np.asarray(want, np.int32)


def edge_cases(W, H, tile, r=7):
    """Squares whose left or right edge lands on, just below and just above a tile edge, in x
    and in y, plus squares clamped at each border and squares outside the image."""
    TW, TH = tile
    mx, my = W / 2.0 + 0.25, H / 2.0 + 0.75        # off-centre, dyadic
    out = []
    for e in (2, 3):                               # interior tile edges
        for d in (0.0, -DELTA, DELTA):
            out.append((TW * e + r + d, my, r))        # left edge of the square near TW e
            out.append((TW * e + 1 - r + d, my, r))    # right edge near TW e + 1
            out.append((mx, TH * e + r + d, r))        # top edge near TH e
            out.append((mx, TH * e + 1 - r + d, r))    # bottom edge near TH e + 1
    out += [(2.5, my, r), (W - 2.5, my, r), (mx, 3.25, r), (mx, H - 3.25, r),  # clamped
            (-r + 1.0, my, r), (-r + 1.0 - DELTA, my, r),                    # reaches pixel 0 or not
            (W + r - DELTA, my, r), (W + r, my, r),                          # starts left of W or not
            (mx, -r + 1.0 - DELTA, r), (mx, H + r, r)]                       # outside in y
    return out


@pytest.mark.parametrize("W,H,tile", [(200, 136, (16, 16)), (128, 128, (16, 16)),
                                      (200, 136, (8, 32)), (97, 161, (8, 32))])
def test_rectangles_match_per_tile_membership(W, H, tile):
    cases = edge_cases(W, H, tile)
    g0, dg, want = build_case(W, H, tile, cases)
    rect, f32 = oracle.decide(g0, dg, np.zeros(1, np.float32), fparams(W, H), len(cases),
                              0x7 | (0x7 << 7) | (0x7 << 11), W, H, tile[0], tile[1])
    np.testing.assert_array_equal(rect, want)
    kept = want[:, 2] > want[:, 0]
    assert 0 < kept.sum() < len(cases)            # both kept and culled squares occur
    u = np.array([c[0] for c in cases], np.float32)
    v = np.array([c[1] for c in cases], np.float32)
    r = np.array([c[2] for c in cases], np.float32)
    np.testing.assert_array_equal(f32[kept, 0], u[kept])   # the screen mean, exactly
    np.testing.assert_array_equal(f32[kept, 1], v[kept])
    np.testing.assert_array_equal(f32[kept, 5], r[kept])   # the 3-sigma radius


def test_membership_rule_flips_at_the_documented_edges():
    """The rule itself, on one tile edge: a square ending at TW e + 1 reaches tile e, one
    ending 1/256 px before does not; a square starting at TW e does not reach tile e - 1."""
    TW, r = 16, 7
    assert expected_range(TW * 3 + 1 - r, r, TW, 10)[1] == 4
    assert expected_range(TW * 3 + 1 - r - DELTA, r, TW, 10)[1] == 3
    assert expected_range(TW * 3 + r, r, TW, 10)[0] == 3
    assert expected_range(TW * 3 + r - DELTA, r, TW, 10)[0] == 2
    assert expected_range(-r + 1.0 - DELTA, r, TW, 10) is None

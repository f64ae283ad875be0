"""Pins for the oracle's Mandelbrot escape counts (Sec. 5, "Integrating OpenCL
Actors": a Mandelbrot image computed by a GPU actor).

The count of c is the number of updates z <- z^2 + c, from z = 0, made
before |z|^2 > 4 is first seen, at most max_iter.  The pins come from the
mathematics, not from the oracle's own formula:

* orbits that are exact in float32 (c = 0, -1, -2, i, 1, 2, 0.5, ...);
* exact rational orbits (Python Fractions) for points whose orbit stays
  well away from the threshold, so no float32 rounding can change the count;
* points strictly inside the main cardioid or the period-2 bulb never
  escape (their attracting cycle has multiplier of modulus < 1);
* |c| > 2 escapes after one update;
* complex conjugation maps the orbit of c to that of conj(c) exactly;
* the fraction of a grid that never escapes estimates the set's area,
  known to be about 1.5066.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle

MAXIT = 500


@pytest.mark.parametrize("c, count", [
    ((0.0, 0.0), MAXIT),        # z stays 0
    ((-1.0, 0.0), MAXIT),       # 0, -1, 0, -1, ...
    ((-2.0, 0.0), MAXIT),       # 0, -2, 2, 2, ...: |z|^2 = 4 is not > 4
    ((0.0, 1.0), MAXIT),        # 0, i, -1+i, -i, -1+i, ...
    ((0.25, 0.0), MAXIT),       # parabolic point: z increases towards 1/2
    ((1.0, 0.0), 3),            # 0, 1, 2, 5
    ((2.0, 0.0), 2),            # 0, 2, 6
    ((0.5, 0.0), 5),            # 0, .5, .75, 1.0625, 1.62890625, 3.15...
    ((3.0, 0.0), 1),
    ((1.5, 1.5), 1),            # |c|^2 = 4.5
    ((-2.0, 0.5), 1),           # |c|^2 = 4.25
])
def test_closed_form_orbits(c, count):
    assert oracle.mandel_point(c[0], c[1], MAXIT) == count


def test_max_iter_zero_and_one():
    assert oracle.mandel_point(0.0, 0.0, 0) == 0
    assert oracle.mandel_point(3.0, 0.0, 0) == 0
    assert oracle.mandel_point(0.0, 0.0, 1) == 1
    assert oracle.mandel_point(3.0, 0.0, 1) == 1


def _exact_escape(cx: float, cy: float, kmax: int, margin: Fraction):
    """Exact escape step of c (Fractions), or None if some |z_k|^2 (k up to the
    escape) lies within `margin` of 4 or the orbit does not escape by kmax."""
    cr, ci = Fraction(cx), Fraction(cy)
    zr = zi = Fraction(0)
    for k in range(kmax + 1):
        m = zr * zr + zi * zi
        if abs(m - 4) < margin:
            return None
        if m > 4:
            return k
        zr, zi = zr * zr - zi * zi + cr, 2 * zr * zi + ci
    return None


def test_exact_rational_orbits():
    rng = random.Random(1505)
    checked = 0
    while checked < 400:
        cx = float(np.float32(rng.uniform(-2.2, 1.0)))
        cy = float(np.float32(rng.uniform(-1.5, 1.5)))
        k = _exact_escape(cx, cy, 6, Fraction(1, 20))
        if k is None:
            continue
        assert oracle.mandel_point(cx, cy, MAXIT) == k, (cx, cy)
        checked += 1


def test_interior_points_never_escape():
    rng = random.Random(7368)
    for _ in range(300):
        r = rng.uniform(0.0, 0.8)
        t = rng.uniform(0.0, 2 * math.pi)
        w = complex(r * math.cos(t), r * math.sin(t)) / 2
        c = w * (1 - w)                                  # main cardioid: fixed point with multiplier 2w
        assert oracle.mandel_point(c.real, c.imag, 2000) == 2000, c
        c2 = complex(-1.0, 0.0) + complex(r * math.cos(t), r * math.sin(t)) / 4   # period-2 bulb
        assert oracle.mandel_point(c2.real, c2.imag, 2000) == 2000, c2


def test_outside_radius_two_escapes_at_once():
    rng = random.Random(11)
    for _ in range(300):
        r = rng.uniform(2.01, 50.0)
        t = rng.uniform(0.0, 2 * math.pi)
        assert oracle.mandel_point(r * math.cos(t), r * math.sin(t), MAXIT) == 1


def test_conjugate_symmetry_exact():
    # boundary-rich region: many counts between 1 and MAXIT
    counts, _ = oracle.mandel_rows(-0.80, 0.05, 0.004, 0.003, 64, 0, 48, MAXIT)
    mirrored, _ = oracle.mandel_rows(-0.80, -0.05, 0.004, -0.003, 64, 0, 48, MAXIT)
    assert len(np.unique(counts)) > 20
    assert np.array_equal(counts, mirrored)


def test_area_estimate():
    # grid over [-2, 0.5] x [0, 1.25] (upper half; the set is symmetric), pixel centres
    w, h = 500, 250
    dx = 2.5 / w
    dy = 1.25 / h
    counts, _ = oracle.mandel_rows(-2.0 + dx / 2, dy / 2, dx, dy, w, 0, h, 1000)
    area = 2 * (counts == 1000).sum() * dx * dy
    assert 1.49 < area < 1.54, area


def test_rows_layout_and_sum():
    # row0 offsets the imaginary part; out is row-major (rows, width)
    x0, y0, dx, dy = -0.7, -0.3, 0.01, 0.02
    full, s_full = oracle.mandel_rows(x0, y0, dx, dy, 37, 0, 11, 200)
    part, s_part = oracle.mandel_rows(x0, y0, dx, dy, 37, 4, 5, 200)
    assert full.shape == (11, 37) and part.shape == (5, 37)
    assert np.array_equal(part, full[4:9])
    assert s_full == int(full.astype(np.uint64).sum()) and s_part == int(part.astype(np.uint64).sum())
    f32 = np.float32
    for (j, i) in [(0, 0), (3, 36), (10, 17)]:
        cx = f32(f32(x0) + f32(f32(i) * f32(dx)))
        cy = f32(f32(y0) + f32(f32(j) * f32(dy)))
        assert full[j, i] == oracle.mandel_point(float(cx), float(cy), 200)


def test_no_fused_multiply_add():
    """Build-flag check (not a pin): numpy's float32 arithmetic rounds every
    operation, so the oracle library must agree with it bit for bit."""
    f32 = np.float32
    w, h, it = 48, 32, 300
    x0, y0, dx, dy = f32(-0.76), f32(0.04), f32(0.0021), f32(0.0017)
    cx = (x0 + np.arange(w, dtype=f32) * dx)[None, :].repeat(h, 0)
    cy = (y0 + np.arange(h, dtype=f32) * dy)[:, None].repeat(w, 1)
    zr = np.zeros((h, w), f32)
    zi = np.zeros((h, w), f32)
    k = np.zeros((h, w), np.uint32)
    live = np.ones((h, w), bool)
    with np.errstate(over="ignore", invalid="ignore"):
        for _ in range(it):
            x2 = zr * zr
            y2 = zi * zi
            live &= ~(x2 + y2 > f32(4))
            xy = zr * zi
            zi = np.where(live, (xy + xy) + cy, zi)
            zr = np.where(live, (x2 - y2) + cx, zr)
            k += live
    counts, _ = oracle.mandel_rows(float(x0), float(y0), float(dx), float(dy), w, 0, h, it)
    assert np.array_equal(counts, k)

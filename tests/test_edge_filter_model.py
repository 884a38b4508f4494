"""CPU check of a2's FP32 edge filter (no GPU).

a2 decides "certainly inside edge k" or "certainly outside" from the FP32
evaluation d = fma(A, Y, fma(-B, X, C)) of the edge function orient(E_k,
E_{k+1}, P) = A py - B px + C on the point's FP32 views X, Y, where A, B, C
are the edge's float64 coefficients rounded to float32 and E is a bound on
the evaluation's error, rounded up (the derivation sits beside
`edge_filter` in csrc/k_round1.cu).  Only |d| <= E goes to the exact test.
This module restates the view (significand truncation of the float64 bits),
the coefficients, the bound and both fused multiply-adds (each rounded to
nearest float32 from the exact rational value), and checks against the exact
orientation of the float64 points that |d| > E never gives the wrong side:
on points exactly on the edge line, points a few float64 ulps off it, and
random points of the bounding box, at magnitudes across the domain the
filter is used in (coordinates below 2^60).
"""
from fractions import Fraction
import math
import sys

import numpy as np
import pytest

U = 5.9604644775390625e-08        # 2^-24


def trunc_view(x):
    """The FP32 view of float64 values, bit for bit as the device forms it:
    exponent rebiased, significand truncated, below 2^-126 a signed zero."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.int64)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(np.int64)
    t = (hi & 0x7FFFFFFF) - 0x38000000
    sign = hi & 0x80000000
    body = ((t << 3) | (lo >> 29)) & 0xFFFFFFFF
    bits = np.where(t < 0, sign, sign | body).astype(np.uint32)
    return bits.view(np.float32)


def rn32(q):
    """A rational rounded to the nearest float32 (ties to even), subnormals
    included."""
    if q == 0:
        return np.float32(0.0)
    neg = q < 0
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    e = max(e, -126)                          # below: the subnormal grid
    scaled = q / Fraction(2) ** (e - 23)      # in [2^23, 2^24) for normals
    m = math.floor(scaled)
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    v = math.ldexp(m, e - 23)
    return np.float32(-v if neg else v)


def edge_coeffs(ax, ay, bx, by, xm, ym):
    """edge_filter: float64 coefficients, rounded to float32; the bound
    rounded up."""
    A, B = bx - ax, by - ay
    C = B * ax - A * ay
    Mc = abs(B) * abs(ax) + abs(A) * abs(ay)
    E = 6.0 * U * (abs(A) * ym + abs(B) * xm + Mc) + (abs(A) + abs(B)) * 2.0 ** -125 \
        + 2.0 ** -147 * (xm + ym + 1.0)
    fE = np.float32(E)
    if float(fE) < E:
        fE = np.nextafter(fE, np.float32(np.inf))
    return np.float32(A), np.float32(B), np.float32(C), fE


def device_d(fA, fB, fC, X, Y):
    """fma(A, Y, fma(-B, X, C)) in FP32, each step rounded once."""
    inner = rn32(-Fraction(float(fB)) * Fraction(float(X)) + Fraction(float(fC)))
    return rn32(Fraction(float(fA)) * Fraction(float(Y)) + Fraction(float(inner)))


def orient(ax, ay, bx, by, px, py):
    q = (Fraction(bx) - Fraction(ax)) * (Fraction(py) - Fraction(ay)) \
        - (Fraction(by) - Fraction(ay)) * (Fraction(px) - Fraction(ax))
    return (q > 0) - (q < 0)


def check_edge(ax, ay, bx, by, pts, xm, ym):
    fA, fB, fC, fE = edge_coeffs(ax, ay, bx, by, xm, ym)
    X = trunc_view(pts[:, 0])
    Y = trunc_view(pts[:, 1])
    decided = 0
    for k in range(len(pts)):
        d = device_d(fA, fB, fC, X[k], Y[k])
        o = orient(ax, ay, bx, by, float(pts[k, 0]), float(pts[k, 1]))
        if d > fE:
            assert o > 0, (ax, ay, bx, by, pts[k], d, fE)
            decided += 1
        elif d < -fE:
            assert o < 0, (ax, ay, bx, by, pts[k], d, fE)
            decided += 1
    return decided


@pytest.mark.parametrize("scale", [2.0 ** -90, 1e-9, 1.0, 3.7e5, 2.0 ** 40, 2.0 ** 59])
def test_filter_never_decides_the_wrong_side(scale):
    rng = np.random.default_rng(int(math.log2(scale) + 200))
    decided = total = 0
    for _ in range(12):
        # an edge between two bounding-box extremes (like E1 -> E2) and the box
        ax, ay = -scale * rng.uniform(0.5, 1.0), scale * rng.uniform(-0.5, 0.5)
        bx, by = scale * rng.uniform(-0.5, 0.5), -scale * rng.uniform(0.5, 1.0)
        xm = ym = scale
        pts = []
        # on the line through the edge (exactly, where the float64 sum is exact)
        for t in rng.uniform(0, 1, 20):
            px, py = ax + t * (bx - ax), ay + t * (by - ay)
            pts.append((px, py))
            # a few float64 ulps off the line, both ways
            for s in (-3, -1, 1, 3):
                pts.append((px + s * math.ulp(px), py - s * math.ulp(py)))
        # anywhere in the box
        pts += list(zip(rng.uniform(-scale, scale, 40), rng.uniform(-scale, scale, 40)))
        pts = np.array(pts, dtype=np.float64)
        pts = np.clip(pts, -xm, xm)
        decided += check_edge(ax, ay, bx, by, pts, xm, ym)
        total += len(pts)
    # where the products of coordinates are normal FP32 numbers the filter
    # decides most points of the box (it is not trivially silent); at 2^-90
    # they underflow and every point takes the exact test
    if scale >= 1e-9:
        assert decided > total // 4, (decided, total)


def test_view_truncates_toward_zero_and_flushes_below_the_normal_range():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 18, 2000),
                        [0.0, -0.0, 2.0 ** -126, -(2.0 ** -127), 1.0 + 2.0 ** -30]])
    v = trunc_view(x).astype(np.float64)
    big = np.abs(x) >= 2.0 ** -126
    assert np.all(np.abs(v[big]) <= np.abs(x[big]))
    assert np.all(np.abs(x[big] - v[big]) < np.abs(x[big]) * 2.0 ** -23)
    assert np.all(np.sign(v[big]) == np.sign(x[big]))
    assert np.all(v[~big] == 0)


def test_rounding_helper_matches_numpy_float32_rounding():
    rng = np.random.default_rng(4)
    for x in rng.standard_normal(3000) * 10.0 ** rng.integers(-40, 38, 3000):
        assert rn32(Fraction(float(x))) == np.float32(x)


def test_planted_loose_bound_is_caught(monkeypatch):
    """With the bound cut to a twelfth (0.5 u instead of 6 u) the filter
    decides points near the edge on the wrong side: the check has teeth."""
    monkeypatch.setattr(sys.modules[__name__], "U", U / 12)
    rng = np.random.default_rng(200)
    wrong = 0
    for _ in range(12):
        ax, ay = -rng.uniform(0.5, 1.0), rng.uniform(-0.5, 0.5)
        bx, by = rng.uniform(-0.5, 0.5), -rng.uniform(0.5, 1.0)
        fA, fB, fC, fE = edge_coeffs(ax, ay, bx, by, 1.0, 1.0)
        for t in rng.uniform(0, 1, 20):
            px, py = ax + t * (bx - ax), ay + t * (by - ay)
            for s in (0, -3, -1, 1, 3):
                qx, qy = px + s * math.ulp(px), py - s * math.ulp(py)
                d = device_d(fA, fB, fC, trunc_view(np.array([qx]))[0], trunc_view(np.array([qy]))[0])
                o = orient(ax, ay, bx, by, qx, qy)
                wrong += (d > fE and o <= 0) or (d < -fE and o >= 0)
    assert wrong > 0

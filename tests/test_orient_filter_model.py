"""CPU check of the chain hull's two FP32 orientation filters (no GPU).

The chain stage decides orient(a, b, c) of float64 points first from FP32
arithmetic: `orient_f32_filter` on the points' truncated FP32 views, then
`orient_split_filter` on split points (the view plus a float for the cleared
low significand bits); only triples neither decides go on to FP64 and the
exact expansion.  Each filter carries a derived error bound (the comments at
the functions in csrc/cch_internal.cuh).  This module restates both filters
operation by operation -- round-to-nearest and directed roundings taken from
the exact rational result -- and checks against the exact orientation of the
float64 points that a decided sign is never wrong: on collinear triples, on
triples a few float64 ulps off a line and on random triples, at magnitudes
from 2^-55 to 2^59 and spreads from the full magnitude down to a few ulps.
Shrunken bounds planted in the restatement are caught on the same inputs.
"""
from fractions import Fraction
import math

import numpy as np

F = Fraction
MU = 5.9604645e-08


def trunc_view(x):
    """f64_trunc_f32: exponent rebiased, significand truncated, a signed zero
    below 2^-126."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.int64)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(np.int64)
    t = (hi & 0x7FFFFFFF) - 0x38000000
    sign = hi & 0x80000000
    body = ((t << 3) | (lo >> 29)) & 0xFFFFFFFF
    return np.where(t < 0, sign, sign | body).astype(np.uint32).view(np.float32)


def _round32(q, mode):
    """A rational to float32: 'n' nearest-even, 'u' up, 'd' down."""
    if q == 0:
        return np.float32(0.0)
    neg = q < 0
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if F(2) ** e > a:
        e -= 1
    e = max(e, -126)
    s = a / F(2) ** (e - 23)
    m = math.floor(s)
    rem = s - m
    if mode == "n":
        if rem > F(1, 2) or (rem == F(1, 2) and m % 2 == 1):
            m += 1
    elif rem != 0 and ((mode == "u") != neg):      # away from zero when rounding outward
        m += 1
    v = math.ldexp(m, e - 23)
    if v > 3.4028234663852886e38:
        v = math.inf
    return np.float32(-v if neg else v)


def rn(q):
    return _round32(q, "n")


def ru(q):
    return _round32(q, "u")


def rd(q):
    return _round32(q, "d")


def fr(x):
    return F(float(x))


def sub_rn(a, b):
    return rn(fr(a) - fr(b))


def mul_rn(a, b):
    return rn(fr(a) * fr(b))


def add_rn(a, b):
    return rn(fr(a) + fr(b))


def fma_rn(a, b, c):
    return rn(fr(a) * fr(b) + fr(c))


def fma_ru(a, b, c):
    return ru(fr(a) * fr(b) + fr(c))


def f32_filter(A, B, C, loose=1.0):
    """orient_f32_filter on views A, B, C (pairs of float32)."""
    M = max(abs(float(v)) for v in (*A, *B, *C))
    if not (8.6736174e-19 <= M <= 1.1529215e+18):
        return 0
    u1, v1 = sub_rn(B[0], A[0]), sub_rn(B[1], A[1])
    u2, v2 = sub_rn(C[0], A[0]), sub_rn(C[1], A[1])
    U = np.float32(max(abs(float(u1)), abs(float(v1)), abs(float(u2)), abs(float(v2))))
    det = fma_rn(u1, v2, -mul_rn(v1, u2))
    mu = np.float32(MU)
    ed = add_rn(mul_rn(np.float32(2.3841870e-07 * loose), np.float32(M)),
                add_rn(np.float32(4.7020e-38), mul_rn(np.float32(6.0200692e-08), U)))
    e0 = add_rn(add_rn(mul_rn(np.float32(4.0), mul_rn(ed, U)), mul_rn(np.float32(2.0), mul_rn(ed, ed))),
                add_rn(mul_rn(mu, mul_rn(U, U)), np.float32(5.6e-45)))
    lhs = mul_rn(np.float32(abs(float(det))), np.float32(0.99999988))
    if float(lhs) > float(mul_rn(np.float32(1.01), e0)):
        return 1 if float(det) > 0 else -1
    return 0


def split(x):
    """f64_split: (view, float of the cleared 29 low bits), or NaN outside
    2^-60 .. 2^60."""
    x = float(x)
    b = int(np.array([x]).view(np.uint64)[0])
    if (b << 1) & ((1 << 64) - 1) == 0:
        return np.float32(0.0), np.float32(0.0)
    e = (b >> 52) & 0x7FF
    if e < 1023 - 60 or e > 1023 + 60:
        return np.float32(np.nan), np.float32(0.0)
    lo = np.float32(b & 0x1FFFFFFF) * np.float32(2.0 ** (e - 1075))
    h = trunc_view(np.array([x]))[0]
    return h, (-lo if x < 0 else lo)


def split_filter(A, B, C, loose=1.0):
    """orient_split_filter on split points (hx, hy, lx, ly)."""
    mu = np.float32(MU)
    if any(math.isnan(float(v)) for v in (*A, *B, *C)):
        return 0          # a NaN view (|x| outside 2^-60 .. 2^60) makes det NaN: undecided
    M = max(abs(float(v)) for v in (A[0], A[1], B[0], B[1], C[0], C[1]))
    c0 = fma_ru(np.float32(1.4210859e-14 * loose), np.float32(M), np.float32(4.3e-45))

    def diff(P, Q, i):
        dh, dl = sub_rn(P[i], Q[i]), sub_rn(P[i + 2], Q[i + 2])
        D = add_rn(dh, dl)
        s = ru(fr(ru(fr(abs(float(dh))) + fr(abs(float(dl))))) + fr(abs(float(D))))
        return D, fma_ru(mu, s, c0)

    U1, e1 = diff(B, A, 0)
    V1, e2 = diff(B, A, 1)
    U2, e3 = diff(C, A, 0)
    V2, e4 = diff(C, A, 1)
    p = mul_rn(V1, U2)
    det = fma_rn(U1, V2, -p)
    E = ru(fr(e1) * fr(abs(float(V2))))
    E = fma_ru(e4, np.float32(abs(float(U1))), E)
    E = fma_ru(e1, e4, E)
    E = fma_ru(e2, np.float32(abs(float(U2))), E)
    E = fma_ru(e3, np.float32(abs(float(V1))), E)
    E = fma_ru(e2, e3, E)
    E = fma_ru(mu, ru(fr(abs(float(p))) + fr(abs(float(det)))), E)
    E = fma_ru(np.float32(1.01), E, np.float32(1.5e-44))
    if float(rd(fr(abs(float(det))) * fr(np.float32(0.99999988)))) > float(E):
        return 1 if float(det) > 0 else -1
    return 0


def orient(a, b, c):
    q = (F(b[0]) - F(a[0])) * (F(c[1]) - F(a[1])) - (F(b[1]) - F(a[1])) * (F(c[0]) - F(a[0]))
    return (q > 0) - (q < 0)


def triples(rng, scale, spread, count):
    """Collinear, nearly collinear and random triples around a point of the
    given magnitude, spread over the given width."""
    out = []
    for _ in range(count):
        cx, cy = scale * rng.uniform(0.5, 1.0), scale * rng.uniform(-1.0, 1.0)
        dx, dy = spread * rng.uniform(-1, 1), spread * rng.uniform(-1, 1)
        a = (cx, cy)
        b = (cx + dx, cy + dy)
        t = rng.uniform(-2, 2)
        c = (cx + t * dx, cy + t * dy)
        out.append((a, b, c))
        for s in (-2, -1, 1, 2):
            out.append((a, b, (c[0] + s * math.ulp(c[0]), c[1] - s * math.ulp(c[1]))))
        out.append((a, b, (cx + spread * rng.uniform(-1, 1), cy + spread * rng.uniform(-1, 1))))
    return out


CASES = [(s, w) for s in (2.0 ** -55, 1e-9, 1.0, 3.7e5, 2.0 ** 40, 2.0 ** 59) for w in (1.0, 1e-6, 1e-12)]


def run_filters(loose_view=1.0, loose_split=1.0):
    wrong_view = wrong_split = decided_view = decided_split = 0
    rng = np.random.default_rng(9)
    for scale, rel in CASES:
        for a, b, c in triples(rng, scale, scale * rel, 10):
            o = orient(a, b, c)
            V = [trunc_view(np.array(p)) for p in (a, b, c)]
            f = f32_filter(*V, loose=loose_view)
            if f:
                decided_view += 1
                wrong_view += f != o
            S = [(*(lambda hx, lx, hy, ly: (hx, hy, lx, ly))(*split(p[0]), *split(p[1])),) for p in (a, b, c)]
            g = split_filter(*S, loose=loose_split)
            if g:
                decided_split += 1
                wrong_split += g != o
    return wrong_view, wrong_split, decided_view, decided_split


def test_orientation_filters_never_decide_a_wrong_sign():
    wv, ws, dv, ds = run_filters()
    assert wv == 0 and ws == 0, (wv, ws)
    # both filters decide a good share of these triples (neither is silent)
    assert dv > 40 and ds > 100, (dv, ds)


def test_planted_shrunken_bounds_are_caught():
    wv, ws, _, _ = run_filters(loose_view=1e-3, loose_split=1e-3)
    assert wv > 0 and ws > 0, (wv, ws)


def test_directed_roundings_bracket_the_value():
    rng = np.random.default_rng(2)
    for x in rng.standard_normal(2000) * 10.0 ** rng.integers(-40, 36, 2000):
        q = F(float(x)) * F(3, 7)
        lo, hi = rd(q), ru(q)
        assert F(float(lo)) <= q <= F(float(hi))
        assert lo == hi or np.nextafter(lo, np.float32(np.inf)) == hi
        assert rn(F(float(x))) == np.float32(x)

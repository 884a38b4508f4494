"""CPU checks of the numeric facts the kernels rely on (no GPU).

These restate, in numpy, two bit-level maps the CUDA code uses and check
them against IEEE 754 arithmetic, so that the reasoning behind the kernels is
pinned independently of the kernels themselves (which the GPU tests check
end to end against the oracle):

* a1's float64 filter reads the top 32 bits of a coordinate as an FP32
  number: that reading must be non-decreasing in the coordinate wherever it
  is not NaN (+-Inf included), equal for -0.0 and +0.0, and NaN or +-Inf only
  for values the domain check rejects at the top (|c| >= 2^1017, Inf, NaN);
  the warp's integer key bound maps back to those bits exactly;
* cch_hull_f32soa widens float32 to float64 from the IEEE bit fields;
* a1 reduces its lexicographic keys across a warp one 32-bit word at a time
  (the minimum of each word over the lanes still tied on the earlier ones);
* the sort and SPA keys preserve the order of the coordinates (-0.0 and
  +0.0 equal), and a2's three-operation FP32 view equals the truncated view
  for every magnitude in [2^-126, 2^60].
"""
import numpy as np


def top_reading(d):
    """The top 32 bits of float64 values read as float32."""
    bits = np.asarray(d, dtype=np.float64).view(np.uint64)
    return (bits >> np.uint64(32)).astype(np.uint32).view(np.float32)


def key_hi(d):
    """Order-preserving key of the top word (-0.0 made +0.0), as a1 builds it."""
    bits = np.asarray(d, dtype=np.float64).view(np.uint64)
    h = (bits >> np.uint64(32)).astype(np.uint32)
    lo = (bits & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    nz = ((h & np.uint32(0x7FFFFFFF)) | lo) != 0
    h = np.where(nz, h, np.uint32(0))
    m = np.where(h >> np.uint32(31) == 1, np.uint32(0xFFFFFFFF), np.uint32(0))
    return h ^ (m | np.uint32(0x80000000))


def bound_bits(k):
    """a1_bound_f: a key's top word back to raw bits."""
    k = np.asarray(k, dtype=np.uint32)
    return np.where(k & np.uint32(0x80000000) != 0, k ^ np.uint32(0x80000000), ~k)


def sample_doubles(rng, n):
    e = rng.integers(-1074, 1024, n).astype(np.float64)
    v = rng.random(n) * np.exp2(e)
    v *= np.where(rng.random(n) < 0.5, -1.0, 1.0)
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 2.0 ** -400, -(2.0 ** -400), 2.0 ** 400, 2.0 ** 1016,
                        2.0 ** 1017, -(2.0 ** 1017), np.finfo(np.float64).max, np.inf, -np.inf, 1.0, -1.0])
    return np.concatenate([v, special])


def test_top_word_reading_is_monotone_and_non_finite_only_out_of_domain():
    rng = np.random.default_rng(41)
    d = sample_doubles(rng, 200_000)
    d = d[~np.isnan(d)]
    d = np.sort(d)
    t = top_reading(d)
    biased = (d.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)
    out = biased >= 2040                             # |c| >= 2^1017, Inf
    assert np.array_equal(~np.isfinite(t), out)      # NaN or +-Inf exactly there
    assert not np.isnan(t[~out]).any()
    ok = ~np.isnan(t)
    tt = t[ok]
    assert np.all(tt[1:] >= tt[:-1])                 # non-decreasing in the coordinate
    assert top_reading(-0.0) == top_reading(0.0)
    # the largest in-domain magnitude reads below every out-of-domain one
    assert top_reading(np.nextafter(2.0 ** 400, 0)) < top_reading(2.0 ** 1017)


def test_key_bound_maps_back_to_the_top_bits():
    rng = np.random.default_rng(43)
    d = sample_doubles(rng, 100_000)
    d = d[~np.isnan(d) & (d != 0)]                   # -0.0 is normalised by the key, checked below
    k = key_hi(d)
    raw = (d.view(np.uint64) >> np.uint64(32)).astype(np.uint32)
    assert np.array_equal(bound_bits(k), raw)
    # the complemented (maximum) bound: the kernel stores ~key and maps ~(~key)
    assert np.array_equal(bound_bits(~(~k)), raw)
    # -0.0 and +0.0 share a key; its bits read as +0.0, which compares equal to -0.0
    assert key_hi(-0.0) == key_hi(0.0)
    assert bound_bits(key_hi(-0.0)).view(np.float32) == np.float32(0.0)
    # ordering: key order equals value order, so a point whose top word reads at
    # or below the bound's reading has key <= the bound's key or ties it
    a, b = np.sort(rng.choice(d, 2, replace=False))
    assert key_hi(a) <= key_hi(b)


def test_the_no_extreme_bound_lets_everything_through():
    # no extreme yet: the running minimum key is all ones, its bits read as NaN
    assert np.isnan(bound_bits(np.uint32(0xFFFFFFFF)).view(np.float32))
    assert np.isnan(bound_bits(~np.uint32(0xFFFFFFFF)).view(np.float32))


def widen(u):
    """cch_hull_f32soa's widening, from the float32 bit fields."""
    sign = (u >> 31) << 63
    e = (u >> 23) & 0xFF
    m = u & 0x7FFFFF
    if e == 0xFF:
        return sign | (0x7FF << 52) | (m << 29)
    if e != 0:
        return sign | ((e + 896) << 52) | (m << 29)
    if m == 0:
        return sign
    p = m.bit_length() - 1
    return sign | ((p + 874) << 52) | ((m << (52 - p)) & ((1 << 52) - 1))


def test_widening_matches_ieee_conversion():
    rng = np.random.default_rng(47)
    u = np.concatenate([rng.integers(0, 2 ** 32, 50_000, dtype=np.uint64).astype(np.uint32),
                        np.arange(0, 3000, dtype=np.uint32), np.arange(0x80000000, 0x80000800, dtype=np.uint32),
                        np.array([0x7F800000, 0xFF800000, 0x007FFFFF, 0x00800000, 0x807FFFFF, 0x7F7FFFFF,
                                  0x7FC00000, 0xFFC00001], dtype=np.uint32)])
    f = u.view(np.float32)
    with np.errstate(invalid="ignore"):
        ref = f.astype(np.float64)
    for x, r in zip(u.tolist(), ref.tolist()):
        w = np.uint64(widen(x)).view(np.float64)
        if np.isnan(r):
            assert np.isnan(w)
        else:
            assert w == r and np.signbit(w) == np.signbit(r), hex(x)


# ---------------------------------------------------------------------------
# a1's warp minima: one redux.sync minimum per 32-bit word, each over the
# lanes still tied on the earlier words, must give the lexicographic minimum
# of (k1, k2, idx) -- ties, all-ones words and all-tied warps included.

def warp_lex_min(k1, k2, idx):
    """The word-by-word reduction of one warp (32 lanes), as lex_warp_min does."""
    words = [k1 >> np.uint64(32), k1 & np.uint64(0xFFFFFFFF), k2 >> np.uint64(32), k2 & np.uint64(0xFFFFFFFF),
             idx.astype(np.uint64)]
    tied = np.ones(32, bool)
    out = []
    for wd in words:
        m = np.where(tied, wd, np.uint64(0xFFFFFFFF)).min()
        tied &= wd == m
        out.append(int(m))
    return (out[0] << 32 | out[1], out[2] << 32 | out[3], out[4])


def test_word_by_word_warp_minimum_is_the_lexicographic_minimum():
    rng = np.random.default_rng(5)
    for t in range(3000):
        # few distinct words so that ties reach every level
        pool = np.array([0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF], dtype=np.uint64)
        w = pool[rng.integers(0, len(pool) if t % 3 else 2, size=(32, 4))]
        k1 = (w[:, 0] << np.uint64(32)) | w[:, 1]
        k2 = (w[:, 2] << np.uint64(32)) | w[:, 3]
        idx = pool[rng.integers(0, len(pool), size=32)].astype(np.uint32)
        want = min(zip(k1.tolist(), k2.tolist(), idx.tolist()))
        assert warp_lex_min(k1, k2, idx) == want


def test_word_by_word_warp_minimum_of_64_bit_keys():
    rng = np.random.default_rng(6)
    for _ in range(2000):
        v = rng.integers(0, 4, size=32).astype(np.uint64) << np.uint64(32) | rng.integers(0, 3, size=32).astype(np.uint64)
        hi = (v >> np.uint64(32)).min()
        lo = np.where((v >> np.uint64(32)) == hi, v & np.uint64(0xFFFFFFFF), np.uint64(0xFFFFFFFF)).min()
        assert int(hi) << 32 | int(lo) == int(v.min())


# ---------------------------------------------------------------------------
# Order-preserving keys of the sort and SPA stages, and a2's three-operation
# FP32 view of sets whose coordinates all have magnitude in [2^-126, 2^60].

def key_f64(x):
    """key_f64 on the float64 bits: -0.0 made +0.0, then the sign-magnitude
    to unsigned order map."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64).copy()
    b[b == np.uint64(0x8000000000000000)] = np.uint64(0)
    neg = (b >> np.uint64(63)) != 0
    return np.where(neg, ~b, b | np.uint64(0x8000000000000000))


def key_i32(v):
    return (np.asarray(v, dtype=np.int32).view(np.uint32) ^ np.uint32(0x80000000)).astype(np.uint64)


def test_float64_and_int32_keys_preserve_order_and_equality():
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.integers(-300, 300, 3000),
                        [0.0, -0.0, 5e-324, -5e-324, np.inf, -np.inf, 1.0, np.nextafter(1.0, 2.0)]])
    k = key_f64(x)
    i, j = rng.integers(0, len(x), 20000), rng.integers(0, len(x), 20000)
    assert np.array_equal(k[i] < k[j], x[i] < x[j])
    assert np.array_equal(k[i] == k[j], x[i] == x[j])
    v = np.concatenate([rng.integers(-2 ** 31, 2 ** 31, 3000), [-2 ** 31, -1, 0, 1, 2 ** 31 - 1]]).astype(np.int64)
    kv = key_i32(v)
    i, j = rng.integers(0, len(v), 20000), rng.integers(0, len(v), 20000)
    assert np.array_equal(kv[i] < kv[j], v[i] < v[j])
    # the descending regions complement the key: the order reverses
    assert np.array_equal(~k[i] < ~k[j], x[i] > x[j])


def view_short(x):
    """f64_view_short: the top word rebiased by subtraction on the signed word
    and funnel-shifted with the low word's three leading bits, sign put back."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.uint64)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(np.uint64)
    t = (hi - np.uint64(0x38000000)) & np.uint64(0xFFFFFFFF)
    shifted = ((t << np.uint64(3)) | (lo >> np.uint64(29))) & np.uint64(0xFFFFFFFF)
    return (shifted | (hi & np.uint64(0x80000000))).astype(np.uint32).view(np.float32)


def test_short_view_equals_the_truncated_view_in_its_domain():
    rng = np.random.default_rng(12)
    mag = 2.0 ** rng.uniform(-126, 60, 20000)
    x = np.where(rng.integers(0, 2, 20000) == 1, -mag, mag)
    x = np.concatenate([x, [2.0 ** -126, -(2.0 ** -126), np.nextafter(2.0 ** 60, 0), -np.nextafter(2.0 ** 60, 0)]])
    # f64_trunc_f32: exponent rebiased on the magnitude, significand truncated
    b = x.view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.int64)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(np.int64)
    t = (hi & 0x7FFFFFFF) - 0x38000000
    full = np.where(t < 0, hi & 0x80000000, (hi & 0x80000000) | (((t << 3) | (lo >> 29)) & 0xFFFFFFFF))
    assert np.array_equal(view_short(x).view(np.uint32), full.astype(np.uint32))

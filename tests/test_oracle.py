"""Pins for the CPU oracle (no GPU): the oracle is checked against things
other than itself -- exact rational brute force, closed forms, invariants and
the worked example of Fig. 4 -- so that a dropped term, a flipped sign or a
swapped operand in it fails here before the GPU path is compared with it."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import bruteforce as bf
from paper_1508_05488_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------- predicates

def _near_collinear_f64(rng, m):
    """Triples whose third point is a rounded point of the line through the
    first two: the exact orientation is tiny and often of either sign."""
    out = []
    for _ in range(m):
        scale = 2.0 ** int(rng.integers(-30, 30))
        a = rng.standard_normal(2) * scale
        b = rng.standard_normal(2) * scale
        t = rng.standard_normal() * 3
        c = a + t * (b - a)
        if rng.random() < 0.3:
            c = c + np.nextafter(0, 1) * 0 + rng.choice([-1, 1]) * np.spacing(c) * rng.integers(0, 3)
        out.append((a, b, c))
    return out


def test_orient_f64_matches_exact_rationals():
    rng = np.random.default_rng(11)
    cases = _near_collinear_f64(rng, 3000)
    for _ in range(1000):
        cases.append(tuple(rng.standard_normal(2) * 10.0 ** rng.integers(-5, 5) for _ in range(3)))
    # exact collinear dyadic triples and repeated points
    for _ in range(500):
        a = rng.integers(-1000, 1000, 2) / 64.0
        d = rng.integers(-50, 50, 2) / 64.0
        cases.append((a, a + d, a + rng.integers(-5, 6) * d))
        cases.append((a, a, a + d))
    naive_wrong = 0
    for a, b, c in cases:
        want = bf.orient(a, b, c)
        got = oracle.orient(a, b, c)
        assert got == want, (a, b, c, got, want)
        naive = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
        naive_wrong += int(np.sign(naive)) != want
    # the case set must be able to catch an inexact predicate
    assert naive_wrong > 50


def test_orient_f64_extreme_magnitudes():
    rng = np.random.default_rng(12)
    for _ in range(500):
        e = int(rng.integers(-395, 395))
        a, b = rng.standard_normal(2) * 2.0 ** e, rng.standard_normal(2) * 2.0 ** e
        c = a + rng.standard_normal() * (b - a)
        assert oracle.orient(a, b, c) == bf.orient(a, b, c)


def test_orient_i32_full_range():
    rng = np.random.default_rng(13)
    lo, hi = -2 ** 31, 2 ** 31
    for _ in range(3000):
        p = rng.integers(lo, hi, size=6, dtype=np.int64)
        a, b, c = p[0:2], p[2:4], p[4:6]
        if rng.random() < 0.3:  # force collinear with a huge span
            c = a
        want = bf.orient(a.tolist(), b.tolist(), c.tolist())
        assert oracle.orient(a, b, c, np.int32) == want
    # int64 overflow territory: differences of 2^32 - 1
    a, b, c = (lo, lo), (hi - 1, hi - 1), (lo, hi - 1)
    assert oracle.orient(a, b, c, np.int32) == 1
    assert oracle.orient(b, a, c, np.int32) == -1


# --------------------------------------------------------------- the hull

@pytest.mark.parametrize("seed", range(160))
def test_hull_matches_bruteforce(seed):
    p = inputs.small_cases(seed)
    assert oracle.hull(p).tolist() == bf.hull(p)


def test_hull_empty_single_identical():
    assert oracle.hull(np.zeros((0, 2))).tolist() == []
    assert oracle.hull(np.array([[3, 4]], np.int32)).tolist() == [0]
    p = np.tile(np.array([[1.5, -2.0]]), (7, 1))
    assert oracle.hull(p).tolist() == [0]
    # -0.0 and +0.0 are the same coordinate
    q = np.array([[0.0, 1.0], [-0.0, 1.0], [0.0, -0.0]])
    assert oracle.hull(q).tolist() == [2, 0]


def test_hull_collinear_returns_two_extremes():
    t = np.arange(50)
    rng = np.random.default_rng(3)
    for d in [(1, 2), (1, -3), (0, 1), (1, 0)]:
        p = np.stack([5 + d[0] * t, 7 + d[1] * t], 1).astype(np.int32)
        perm = rng.permutation(50)
        q = p[perm]
        h = oracle.hull(q).tolist()
        lo = int(np.argmin(perm)) if d[0] > 0 or (d[0] == 0 and d[1] > 0) else int(np.argmax(perm))
        assert len(h) == 2
        assert sorted(map(tuple, q[h].tolist())) == sorted([tuple(p[0]), tuple(p[-1])])
        assert tuple(q[h[0]]) == min(map(tuple, q.tolist()))
        del lo


def test_hull_regular_polygon_keeps_every_vertex():
    rng = np.random.default_rng(5)
    for n in [3, 4, 7, 100, 1000, 20_000]:
        t = rng.random() + 2 * np.pi * np.arange(n) / n
        p = np.stack([np.cos(t), np.sin(t)], 1) * 3.0
        perm = rng.permutation(n)
        h = oracle.hull(p[perm])
        assert len(h) == n
        # CCW from the lexicographic minimum: angles increase cyclically
        ang = np.unwrap(np.arctan2(p[perm][h][:, 1], p[perm][h][:, 0]))
        assert np.all(np.diff(ang) > 0)


def test_hull_grid_gives_four_corners():
    for k in [2, 3, 10, 41]:
        g = np.stack(np.meshgrid(np.arange(k), np.arange(k)), -1).reshape(-1, 2).astype(np.int32)
        g = g[np.random.default_rng(k).permutation(len(g))]
        h = oracle.hull(g)
        assert sorted(map(tuple, g[h].tolist())) == [(0, 0), (0, k - 1), (k - 1, 0), (k - 1, k - 1)]
        assert tuple(g[h[0]]) == (0, 0) and tuple(g[h[1]]) == (k - 1, 0)


def test_hull_parabola_all_vertices_and_square_plus_interior():
    i = np.arange(-300, 301)
    p = np.stack([i, i * i], 1).astype(np.int32)
    assert len(oracle.hull(p)) == len(i)
    q = np.concatenate([np.array([[0, 0], [10, 0], [10, 10], [0, 10]]),
                        np.random.default_rng(2).integers(1, 10, (500, 2)),
                        np.array([[5, 0], [10, 5], [0, 5], [5, 10]])]).astype(np.int32)
    assert oracle.hull(q).tolist() == [0, 1, 2, 3]


def test_hull_circle_config_is_all_extreme():
    p = inputs.circle_f64(200_000, seed=6)
    assert len(oracle.hull(p)) == 200_000


def _exact_inside_all(p, h):
    """Every point is on the closed inner side of every hull edge (exact)."""
    hv = p[h]
    m = len(h)
    is_int = p.dtype == np.int32
    for k in range(m):
        a, b = hv[k], hv[(k + 1) % m]
        if is_int:
            a64, b64, p64 = a.astype(object), b.astype(object), p.astype(object)
            d = (b64[0] - a64[0]) * (p64[:, 1] - a64[1]) - (b64[1] - a64[1]) * (p64[:, 0] - a64[0])
            assert all(v >= 0 for v in d)
        else:
            d = (b[0] - a[0]) * (p[:, 1] - a[1]) - (b[1] - a[1]) * (p[:, 0] - a[0])
            scale = (abs(b[0] - a[0]) + abs(b[1] - a[1])) * (np.abs(p).max() + np.abs(a).max()) * 1e-12
            close = np.nonzero(d < scale)[0]
            for i in close:
                assert bf.orient(a, b, p[i]) >= 0


@pytest.mark.parametrize("kind", ["i32", "square", "disk", "gauss"])
def test_hull_invariants_medium(kind):
    n = 30_000
    p = {"i32": lambda: inputs.square_i32(n, 9),
         "square": lambda: inputs.square_f64(n, 9),
         "disk": lambda: inputs.disk_f64(n, 9),
         "gauss": lambda: inputs.gauss_f64(n, 9)}[kind]()
    h = oracle.hull(p)
    m = len(h)
    assert m >= 3 and len(set(h.tolist())) == m
    assert tuple(p[h[0]]) == min(map(tuple, p.tolist()))
    for k in range(m):  # strictly convex, counter-clockwise
        assert bf.orient(p[h[k]], p[h[(k + 1) % m]], p[h[(k + 2) % m]]) > 0
    _exact_inside_all(p, h)
    # each vertex is the smallest index of its coordinates
    first = {}
    for i, q in enumerate(map(tuple, p.tolist())):
        first.setdefault(q, i)
    assert all(first[tuple(p[i])] == i for i in h)


# ------------------------------------------------------------- the method

@pytest.mark.parametrize("seed", range(120))
def test_method_stages_match_bruteforce(seed):
    p = inputs.small_cases(seed)
    m = oracle.method(p)
    ext = bf.extremes(p)
    assert m["ext"].tolist() == ext
    reg = bf.regions(p, ext)
    assert m["region"].tolist() == reg
    for k in range(4):
        members = [i for i, r in enumerate(reg) if r == k + 1]
        assert m["r1"][k].tolist() == members                # index order
        assert sorted(m["sorted"][k].tolist()) == members    # a permutation
    spa = bf.spa_survivors(p, ext, reg)
    for k in range(4):
        assert set(m["spa"][k].tolist()) == spa[k]
    assert m["hull"].tolist() == bf.hull(p)


def _table1_key(p, k, i):
    x, y = p[i]
    return [(x, i), (y, i), (-x, i), (-y, i)][k]


@pytest.mark.parametrize("kind", ["i32", "square", "disk", "gauss", "degenerate"])
def test_method_medium(kind):
    n = 20_000
    p = {"i32": lambda: inputs.square_i32(n, 21),
         "square": lambda: inputs.square_f64(n, 21),
         "disk": lambda: inputs.disk_f64(n, 21),
         "gauss": lambda: inputs.gauss_f64(n, 21),
         "degenerate": lambda: inputs.degenerate_f64(n, 21)}[kind]()
    m = oracle.method(p)
    h = oracle.hull(p)
    assert m["hull"].tolist() == h.tolist()
    pl = p.tolist()
    for k in range(4):
        s = m["sorted"][k].tolist()
        keys = [_table1_key(pl, k, i) for i in s]
        assert keys == sorted(keys)                           # Table 1 order, stable
        sp = m["spa"][k].tolist()
        pos = {i: j for j, i in enumerate(s)}
        assert [pos[i] for i in sp] == sorted(pos[i] for i in sp)  # subsequence
    # every hull vertex is an extreme or survives both rounds (Sec. 4.2)
    kept = set(m["ext"].tolist()).union(*[set(a.tolist()) for a in m["spa"]])
    assert set(h.tolist()) <= kept
    # every R0 point is inside or on the quadrilateral (exact)
    E = [pl[i] for i in m["ext"]] + [pl[m["ext"][0]]]
    r0 = np.nonzero(m["region"] == 0)[0]
    rng = np.random.default_rng(0)
    for i in rng.choice(r0, size=min(300, len(r0)), replace=False):
        assert all(bf.orient(E[k], E[k + 1], pl[i]) >= 0 for k in range(4))


def test_fig4_worked_example():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "fig4_r3_chain.txt"))
            if ln.strip() and not ln.startswith("#")]
    labels = [r[0] for r in rows]
    p = np.array([[int(r[1]), int(r[2])] for r in rows], dtype=np.int32)
    m = oracle.method(p)
    lab = lambda idxs: [labels[i] for i in idxs]
    assert lab(m["ext"]) == ["E1", "E2", "E3", "E4"]
    assert lab(m["sorted"][2]) == ["P1", "P2", "P3", "P4", "P5", "P6", "P7"]
    kept = {r[0] for r in rows if r[3] == "1"}
    assert set(lab(m["spa"][2])) == kept
    assert lab(m["spa"][2]) == ["P1", "P2", "P5", "P6"]
    assert all(len(m["r1"][k]) == 0 for k in (0, 1, 3))


def test_blocked_spa_of_the_paper_is_a_superset():
    """Sec. 2.2.2 runs SPA in independent chunks, each restarting t at its
    chunk's first point; that keeps every point the sequential rule keeps
    (the sequential rule also has every earlier chunk's points and the first
    extreme to discard against)."""
    p = inputs.disk_f64(50_000, 31)
    m = oracle.method(p)
    blocked = oracle.blocked_spa(p, m=m)
    for k in range(4):
        assert set(m["spa"][k].tolist()) <= set(blocked[k].tolist())
        assert len(blocked[k]) < len(m["sorted"][k])        # 1024 chunks of ~10 points still discard


def _blocked_by_dominance(p, sorted_k, k, nchunks):
    """Brute-force definition of the chunked rule: a point is kept iff no
    earlier point of its chunk has a strictly better compared coordinate
    (Fig. 2 / Fig. 3: R1 smaller y, R2 larger x, R3 larger y, R4 smaller x)."""
    c = 1 if k in (0, 2) else 0
    better = (lambda q, r: q < r) if k in (0, 3) else (lambda q, r: q > r)
    n = len(sorted_k)
    L = (n + nchunks - 1) // nchunks if n else 1
    keep = []
    for pos, i in enumerate(sorted_k):
        lo = pos // L * L
        if not any(better(p[sorted_k[e]][c], p[i][c]) for e in range(lo, pos)):
            keep.append(int(i))
    return keep


@pytest.mark.parametrize("seed", range(12))
def test_blocked_spa_equals_its_dominance_definition(seed):
    """The oracle's chunked running minimum equals the pairwise definition on
    small sets with duplicates, ties and negative zeros, for several chunk
    counts (one chunk, a few, one point per chunk)."""
    rng = np.random.default_rng(900 + seed)
    if seed % 3 == 0:
        p = rng.integers(-6, 7, (300, 2)).astype(np.int32)
    elif seed % 3 == 1:
        p = (rng.integers(-8, 9, (300, 2)) / 4.0).astype(np.float64)
        p[rng.random(300) < 0.1] *= -0.0                      # zeros of both signs among them
    else:
        p = inputs.disk_f64(400, 900 + seed)
    m = oracle.method(p)
    pl = p.tolist()
    for nchunks in (1, 3, 7, 1024):
        got = oracle.blocked_spa(p, nchunks=nchunks, m=m)
        for k in range(4):
            assert got[k].tolist() == _blocked_by_dominance(pl, m["sorted"][k].tolist(), k, nchunks), (nchunks, k)


def test_blocked_spa_closed_forms():
    """With at least as many chunks as points every region point is its own
    chunk and is kept; the hull of the extremes and the kept points is the
    hull of the set."""
    p = inputs.square_f64(3000, 32)
    m = oracle.method(p)
    allk = oracle.blocked_spa(p, nchunks=10 ** 6, m=m)
    for k in range(4):
        assert np.array_equal(allk[k], m["sorted"][k])
    for nchunks in (1, 5, 1024):
        b = oracle.blocked_spa(p, nchunks=nchunks, m=m)
        keep = np.unique(np.concatenate([m["ext"]] + b))
        sub = oracle.hull(p[keep])
        assert np.array_equal(np.sort(keep[sub]), np.sort(oracle.hull(p)))


# ------------------------------------------------ octagon round 1

@pytest.mark.parametrize("seed", range(8))
def test_diag_extremes_by_exact_scores(seed):
    """On coordinates whose FP32 views and scores are exact (small integers,
    coarse dyadic grids), the diagonal extremes are the exact minimisers of
    x+y, y-x, -x-y, x-y with the smallest index on ties."""
    rng = np.random.default_rng(700 + seed)
    if seed % 2:
        p = rng.integers(-50, 51, (400, 2)).astype(np.int32)
    else:
        p = (rng.integers(-400, 401, (400, 2)) / 16.0).astype(np.float64)
    pl = [(Fraction(float(x)), Fraction(float(y))) for x, y in p.tolist()]
    fs = [lambda q: q[0] + q[1], lambda q: q[1] - q[0], lambda q: -q[0] - q[1], lambda q: q[0] - q[1]]
    want = [min(range(len(pl)), key=lambda i: (f(pl[i]), i)) for f in fs]
    assert oracle.diag_extremes(p).tolist() == want


def _strictly_inside_hull(verts_pts, q):
    """q strictly inside the convex hull of verts_pts (exact rationals)."""
    h = bf.hull(verts_pts)
    if len(h) < 3:
        return False
    P = [verts_pts[i] for i in h]
    return all(bf.orient(P[k], P[(k + 1) % len(P)], q) > 0 for k in range(len(P)))


@pytest.mark.parametrize("seed", range(10))
def test_octagon_round1_against_brute_force(seed):
    """A point is discarded by the octagon round 1 iff it is strictly inside
    the convex hull of the eight vertices; every used D_r lies strictly
    outside its quadrilateral edge; and the SPA survivors of the reduced
    regions, computed by dominance, are the paper's survivors outside the
    octagon (the octagon's interior never beats a point outside it)."""
    rng = np.random.default_rng(800 + seed)
    kind = seed % 3
    if kind == 0:
        p = inputs.disk_f64(300, 800 + seed)
    elif kind == 1:
        p = rng.integers(-12, 13, (300, 2)).astype(np.int32)
    else:
        p = (rng.integers(-40, 41, (300, 2)) / 8.0).astype(np.float64)
    m = oracle.method(p)
    diag = oracle.octagon_diag(p, m)
    ext = [int(i) for i in m["ext"]]
    pl = p.tolist()
    for r in range(4):
        if diag[r] >= 0:
            assert bf.orient(pl[ext[r]], pl[ext[(r + 1) % 4]], pl[int(diag[r])]) < 0
    o = oracle.octagon_round1(p, diag, m)
    vpts = [pl[i] for i in o["verts"]]
    region = bf.regions(p, ext)
    red = list(region)
    for i in range(len(pl)):
        ins = _strictly_inside_hull(vpts, pl[i])
        if region[i]:
            assert (i not in set(o["r1"][region[i] - 1].tolist())) == ins, i
        if ins:
            red[i] = 0
    spa = bf.spa_survivors(p, ext, red)
    for k in range(4):
        assert set(o["spa"][k].tolist()) == spa[k]
        assert set(o["spa"][k].tolist()) == {i for i in m["spa"][k].tolist() if red[i]}


# ------------------------------------------------ multi-core CPU baseline

@pytest.mark.skipif(not oracle.parallel_available(), reason="gcc without OpenMP")
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_parallel_baseline_equals_oracle(threads):
    """The benchmark's multi-core CPU baseline (octagon filter, parallel merge
    sort, Andrew's chain) returns exactly the oracle's hull."""
    rng = np.random.default_rng(31)
    t = rng.random(3000)
    cases = [inputs.square_f64(60_000, 1), inputs.disk_f64(70_001, 2), inputs.gauss_f64(50_000, 3),
             inputs.square_i32(40_000, 4), inputs.degenerate_f64(50_000, 9), inputs.circle_f64(5_000, 6),
             np.zeros((0, 2)), np.ones((5, 2)), np.array([[1.0, 2.0]]), np.array([[1.0, 2.0], [1.0, 2.0]]),
             np.array([[0.0, 0.0], [1.0, 1.0], [2.0, 2.0], [0.5, 0.5]]),
             rng.integers(0, 3, (1000, 2)).astype(np.int32), rng.integers(-5, 5, (5000, 2)).astype(np.float64),
             np.array([[0, 0], [2, 0], [2, 2], [0, 2], [1, 1], [0, 0], [2, 2]], dtype=np.int32),
             np.stack([t, 0.5 * t + 1e-17 * rng.standard_normal(3000)], 1)]
    for p in cases:
        assert np.array_equal(oracle.parallel_hull(p, threads), oracle.hull(p)), p.shape

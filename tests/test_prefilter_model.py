"""CPU model of the dominance table (no GPU): whatever subset of sample points
reaches the table, the points it drops are never SPA survivors.

The prefilter reads the SPA rule of Sec. 2.2.1 (Fig. 2) as a dominance test:
a point P of region R_r that some point Q precedes strictly in the region's
sort coordinate (Table 1) and beats strictly in the compared coordinate is
discarded by SPA, and such a Q always lies in R_r itself.  The device table
holds, per bucket of a monotone map of the sort coordinate, the best compared
word of some sample points; each bucket then takes the exclusive prefix
minimum over the lower buckets, seeded with E_r (the region's first point).
k_stairs does not put every sample point in: each CTA keeps only the
staircase steps of its own chunk on the chunk's own coarser map (the best
point per local bucket, then the buckets that beat every lower one).  This
model restates that construction in numpy -- FP32 views, order words, bucket
maps, steps, merge, prefix -- and checks it against `oracle.method`: no
point the table (or the dominance box) drops is an SPA survivor, for several
chunk sizes and local bucket counts.  A planted mistake (an inclusive prefix,
so that a point's own bucket counts) must be caught on the same inputs.
"""
import numpy as np
import pytest

import oracle
from paper_1508_05488_gb300 import inputs

NB = 1024      # buckets per region of the final table


def views(p):
    """FP32 views: any map that is non-decreasing in the coordinate will do."""
    return np.asarray(p[:, 0], dtype=np.float32), np.asarray(p[:, 1], dtype=np.float32)


def sort_u(X, Y, r):
    """Sort coordinate of region r (0..3): R1 x up, R2 y up, R3 x down, R4 y down."""
    return (X, Y, -X, -Y)[r]


def order_word(f):
    """Order-preserving unsigned word of float32 values (-0.0 read as +0.0)."""
    u = (np.asarray(f, dtype=np.float32) + np.float32(0.0)).view(np.uint32).astype(np.uint64)
    neg = (u & 0x80000000) != 0
    return np.where(neg, (~u) & 0xFFFFFFFF, u | 0x80000000).astype(np.uint64)


def cmp_word(X, Y, r):
    """Compared coordinate of region r as an order word, smaller is better:
    R1 y, R2 -x, R3 -y, R4 x."""
    return order_word((Y, -X, -Y, X)[r])


def bucket(u, lo, scale, nb):
    """Monotone bucket map of float32 u: floor((u - lo) * scale), clamped."""
    t = (np.asarray(u, dtype=np.float32) - np.float32(lo)) * np.float32(scale)
    b = np.floor(np.nan_to_num(t.astype(np.float64), nan=0.0, posinf=nb, neginf=-1))
    return np.clip(b, 0, nb - 1).astype(np.int64)


def chunk_steps(X, Y, r, nloc):
    """One CTA's steps of region r: the best (word, u) per bucket of the
    chunk's own map over its extent, then the buckets beating all lower ones."""
    u = sort_u(X, Y, r)
    v = cmp_word(X, Y, r)
    a, b = np.float32(u.min()), np.float32(u.max())
    wd = np.float32(b - a)
    scale = np.float32(nloc) / wd if wd > 0 else np.float32(0)
    bk = bucket(u, a, scale, nloc)
    order = np.lexsort((u, v, bk))                 # per bucket: smallest word, then smallest u
    first = np.ones(len(order), bool)
    first[1:] = bk[order][1:] != bk[order][:-1]
    rep = order[first]                             # bucket order
    vv = v[rep]
    steps = np.ones(len(rep), bool)
    steps[1:] = vv[1:] < np.minimum.accumulate(vv)[:-1]
    return u[rep[steps]], vv[steps]


def table(X, Y, m, chunk, nloc, E, inclusive=False):
    """The device table of every region from the last m points in chunks."""
    n = len(X)
    tabs = []
    for r in range(4):
        su, sv = [], []
        for c0 in range(n - m, n, chunk):
            a, b = chunk_steps(X[c0:c0 + chunk], Y[c0:c0 + chunk], r, nloc)
            su.append(a)
            sv.append(b)
        su, sv = np.concatenate(su), np.concatenate(sv)
        lo = sort_u(X[E[r]], Y[E[r]], r)
        hi = sort_u(X[E[(r + 1) % 4]], Y[E[(r + 1) % 4]], r)
        scale = np.float32(NB) / np.float32(hi - lo) if hi > lo else np.float32(0)
        mins = np.full(NB, 0xFFFFFFFF, dtype=np.uint64)
        np.minimum.at(mins, bucket(su, lo, scale, NB), sv)
        run = np.minimum.accumulate(mins)
        pre = run if inclusive else np.concatenate([[np.uint64(0xFFFFFFFF)], run[:-1]])
        pre = np.minimum(pre, cmp_word(X[E[r]:E[r] + 1], Y[E[r]:E[r] + 1], r)[0])
        tabs.append((lo, scale, pre))
    return tabs


def dropped(X, Y, region, tabs):
    """Indices the table test drops: region-r points whose word exceeds the
    prefix of their bucket."""
    out = []
    for r in range(4):
        i = np.nonzero(region == r + 1)[0]
        lo, scale, pre = tabs[r]
        b = bucket(sort_u(X[i], Y[i], r), lo, scale, NB)
        out.append(i[cmp_word(X[i], Y[i], r) > pre[b]])
    return out


def box_dropped(X, Y, m):
    """The dominance box of the last m points: strictly inside it means
    strictly beaten in all four quadrants."""
    sx, sy = X[-m:].astype(np.float64), Y[-m:].astype(np.float64)
    q = [np.argmin(sx + sy), np.argmin(sy - sx), np.argmin(-sx - sy), np.argmin(sx - sy)]
    bx0, bx1 = max(sx[q[0]], sx[q[3]]), min(sx[q[1]], sx[q[2]])
    by0, by1 = max(sy[q[0]], sy[q[1]]), min(sy[q[2]], sy[q[3]])
    inside = (X > bx0) & (X < bx1) & (Y > by0) & (Y < by1)
    return np.nonzero(inside)[0]


SETS = [("square", lambda: inputs.square_f64(40_000, 11)),
        ("disk", lambda: inputs.disk_f64(40_000, 12)),
        ("gauss", lambda: inputs.gauss_f64(40_000, 13)),
        ("shell", lambda: inputs.shell_f64(30_000, 14)),
        ("int32", lambda: inputs.square_i32(40_000, 15).astype(np.float64))]


@pytest.fixture(scope="module")
def cases():
    out = {}
    for name, gen in SETS:
        p = gen()
        m = oracle.method(p)
        X, Y = views(p)
        spa = [set(a.tolist()) for a in m["spa"]]
        out[name] = (p, m, X, Y, spa)
    return out


@pytest.mark.parametrize("name", [s[0] for s in SETS])
@pytest.mark.parametrize("chunk,nloc", [(2048, 512), (512, 64), (8192, 512), (40_000, 1024)])
def test_table_from_chunk_steps_drops_no_spa_survivor(cases, name, chunk, nloc):
    p, m, X, Y, spa = cases[name]
    n = len(X)
    ms = min(n, max(8192, n // 16))
    tabs = table(X, Y, ms, chunk, nloc, m["ext"])
    drop = dropped(X, Y, m["region"], tabs)
    for r in range(4):
        assert not (set(drop[r].tolist()) & spa[r]), (name, chunk, nloc, r)
    # not vacuous: the table removes most round-1 survivors of these sets
    r1 = sum(len(a) for a in m["r1"])
    assert sum(len(d) for d in drop) > 0.5 * r1 or name == "gauss", (name, r1)


@pytest.mark.parametrize("name", [s[0] for s in SETS])
def test_dominance_box_drops_no_spa_survivor(cases, name):
    p, m, X, Y, spa = cases[name]
    n = len(X)
    inside = set(box_dropped(X, Y, min(n, max(8192, n // 16))).tolist())
    assert inside, name
    for r in range(4):
        assert not (inside & spa[r]), (name, r)


def test_planted_inclusive_prefix_is_caught(cases):
    """With the prefix taken over a point's own bucket too, the table drops
    SPA survivors on these inputs: the check above has teeth."""
    hit = 0
    for name in ("square", "disk", "shell"):
        p, m, X, Y, spa = cases[name]
        n = len(X)
        tabs = table(X, Y, min(n, max(8192, n // 16)), 2048, 512, m["ext"], inclusive=True)
        drop = dropped(X, Y, m["region"], tabs)
        hit += sum(len(set(drop[r].tolist()) & spa[r]) for r in range(4))
    assert hit > 0


def chunk_steps_skipping(X, Y, r, nloc):
    """chunk_steps without the points that the chunk's quadrant extreme of
    region r beats strictly in both coordinates (R1 lower-left, R2
    lower-right, R3 upper-right, R4 upper-left), as k_stairs skips them."""
    sx, sy = X.astype(np.float64), Y.astype(np.float64)
    score = (sx + sy, sy - sx, -sx - sy, sx - sy)[r]
    q = int(np.argmin(score))
    qx, qy = X[q], Y[q]
    bx = (qx < X) if r in (0, 3) else (qx > X)
    by = (qy < Y) if r < 2 else (qy > Y)
    keep = ~(bx & by)
    u = sort_u(X, Y, r)
    a, b = np.float32(u.min()), np.float32(u.max())      # the map is the whole chunk's
    wd = np.float32(b - a)
    scale = np.float32(nloc) / wd if wd > 0 else np.float32(0)
    bk = bucket(u, a, scale, nloc)[keep]
    uu, v = u[keep], cmp_word(X, Y, r)[keep]
    order = np.lexsort((uu, v, bk))
    first = np.ones(len(order), bool)
    first[1:] = bk[order][1:] != bk[order][:-1]
    rep = order[first]
    vv = v[rep]
    steps = np.ones(len(rep), bool)
    steps[1:] = vv[1:] < np.minimum.accumulate(vv)[:-1]
    return uu[rep[steps]], vv[steps]


@pytest.mark.parametrize("name", [s[0] for s in SETS])
def test_skipping_points_beaten_by_the_quadrant_extreme_keeps_the_steps(cases, name):
    p, m, X, Y, spa = cases[name]
    n = len(X)
    for c0 in range(n - 8192, n, 2048):
        cx, cy = X[c0:c0 + 2048], Y[c0:c0 + 2048]
        for r in range(4):
            a = chunk_steps(cx, cy, r, 512)
            b = chunk_steps_skipping(cx, cy, r, 512)
            assert np.array_equal(a[1], b[1]), (name, c0, r)
            assert np.array_equal(a[0], b[0]), (name, c0, r)

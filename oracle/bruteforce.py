"""Brute-force definitions on exact rationals -- TEST INFRASTRUCTURE ONLY.

These are the pins for the C oracle: slow (O(n^3) hull, O(n^2) SPA), written
directly from the definitions with ``fractions.Fraction`` (every float64 and
int32 converts to a Fraction exactly), so they involve no floating-point
reasoning at all.  Only the test suite imports this module.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _q(v) -> Fraction:
    """Exact rational value of an int or float coordinate (numpy or Python)."""
    if isinstance(v, Fraction):
        return v
    if isinstance(v, (int, np.integer)):
        return Fraction(int(v))
    return Fraction(float(v))


def _fr(points):
    return [(_q(x), _q(y)) for x, y in np.asarray(points).tolist()]


def orient(a, b, c) -> int:
    """sign((b - a) x (c - a)) in exact rational arithmetic."""
    a, b, c = [tuple(_q(v) for v in p) for p in (a, b, c)]
    d = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    return (d > 0) - (d < 0)


def _classes(P):
    """Distinct coordinates -> smallest index having them."""
    rep = {}
    for i, p in enumerate(P):
        rep.setdefault(p, i)
    return rep


def hull(points) -> list[int]:
    """Strict convex hull vertices, CCW from the lexicographic minimum.

    A directed pair (p, q) of distinct points is a hull edge iff every input
    point r is strictly left of p->q or lies on the closed segment [p, q].
    Following the edges from the lexicographic minimum gives the CCW cycle.
    """
    P = _fr(points)
    if not P:
        return []
    rep = _classes(P)
    Q = sorted(rep)                       # lexicographic (x, y)
    if len(Q) == 1:
        return [rep[Q[0]]]

    def on_segment(p, q, r):
        return (min(p[0], q[0]) <= r[0] <= max(p[0], q[0])
                and min(p[1], q[1]) <= r[1] <= max(p[1], q[1]))

    succ = {}
    for p in Q:
        for q in Q:
            if p == q:
                continue
            ok = True
            for r in Q:
                o = orient(p, q, r)
                if o < 0 or (o == 0 and not on_segment(p, q, r)):
                    ok = False
                    break
            if ok:
                assert p not in succ, "two successors: not a strict hull"
                succ[p] = q
    start = Q[0]
    out = [rep[start]]
    cur = succ[start]
    while cur != start:
        out.append(rep[cur])
        cur = succ[cur]
        assert len(out) <= len(Q)
    return out


def extremes(points) -> list[int]:
    """P_minx = lexmin(x, y), P_miny = lexmin(y, x), P_maxx = lexmax(x, y),
    P_maxy = lexmax(y, x); ties between identical points -> smallest index."""
    P = _fr(points)
    idx = range(len(P))
    e1 = min(idx, key=lambda i: (P[i][0], P[i][1], i))
    e2 = min(idx, key=lambda i: (P[i][1], P[i][0], i))
    e3 = min(idx, key=lambda i: (-P[i][0], -P[i][1], i))
    e4 = min(idx, key=lambda i: (-P[i][1], -P[i][0], i))
    return [e1, e2, e3, e4]


def regions(points, ext) -> list[int]:
    """Region of every point: first k with the point strictly right of the
    directed edge E_k -> E_{k+1} (outside the CCW quadrilateral), else 0."""
    P = _fr(points)
    E = [P[i] for i in ext] + [P[ext[0]]]
    out = []
    for p in P:
        r = 0
        for k in range(4):
            if orient(E[k], E[k + 1], p) < 0:
                r = k + 1
                break
        out.append(r)
    return out


def spa_survivors(points, ext, region) -> list[set[int]]:
    """SPA survivors per region by dominance, without any sorting.

    Region k is ordered by its Table 1 coordinate (x asc, y asc, x desc,
    y desc) with the index breaking ties.  A point P of R_k is discarded iff
    the region's first extreme, or some point of R_k before P in that order,
    is strictly better in the other coordinate (lower y for R1, greater x for
    R2, greater y for R3, lower x for R4) -- Fig. 2 unrolled.
    """
    P = _fr(points)
    out = []
    for k in range(4):
        members = [i for i, r in enumerate(region) if r == k + 1]
        sc = 0 if k in (0, 2) else 1          # sort coordinate
        oc = 1 - sc                            # compared coordinate
        sgn = 1 if k in (0, 1) else -1         # ascending for R1, R2

        def before(q, p):
            a, b = sgn * P[q][sc], sgn * P[p][sc]
            return a < b or (a == b and q < p)

        def better(q, p):
            if k in (0, 3):
                return P[q][oc] < P[p][oc]
            return P[q][oc] > P[p][oc]

        e = ext[k]
        keep = set()
        for p in members:
            if better(e, p):
                continue
            if any(before(q, p) and better(q, p) for q in members if q != p):
                continue
            keep.add(p)
        out.append(keep)
    return out

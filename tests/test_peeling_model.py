"""CPU model of the chain hull by peeling (no GPU).

The device replaces the paper's CPU stage by peeling each region's chain
E_r, SPA survivors in order, E_{r+1}: every point that does not make a strict
left turn with its two current neighbours lies on or inside the segment
between them, so it is no strict vertex of the hull; all such points leave
at once, round after round, and when none is left the chain is convex.  This
module runs that rule in numpy with exact orientation on the chains that
`oracle.method` produces and checks that it ends at the oracle hull's
vertices between E_r and E_{r+1}, for several distributions; it also checks
that each round only removes points that are not strict hull vertices.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1508_05488_gb300 import inputs


def orient(p, a, b, c):
    """Exact sign of (b - a) x (c - b) for rows a, b, c of p."""
    ax, ay = Fraction(float(p[a, 0])), Fraction(float(p[a, 1]))
    bx, by = Fraction(float(p[b, 0])), Fraction(float(p[b, 1]))
    cx, cy = Fraction(float(p[c, 0])), Fraction(float(p[c, 1]))
    q = (bx - ax) * (cy - by) - (by - ay) * (cx - bx)
    return (q > 0) - (q < 0)


def peel(p, chain):
    """Peeling rounds until no interior point fails a strict left turn."""
    chain = list(chain)
    rounds = 0
    while True:
        drop = [i for i in range(1, len(chain) - 1) if orient(p, chain[i - 1], chain[i], chain[i + 1]) <= 0]
        if not drop:
            return chain, rounds
        keep = set(range(len(chain))) - set(drop)
        chain = [chain[i] for i in sorted(keep)]
        rounds += 1


def hull_chain(hull, a, b):
    """The hull's vertices from index a to index b, counter-clockwise."""
    h = hull.tolist()
    i, j = h.index(a), h.index(b)
    return h[i:j + 1] if i <= j else h[i:] + h[:j + 1]


SETS = [("square", lambda: inputs.square_f64(20_000, 21)),
        ("disk", lambda: inputs.disk_f64(20_000, 22)),
        ("gauss", lambda: inputs.gauss_f64(20_000, 23)),
        ("shell", lambda: inputs.shell_f64(6_000, 24)),
        ("circle", lambda: inputs.circle_f64(1_500, 25))]


@pytest.mark.parametrize("name,gen", SETS)
def test_peeling_ends_at_the_hull_chain(name, gen):
    p = gen()
    m = oracle.method(p)
    E = m["ext"].tolist()
    hull = m["hull"]
    hv = set(hull.tolist())
    for r in range(4):
        a, b = E[r], E[(r + 1) % 4]
        if a == b:
            continue
        chain = [a] + m["spa"][r].tolist() + [b]
        out, rounds = peel(p, chain)
        assert out == hull_chain(hull, a, b), (name, r, rounds)
        # nothing a round removes is a strict hull vertex
        assert not (set(chain) - set(out)) & hv

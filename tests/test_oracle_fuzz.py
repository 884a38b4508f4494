"""Property-based pins for the CPU oracle (no GPU; skipped without hypothesis).

Small point sets on coarse grids force the cases a plausible mistake breaks:
duplicates, collinear runs, points on the quadrilateral's edges, ties among
extreme candidates, signed zeros.  Every case is checked against the exact
rational brute force (O(n^3) hull, dominance SPA), and the multi-core CPU
baseline against the oracle.
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import oracle  # noqa: E402
from oracle import bruteforce as bf  # noqa: E402

GRID = st.integers(min_value=-4, max_value=4)
POINT = st.tuples(GRID, GRID)
POINTS = st.lists(POINT, min_size=0, max_size=40)
SCALE = st.sampled_from([1.0, 0.5, -0.25, 1e-3, 3.0e10])


def as_f64(pts, scale):
    """Grid points scaled (a negative scale makes the zeros -0.0)."""
    return np.array(pts, dtype=np.float64).reshape(-1, 2) * scale


@settings(max_examples=300, deadline=None)
@given(POINTS)
def test_hull_int32_matches_bruteforce(pts):
    p = np.array(pts, dtype=np.int32).reshape(-1, 2)
    assert oracle.hull(p).tolist() == bf.hull(p)


@settings(max_examples=300, deadline=None)
@given(POINTS, SCALE)
def test_hull_float64_matches_bruteforce(pts, scale):
    p = as_f64(pts, scale)
    assert oracle.hull(p).tolist() == bf.hull(p)


@settings(max_examples=200, deadline=None)
@given(POINTS, SCALE)
def test_method_stages_match_bruteforce_fuzzed(pts, scale):
    p = as_f64(pts, scale)
    if len(p) == 0:
        return
    m = oracle.method(p)
    ext = bf.extremes(p)
    assert m["ext"].tolist() == ext
    reg = bf.regions(p, ext)
    assert m["region"].tolist() == reg
    for k in range(4):
        members = [i for i, r in enumerate(reg) if r == k + 1]
        assert m["r1"][k].tolist() == members
    spa = bf.spa_survivors(p, ext, reg)
    for k in range(4):
        assert set(m["spa"][k].tolist()) == spa[k]
    # every hull vertex survives both rounds (it is an extreme or an SPA survivor)
    kept = set(ext).union(*[set(m["spa"][k].tolist()) for k in range(4)])
    assert set(m["hull"].tolist()) <= kept
    assert m["hull"].tolist() == bf.hull(p)


@pytest.mark.skipif(not oracle.parallel_available(), reason="gcc without OpenMP")
@settings(max_examples=200, deadline=None)
@given(POINTS, st.integers(min_value=1, max_value=8))
def test_parallel_baseline_matches_oracle_fuzzed(pts, threads):
    p = np.array(pts, dtype=np.int32).reshape(-1, 2)
    assert oracle.parallel_hull(p, threads).tolist() == oracle.hull(p).tolist()
    q = as_f64(pts, 0.5)
    assert oracle.parallel_hull(q, threads).tolist() == oracle.hull(q).tolist()

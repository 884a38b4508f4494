"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Every comparison is element by element on integer index lists: the hull is
unique (strict vertices, CCW from the lexicographic minimum, smallest index
among identical points), so the bar is bit-exact equality.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1508_05488_gb300 as cch
from paper_1508_05488_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def gpu_hull(p):
    return cch.hull(torch.from_numpy(np.ascontiguousarray(p)).to(DEV)).cpu().numpy()


def check(p):
    got = gpu_hull(p)
    want = oracle.hull(p)
    assert np.array_equal(got, want), (p.dtype, p.shape, got[:10], want[:10], len(got), len(want))
    return got


# ------------------------------------------------------------ edge cases

def test_empty_single_two_identical():
    for dt in (np.int32, np.float64):
        assert len(gpu_hull(np.zeros((0, 2), dt))) == 0
        assert gpu_hull(np.array([[5, 7]], dt)).tolist() == [0]
        check(np.array([[5, 7], [1, 2]], dt))
        check(np.array([[5, 7], [5, 7]], dt))
        check(np.tile(np.array([[3, -4]], dt), (10_000, 1)))


def test_signed_zero_is_one_coordinate():
    p = np.array([[0.0, 1.0], [-0.0, 1.0], [0.0, -0.0], [1.0, 1.0], [-0.0, 0.0]])
    check(p)


@pytest.mark.parametrize("d", [(1, 2), (1, -3), (0, 1), (1, 0), (-2, 1)])
def test_collinear(d):
    t = np.random.default_rng(1).permutation(30_000)
    p = np.stack([7 + d[0] * t, -9 + d[1] * t], 1)
    check(p.astype(np.int32))
    check((p / 8.0).astype(np.float64))


def test_grid_and_small_adversarial():
    for k in (2, 3, 17, 300):
        g = np.stack(np.meshgrid(np.arange(k), np.arange(k)), -1).reshape(-1, 2)
        g = g[np.random.default_rng(k).permutation(len(g))]
        check(g.astype(np.int32))
        check(g.astype(np.float64) * 0.5)
    for seed in range(300):
        check(inputs.small_cases(seed))


def test_full_int32_range_uses_wide_products():
    rng = np.random.default_rng(5)
    p = rng.integers(-2 ** 31, 2 ** 31, size=(200_000, 2), dtype=np.int64).astype(np.int32)
    check(p)
    q = np.array([[-2 ** 31, -2 ** 31], [2 ** 31 - 1, 2 ** 31 - 1], [-2 ** 31, 2 ** 31 - 1],
                  [2 ** 31 - 1, -2 ** 31], [0, 0], [-2 ** 31, 0]], dtype=np.int32)
    check(q)


# --------------------------------------------------- several tiles, ragged

@pytest.mark.parametrize("n", [4095, 4096, 4097, 100_003, 1_000_001])
@pytest.mark.parametrize("kind", ["square", "disk", "gauss", "i32", "idisk"])
def test_random_sizes(kind, n):
    seed = n % 97
    p = {"square": lambda: inputs.square_f64(n, seed),
         "disk": lambda: inputs.disk_f64(n, seed),
         "gauss": lambda: inputs.gauss_f64(n, seed),
         "i32": lambda: inputs.square_i32(n, seed),
         "idisk": lambda: inputs.disk_i32(n, seed)}[kind]()
    check(p)


# 16388 / 16392 put about 4096 kept candidates in each region (the edge of
# the shared-memory record path), 20000 about 5000 (the counting path on
# global records), 70000 and up take the multi-block path
@pytest.mark.parametrize("n", [3, 1000, 4098, 16_388, 16_392, 20_000, 70_000, 300_000])
def test_all_extreme_circle(n):
    p = inputs.circle_f64(n, seed=n)
    h = check(p)
    assert len(h) == n


def test_degenerate_grid_duplicates():
    check(inputs.degenerate_f64(400_000, seed=9))


def test_shell_and_far_from_origin():
    check(inputs.shell_f64(300_000, 3))
    # far from the origin the FP32 filter cannot decide: exact path everywhere
    check(inputs.square_f64(200_000, 4) + 1.0e7)
    check(inputs.disk_f64(100_000, 5) * 2.0 ** 70)
    check(inputs.disk_f64(100_000, 5) * 2.0 ** -300)


def test_nearly_collinear_chains():
    """Closely spaced hull points: orientation determinants far below the
    coordinates' FP32 resolution (the split filter and the exact fallback)."""
    rng = np.random.default_rng(41)
    # tiny circle away from the origin: every point is a hull vertex
    t = 2.0 * np.pi * rng.permutation(60_000) / 60_000
    check(np.stack([0.3 + 1e-6 * np.cos(t), -0.7 + 1e-6 * np.sin(t)], 1))
    # dense unit circle: neighbours 3e-6 apart
    check(inputs.circle_f64(2_000_003, seed=8))
    # a line with noise at the last bits, and a parabola on a fine grid
    x = rng.random(200_000)
    check(np.stack([x, 0.5 * x + 0.25 + 1e-15 * rng.standard_normal(200_000)], 1))
    g = np.arange(-50_000, 50_001) / 50_000.0
    g = g[rng.permutation(len(g))]
    check(np.stack([g, g * g], 1))
    check(np.stack([1e5 + g, 3e5 - g * g], 1))


# ------------------------------------------------------------ stages

STAGE_KINDS = {
    "square": lambda n: inputs.square_f64(n, 11),
    "disk": lambda n: inputs.disk_f64(n, 12),
    "gauss": lambda n: inputs.gauss_f64(n, 13),
    "i32": lambda n: inputs.square_i32(n, 14),
    "idisk": lambda n: inputs.disk_i32(n, 16),
    "degenerate": lambda n: inputs.degenerate_f64(n, 15),
    "grid": lambda n: (np.random.default_rng(3).integers(0, 40, (n, 2)) / 8.0),
    "igrid": lambda n: np.random.default_rng(4).integers(-20, 20, (n, 2)).astype(np.int32),
}


@pytest.mark.parametrize("kind", list(STAGE_KINDS))
@pytest.mark.parametrize("exact_only", [False, True])
@pytest.mark.parametrize("prefilter", [False, True])
def test_stage_sets_match_method(kind, exact_only, prefilter):
    """Round-1 sets (paper mode: no prefilter) and SPA survivors (either
    mode: the prefilter removes only SPA-dominated points) equal the
    step-by-step restatement of Sec. 2.1."""
    n = 150_001
    p = STAGE_KINDS[kind](n)
    st = cch.stages(torch.from_numpy(p).to(DEV), exact_only=exact_only, prefilter=prefilter)
    m = oracle.method(p)
    assert st["status"] == 0
    for r in range(4):
        if not prefilter:
            assert np.array_equal(st["r1"][r], m["r1"][r]), ("round 1", r)
        else:
            assert np.isin(st["r1"][r], m["r1"][r]).all(), ("round 1 subset", r)
            assert np.all(np.diff(st["r1"][r]) > 0)
        assert np.array_equal(st["spa"][r], m["spa"][r]), ("SPA", r)
    assert np.array_equal(st["hull"], m["hull"])


@pytest.mark.parametrize("kind,n", [(k, n) for k in STAGE_KINDS for n in (3_000, 150_001)] +
                         [("square", 2_500_003), ("disk", 2_500_003), ("i32", 2_500_003)])
def test_blocked_spa_of_the_paper(kind, n):
    """The paper's chunked GPU SPA (Sec. 2.2.2, cch_hull_stages opts bit 2):
    its survivors equal the oracle's chunked restatement element by element,
    contain the sequential SPA survivors, and the hull is unchanged.  Sizes
    span regions below 1024 points (every point its own chunk) up to chunks
    of hundreds of points."""
    p = STAGE_KINDS[kind](n)
    st = cch.stages(torch.from_numpy(p).to(DEV), blocked=True)
    m = oracle.method(p)
    want = oracle.blocked_spa(p, m=m)
    assert st["status"] == 0
    for r in range(4):
        assert np.array_equal(st["r1"][r], m["r1"][r]), ("round 1", r)
        assert np.array_equal(st["spa"][r], want[r]), ("blocked SPA", r)
        assert np.isin(m["spa"][r], st["spa"][r]).all(), ("superset of the sequential SPA", r)
    assert np.array_equal(st["hull"], m["hull"])


@pytest.mark.parametrize("kind,n", [(k, n) for k in STAGE_KINDS for n in (3_000, 60_001)])
def test_octagon_round1(kind, n):
    """Round 1 with the Akl-Toussaint octagon (cch_hull_stages opts bit 3):
    the diagonal extremes, the round-1 sets and the SPA survivors equal the
    oracle's restatement element by element (the paper's sets without the
    points strictly inside the octagon), and the hull is unchanged."""
    p = STAGE_KINDS[kind](n)
    st = cch.stages(torch.from_numpy(p).to(DEV), octagon=True)
    m = oracle.method(p)
    diag = oracle.octagon_diag(p, m)
    assert st["status"] == 0
    assert st["diag"].tolist() == diag.tolist()
    o = oracle.octagon_round1(p, diag, m)
    for r in range(4):
        assert np.array_equal(st["r1"][r], o["r1"][r]), ("round 1", r)
        assert np.array_equal(st["spa"][r], o["spa"][r]), ("SPA", r)
    assert np.array_equal(st["hull"], m["hull"])


def test_prefilter_shrinks_round1_on_uniform_sets():
    for p in (inputs.square_f64(1_000_000, 5), inputs.disk_f64(1_000_000, 6)):
        t = torch.from_numpy(p).to(DEV)
        on = cch.stages(t)
        off = cch.stages(t, prefilter=False)
        assert on["counts"][0] * 5 < off["counts"][0]
        assert np.array_equal(on["hull"], off["hull"])


# ------------------------------------------------------------ batched

def test_batched_matches_per_set():
    rng = np.random.default_rng(21)
    sizes = [0, 1, 2, 3, 5000, 0, 4096, 4097, 70_000, 7, 130_000, 1]
    parts = []
    for i, n in enumerate(sizes):
        kind = i % 3
        q = (inputs.square_f64(n, i) if kind == 0 else inputs.disk_f64(n, i) if kind == 1
             else inputs.circle_f64(n, i))
        parts.append(q)
    parts[5] = np.zeros((0, 2))
    p = np.concatenate(parts)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    res = cch.hull_batched(torch.from_numpy(p).to(DEV), off)
    for s in range(len(sizes)):
        want = oracle.hull(p[off[s]:off[s + 1]])
        assert np.array_equal(res[s].cpu().numpy(), want), s
    del rng


def test_batched_few_large_sets_cluster_split():
    """A batched call of three sets (the cluster form of the per-region
    sort): the 5M disk's regions hold about 6k round-1 survivors each and are
    split over their clusters; the other two sets' regions are not."""
    parts = [inputs.disk_f64(5_000_000, 31), inputs.square_f64(20_000, 32), inputs.gauss_f64(3_000_000, 33)]
    p = np.concatenate(parts)
    off = np.concatenate([[0], np.cumsum([len(q) for q in parts])]).astype(np.int64)
    st = cch.stages(torch.from_numpy(parts[0]).to(DEV))
    assert int(st["counts"][1:5].max()) >= 4096, st["counts"][:5]
    res = cch.hull_batched(torch.from_numpy(p).to(DEV), off)
    for s in range(3):
        assert np.array_equal(res[s].cpu().numpy(), oracle.hull(parts[s])), s


def test_batched_int32_many_sets():
    p, off = inputs.batched_i32(300, seed=3, lo=16, hi=20_000)
    res = cch.hull_batched(torch.from_numpy(p).to(DEV), off)
    for s in range(300):
        assert np.array_equal(res[s].cpu().numpy(), oracle.hull(p[off[s]:off[s + 1]])), s


# ------------------------------------------------------------ host e2e, errors

def test_host_entry_point():
    p = inputs.disk_f64(500_000, 17)
    assert np.array_equal(cch.hull_host(p), oracle.hull(p))
    q = inputs.square_i32(300_000, 18)
    assert np.array_equal(cch.hull_host(q), oracle.hull(q))


def test_device_errors_are_reported_in_the_count():
    p = inputs.square_f64(10_000, 1)
    p[77, 1] = np.nan
    _, cnt = cch.hull_async(torch.from_numpy(p).to(DEV))
    assert int(cnt.item()) == -3
    p[77, 1] = 2.0 ** 450
    _, cnt = cch.hull_async(torch.from_numpy(p).to(DEV))
    assert int(cnt.item()) == -4
    p[77, 1] = 5e-324
    _, cnt = cch.hull_async(torch.from_numpy(p).to(DEV))
    assert int(cnt.item()) == -4
    # the context stays usable
    check(inputs.square_f64(10_000, 2))


# ---------------------------------------- float32 SoA input (Fig. 6 form)

def f32soa_hull(x, y):
    tx = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(DEV)
    ty = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).to(DEV)
    return cch.hull_f32soa(tx, ty).cpu().numpy()


def check_f32(p32):
    """float32 points: the oracle's hull of their exact float64 values."""
    got = f32soa_hull(p32[:, 0], p32[:, 1])
    want = oracle.hull(p32.astype(np.float64))
    assert np.array_equal(got, want), (p32.shape, got[:10], want[:10], len(got), len(want))
    return got


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4097, 100_003, 1_000_001])
@pytest.mark.parametrize("kind", ["square", "disk", "gauss"])
def test_f32soa_matches_oracle(kind, n):
    seed = n % 89
    p = {"square": lambda: inputs.square_f64(n, seed),
         "disk": lambda: inputs.disk_f64(n, seed),
         "gauss": lambda: inputs.gauss_f64(n, seed)}[kind]()
    check_f32(p.astype(np.float32))


def test_f32soa_special_values_and_unaligned_vectors():
    """Subnormal, signed-zero, huge and duplicate float32 coordinates (the
    widening normalises subnormals), and x / y views that start one float
    into their buffers."""
    rng = np.random.default_rng(23)
    sub = rng.integers(1, 1 << 23, (3000, 2), dtype=np.uint32)
    sub |= (rng.integers(0, 2, (3000, 2), dtype=np.uint32) << 31)
    tiny = sub.view(np.float32)
    big = (rng.random((3000, 2)) * 2 - 1).astype(np.float32) * np.float32(3.0e38)
    zeros = np.array([[0.0, -0.0], [-0.0, 0.0], [0.0, 0.0], [-0.0, -0.0]], dtype=np.float32)
    for p in (tiny, big, np.concatenate([tiny, zeros, tiny[:50]]), np.concatenate([big, tiny, zeros])):
        check_f32(p)
    base = inputs.disk_f64(100_001, 7).astype(np.float32)
    bx = torch.from_numpy(np.ascontiguousarray(base[:, 0])).to(DEV)
    by = torch.from_numpy(np.ascontiguousarray(base[:, 1])).to(DEV)
    got = cch.hull_f32soa(bx[1:], by[1:]).cpu().numpy()
    assert np.array_equal(got, oracle.hull(base[1:].astype(np.float64)))


def test_f32soa_tiny_sets():
    """1..12 float32 points, mixed signs: tiles that the plain loads fill
    alone (no bulk bytes), or nearly so."""
    rng = np.random.default_rng(31)
    for t in range(240):
        n = 1 + t % 12
        p = (rng.random((n, 2)) * 2 - 1).astype(np.float32)
        if t % 3 == 0:
            p = np.abs(p)
        check_f32(p)


@pytest.mark.parametrize("n", [5, 4095, 4097, 70_001])
def test_f32soa_every_vector_alignment(n):
    """x and y starting 0..3 floats past a 16-byte boundary, independently:
    the tiles' leading and trailing points of each vector that the bulk
    copies cannot take."""
    base = inputs.disk_f64(n + 3, n % 13).astype(np.float32)
    bx = torch.from_numpy(np.ascontiguousarray(base[:, 0])).to(DEV)
    by = torch.from_numpy(np.ascontiguousarray(base[:, 1])).to(DEV)
    for ox in range(4):
        for oy in range(4):
            got = cch.hull_f32soa(bx[ox:ox + n], by[oy:oy + n]).cpu().numpy()
            q = np.stack([base[ox:ox + n, 0], base[oy:oy + n, 1]], axis=1).astype(np.float64)
            assert np.array_equal(got, oracle.hull(q)), (n, ox, oy)


def test_f32soa_multiblock_sort_path():
    """A float32 circle: about n / 4 round-1 survivors in every region, far
    above the shared-memory sort's limit, so the multi-block sort and SPA
    read the float32 vectors."""
    n = 300_000
    t = 2 * np.pi * np.arange(n) / n
    p = np.stack([np.cos(t), np.sin(t)], axis=1).astype(np.float32)
    check_f32(p[np.random.default_rng(4).permutation(n)])


def test_f32soa_nonfinite_is_reported():
    p = inputs.square_f64(5000, 3).astype(np.float32)
    for bad in (np.nan, np.inf, -np.inf):
        q = p.copy()
        q[1234, 1] = bad
        x = torch.from_numpy(np.ascontiguousarray(q[:, 0])).to(DEV)
        y = torch.from_numpy(np.ascontiguousarray(q[:, 1])).to(DEV)
        _, cnt = cch.hull_f32soa_async(x, y)
        assert int(cnt.item()) == -3
    assert np.array_equal(f32soa_hull(p[:, 0], p[:, 1]), oracle.hull(p.astype(np.float64)))


def test_host_errors_return_codes():
    lib = cch.lib()
    x = torch.zeros(4, 2, dtype=torch.float64, device=DEV)
    o = torch.zeros(4, dtype=torch.int32, device=DEV)
    c = torch.zeros(1, dtype=torch.int32, device=DEV)
    assert lib.cch_hull(x.data_ptr(), 4, 7, o.data_ptr(), c.data_ptr(), None) == -2
    assert lib.cch_hull(x.data_ptr(), -1, 2, o.data_ptr(), c.data_ptr(), None) == -1
    assert lib.cch_hull(x.data_ptr() + 8, 3, 2, o.data_ptr(), c.data_ptr(), None) == -1
    assert lib.cch_hull(x.data_ptr(), 4, 2, None, c.data_ptr(), None) == -1


def test_bounded_wait_reports_timeout_and_context_survives():
    """The device-side failure path: a wait on a flag nothing sets gives up
    within its bound and reports CCH_ERR_TIMEOUT; later calls still work."""
    import time
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    t0 = time.time()
    assert cch.lib().cch_selftest_wait(st.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert time.time() - t0 < 10.0
    assert int(st.item()) == -7
    check(inputs.disk_f64(50_000, 9))


def test_repeated_calls_and_streams_are_independent():
    a = inputs.disk_f64(200_000, 31)
    b = inputs.square_i32(300_000, 32)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ta, tb = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    torch.cuda.synchronize()
    outs = []
    for _ in range(5):
        outs.append((cch.hull_async(ta, stream=s1), cch.hull_async(tb, stream=s2)))
    torch.cuda.synchronize()
    wa, wb = oracle.hull(a), oracle.hull(b)
    for (ia, ca), (ib, cb) in outs:
        assert np.array_equal(ia[:int(ca.item())].cpu().numpy(), wa)
        assert np.array_equal(ib[:int(cb.item())].cpu().numpy(), wb)


# ------------------------------- shared-memory sort, cluster form, crowded

def test_cluster_sort_crowded_region():
    """One region of about 10k round-1 survivors in columns of 40 equal
    sort coordinates: the region is split over the cluster and the leader
    sorts with the radix path (crowded buckets).  The lower-left arc is the
    quarter circle of radius 1 around (1, 1); column k holds the arc point
    and 39 points just above it."""
    xs = np.arange(1, 256) / 256.0
    g = 1.0 - np.sqrt(1.0 - (xs - 1.0) ** 2)
    pts = [np.array([[0.0, 1.0], [1.0, 0.0], [2.0, 1.0], [1.0, 2.0]])]
    for jj in range(40):
        pts.append(np.stack([xs, g + jj * 1e-7], axis=1))
    p = np.concatenate(pts)
    p = p[np.random.default_rng(12).permutation(len(p))]
    st = cch.stages(torch.from_numpy(p).to(DEV))
    assert int(st["counts"][1]) >= 4096, st["counts"][:5]
    check(p)

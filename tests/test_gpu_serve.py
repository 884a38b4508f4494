"""Serving: requests admitted by a memory budget and batched onto a pool of
streams while others run.  Every result must be the hull of the request
alone (element-wise equal to the CPU oracle), whatever it was batched with."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1508_05488_gb300 as cch
from paper_1508_05488_gb300 import inputs

pytestmark = pytest.mark.gpu


def drain(srv, want, timeout=120.0):
    got = {}
    t0 = time.time()
    while len(got) < want:
        for t, st, h, lat in srv.poll():
            got[t] = (st, h, lat)
        if time.time() - t0 > timeout:
            raise TimeoutError(f"{len(got)} of {want} requests finished")
        time.sleep(0.001)
    return got


def mixed_requests(seed=0):
    rng = np.random.default_rng(seed)
    kinds = [inputs.square_f64, inputs.disk_f64, inputs.gauss_f64, inputs.shell_f64]
    sizes = [0, 1, 2, 3, 17, 1000, 4097, 65_536, 100_003, 1_500_000, 20_000, 300_000]
    reqs = []
    for i, n in enumerate(sizes):
        reqs.append(kinds[i % 4](n, int(rng.integers(1 << 30))) if n else np.zeros((0, 2)))
    reqs.append(inputs.circle_f64(200_000, 3))
    return reqs


def test_results_alone_equal_results_in_the_mix():
    reqs = mixed_requests()
    want = [oracle.hull(p) for p in reqs]
    with cch.Server(np.float64, num_streams=3, max_batch=5) as srv:
        # alone: one request at a time
        for p, w in zip(reqs, want):
            t = srv.submit(p)
            got = drain(srv, 1)
            st, h, _ = got[t]
            assert st == 0 and np.array_equal(h, w), (len(p), len(h), len(w))
        # in the mix: everything at once, twice over, small and large interleaved
        tickets = [srv.submit(p) for p in reqs + reqs[::-1]]
        got = drain(srv, len(tickets))
        for t, w in zip(tickets, want + want[::-1]):
            st, h, _ = got[t]
            assert st == 0 and np.array_equal(h, w)
        s = srv.stats()
        assert s["finished"] == 3 * len(reqs)
        assert s["p99_ms"] >= s["p50_ms"] > 0.0


def test_int32_server_and_device_errors():
    with cch.Server(np.int32) as srv:
        ps = [inputs.square_i32(50_000, 5), inputs.disk_i32(70_001, 6), np.array([[3, 4]], np.int32)]
        ts = [srv.submit(p) for p in ps]
        got = drain(srv, len(ts))
        for t, p in zip(ts, ps):
            assert got[t][0] == 0 and np.array_equal(got[t][1], oracle.hull(p))
    with cch.Server(np.float64) as srv:
        p = inputs.square_f64(10_000, 1)
        p[5, 0] = np.nan
        q = inputs.square_f64(10_000, 2)
        t1, t2 = srv.submit(p), srv.submit(q)
        got = drain(srv, 2)
        assert got[t1][0] == -3                       # non-finite, reported per request
        assert got[t2][0] == 0 and np.array_equal(got[t2][1], oracle.hull(q))


def test_budget_admission_and_queue_limit():
    one = cch.lib().cch_workspace_bytes(200_000, cch.CCH_F64) + 200_000 * 24 + 8192
    with cch.Server(np.float64, budget_bytes=one, max_pending=4, num_streams=2) as srv:
        with pytest.raises(cch.CchError) as e:
            srv.submit(inputs.square_f64(2_000_000, 3))      # alone above the budget
        assert e.value.code == -4
        p = inputs.disk_f64(150_000, 4)
        w = oracle.hull(p)
        ok, busy = [], 0
        for _ in range(64):
            try:
                ok.append(srv.submit(p))
            except cch.CchError as ex:
                assert ex.code == -8
                busy += 1
        got = drain(srv, len(ok))
        assert busy > 0
        for t in ok:
            assert got[t][0] == 0 and np.array_equal(got[t][1], w)
    srv = cch.Server(np.float64)
    assert cch.lib().cch_serve_release(srv._h, 12345) == -9
    srv.close()


def test_device_submitted_requests_stay_on_the_device_and_match_alone():
    """Requests submitted from device memory (cch_serve_submit_device) --
    mixed with host submits, the caller's buffer overwritten right after each
    submit -- give the oracle's hull of each request."""
    reqs = mixed_requests(1)
    want = [oracle.hull(p) for p in reqs]
    with cch.Server(np.float64, num_streams=3, max_batch=4) as srv:
        tickets, scratch = [], torch.empty((2_000_000, 2), dtype=torch.float64, device="cuda")
        for i, p in enumerate(reqs + reqs[::-1]):
            if i % 3 == 2:
                tickets.append(srv.submit(p))                     # host submit
                continue
            d = scratch[:len(p)]
            d.copy_(torch.from_numpy(p))
            tickets.append(srv.submit(d))                         # device submit, copied before return
            d.fill_(float("nan"))                                 # the caller reuses its buffer at once
        got = drain(srv, len(tickets))
        for t, w in zip(tickets, want + want[::-1]):
            st, h, _ = got[t]
            assert st == 0 and np.array_equal(h, w)
    with cch.Server(np.int32) as srv:
        p = inputs.disk_i32(80_000, 9)
        t = srv.submit(torch.from_numpy(p).cuda())
        got = drain(srv, 1)
        assert got[t][0] == 0 and np.array_equal(got[t][1], oracle.hull(p))
        with pytest.raises(TypeError):
            srv.submit(torch.zeros((5, 2), dtype=torch.float64, device="cuda"))   # wrong dtype

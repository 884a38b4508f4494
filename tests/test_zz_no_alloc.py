"""cch_hull_noalloc: the allocation-free form of cch_hull.

Some callers cannot allocate device memory (graph capture that forbids it,
fixed-footprint real-time code, code inside an allocator callback); this entry
point serves them from a fixed array in the library's device code.  Its
output must equal cch_hull's for the same input.  The file is collected last
so that a failure here does not hide any other test's result; it also passes
alone in a fresh process (the first call on the device does the set-up).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1508_05488_gb300 as cch
from paper_1508_05488_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _noalloc(t, stream):
    n = t.shape[0]
    out = torch.full((max(n, 1),), -7, dtype=torch.int32, device=DEV)
    cnt = torch.full((1,), -7, dtype=torch.int32, device=DEV)
    dt = cch.CCH_F64 if t.dtype == torch.float64 else cch.CCH_I32
    rc = cch.lib().cch_hull_noalloc(t.data_ptr() if n else None, n, dt, out.data_ptr(),
                                    cnt.data_ptr(), stream.cuda_stream)
    assert rc == 0, rc
    return out, cnt


def test_noalloc_matches_cch_hull_on_two_calls_in_a_row():
    stream = torch.cuda.current_stream()
    a = torch.from_numpy(inputs.disk_f64(100_000, 41)).to(DEV)
    b = torch.from_numpy(inputs.square_i32(131_072, 42)).to(DEV)
    oa, ca = _noalloc(a, stream)     # first call on the device: set-up
    ob, cb = _noalloc(b, stream)     # second call reuses the array
    torch.cuda.synchronize()
    wa = cch.hull(a).cpu().numpy()
    wb = cch.hull(b).cpu().numpy()
    assert int(ca.item()) == len(wa) and np.array_equal(oa[:len(wa)].cpu().numpy(), wa)
    assert int(cb.item()) == len(wb) and np.array_equal(ob[:len(wb)].cpu().numpy(), wb)
    # the same inputs again, in the other order, on the kept array contents
    ob2, cb2 = _noalloc(b, stream)
    oa2, ca2 = _noalloc(a, stream)
    torch.cuda.synchronize()
    assert np.array_equal(oa2[:int(ca2.item())].cpu().numpy(), wa)
    assert np.array_equal(ob2[:int(cb2.item())].cpu().numpy(), wb)


def test_noalloc_rejects_sets_above_its_limit():
    t = torch.zeros((131_073, 2), dtype=torch.float64, device=DEV)
    o = torch.zeros(131_073, dtype=torch.int32, device=DEV)
    c = torch.zeros(1, dtype=torch.int32, device=DEV)
    rc = cch.lib().cch_hull_noalloc(t.data_ptr(), 131_073, cch.CCH_F64, o.data_ptr(), c.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == -4


def test_noalloc_many_calls_of_mixed_sizes_across_the_epoch_wrap():
    """4200 calls on one stream, cycling through sizes that use different
    parts of the shared array -- a small float64 disk, the largest size as an
    all-extreme circle (multi-block sort, SPA and chain look-backs), a mid
    int32 square and an empty set -- so that the look-back epoch wraps (every
    4095 calls) while smaller and larger calls alternate.  Every result must
    equal cch_hull's on the same input."""
    stream = torch.cuda.current_stream()
    cases = [torch.from_numpy(inputs.disk_f64(5_000, 51)).to(DEV),
             torch.from_numpy(inputs.circle_f64(131_072, 52)).to(DEV),
             torch.from_numpy(inputs.square_i32(40_000, 53)).to(DEV),
             torch.zeros((0, 2), dtype=torch.float64, device=DEV)]
    want = [cch.hull(t) if t.shape[0] else torch.zeros(0, dtype=torch.int32, device=DEV) for t in cases]
    slots = 64
    outs = torch.full((slots, 131_072), -7, dtype=torch.int32, device=DEV)
    cnts = torch.full((slots,), -7, dtype=torch.int32, device=DEV)
    lib = cch.lib()
    calls = 4200
    for i0 in range(0, calls, slots):
        used = []
        cnts.fill_(-7)            # a call that writes no count cannot pass on an earlier one's
        for k in range(min(slots, calls - i0)):
            c = (i0 + k) % len(cases)
            t = cases[c]
            n = t.shape[0]
            dt = cch.CCH_F64 if t.dtype == torch.float64 else cch.CCH_I32
            rc = lib.cch_hull_noalloc(t.data_ptr() if n else None, n, dt, outs[k].data_ptr(),
                                      cnts[k:k + 1].data_ptr(), stream.cuda_stream)
            assert rc == 0, (i0 + k, rc)
            used.append(c)
        torch.cuda.synchronize()
        got_counts = cnts.cpu().tolist()
        for k, c in enumerate(used):
            h = got_counts[k]
            assert h >= 0, (i0 + k, lib.cch_status_string(h))
            assert h == want[c].shape[0], (i0 + k, c, h, want[c].shape[0])
            assert torch.equal(outs[k, :h], want[c]), (i0 + k, c)

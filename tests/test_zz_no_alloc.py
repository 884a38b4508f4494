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

"""Every run-time choice the tuner can make returns the oracle's hulls: the
batched path under each candidate value of each choice, and after the
tuner has picked its own."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1508_05488_gb300 as cch
from paper_1508_05488_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CANDIDATES = [dict(small_max=v) for v in (16384, 8192, 4096, 1)] + \
             [dict(stair_div=d, stair_min=a, stair_max=b) for d, a, b in
              ((16, 8192, 1 << 20), (32, 4096, 1 << 19), (8, 16384, 1 << 21), (64, 2048, 1 << 18), (1, 1, 1))] + \
             [dict(a1_len_min=v) for v in (4096, 16384, 65536, 262144)] + [dict(cls_per_sm=v) for v in (1, 2)]


def _batch(dtype, seed):
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(200), np.log(120_000), 60))).astype(np.int64)
    sizes[:3] = (0, 1, 3)
    sets = []
    for i, n in enumerate(sizes):
        if dtype == np.int32:
            sets.append(inputs.square_i32(int(n), seed + i) if i % 2 else inputs.disk_i32(int(n), seed + i))
        else:
            sets.append(inputs.disk_f64(int(n), seed + i) if i % 2 else inputs.gauss_f64(int(n), seed + i))
    off = np.concatenate([[0], np.cumsum([len(s) for s in sets])]).astype(np.int64)
    return sets, np.concatenate(sets).astype(dtype), off


@pytest.mark.parametrize("dtype", [np.int32, np.float64])
def test_every_tuned_choice_returns_the_oracle_hulls(dtype):
    sets, pts, off = _batch(dtype, 41 if dtype == np.int32 else 42)
    want = [oracle.hull(s) for s in sets]
    code = cch.CCH_I32 if dtype == np.int32 else cch.CCH_F64
    bucket = cch.lib().cch_tune_bucket(int(off[-1]), len(sets))
    d = torch.from_numpy(pts).to(DEV)
    base, _ = cch.tune_get(code, True, bucket)
    try:
        for cand in CANDIDATES:
            cch.tune_set(dict(base, **cand), code, True, bucket)
            got = cch.hull_batched(d, off)
            for s, w in enumerate(want):
                assert np.array_equal(got[s].cpu().numpy(), w), (cand, s)
        best = cch.autotune_batched(d, off, reps=1)
        got, found = cch.tune_get(code, True, bucket)
        assert found and got == best
        got = cch.hull_batched(d, off)
        for s, w in enumerate(want):
            assert np.array_equal(got[s].cpu().numpy(), w), ("tuned", s)
    finally:
        cch.lib().cch_tune_clear()

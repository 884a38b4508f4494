"""Parity at the benchmark sizes: the hulls of the full 20M-point float64
sets the benchmark times (uniform square, unit disk, Gaussian), the 20M
degenerate stress set, the 2M all-extreme circle and the 1M int32 set,
computed through the same entry point the benchmark calls, compared element
by element with the CPU oracle's hull of the whole set."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1508_05488_gb300 as cch
from paper_1508_05488_gb300 import inputs

pytestmark = pytest.mark.gpu

CONFIGS = {
    "square20M": lambda: inputs.headline_f64("square"),
    "disk20M": lambda: inputs.headline_f64("disk"),
    "gauss20M": lambda: inputs.headline_f64("gauss"),
    "degenerate20M": lambda: inputs.degenerate_f64(20_000_000, 5),
    "circle2M": lambda: inputs.circle_f64(2_000_000, 6),
    "int32_1M": lambda: inputs.square_i32(1_000_000, 1),
}


@pytest.mark.parametrize("name", list(CONFIGS))
def test_full_size_hull_equals_oracle(name):
    p = CONFIGS[name]()
    t = torch.from_numpy(p).to("cuda:0")
    idx, cnt = cch.hull_async(t)
    torch.cuda.synchronize()
    got = idx[:int(cnt.item())].cpu().numpy()
    want = oracle.hull(p)
    assert np.array_equal(got, want), (name, len(got), len(want))
    if name == "circle2M":
        assert len(got) == 2_000_000

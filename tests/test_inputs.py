"""The seeded generators: SplitMix64 against its published first outputs."""
import os

import numpy as np

from paper_2001_04886_gb300 import inputs


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: the first outputs published with the generator
    # (tests/golden/splitmix64_seed0.txt carries the values and their source)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64_seed0.txt")
    want = [int(ln, 16) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(want) == 3
    z = inputs.splitmix64(0, len(want))
    assert [int(v) for v in z] == want


def test_offsets_and_ranges():
    a = inputs.uniform01(7, 100)
    b = inputs.uniform01(7, 60, offset=40)
    assert np.array_equal(a[40:], b)
    x = inputs.x_true(3, 10000)
    assert x.min() >= -1.0 and x.max() < 1.0 and abs(x.mean()) < 0.05


def test_batched_draws():
    sy = inputs.batched_systems(0, 512)
    Ls = np.array([d["L"] for d in sy])
    bs = np.array([d["beta"] for d in sy])
    assert Ls.min() >= 32 and Ls.max() <= 256 and bs.min() >= 0 and bs.max() < 50
    assert sy[:5] == inputs.batched_systems(0, 5)

"""The seeded generators: SplitMix64 against its published first outputs."""
import numpy as np

from paper_2001_04886_gb300 import inputs


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: first outputs as published with the reference
    # C implementation (Steele, Lea, Flood 2014; also Vigna's splitmix64.c).
    z = inputs.splitmix64(0, 3)
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4
    assert int(z[2]) == 0x06C45D188009454F


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

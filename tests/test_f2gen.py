"""The seeded input generator: published SplitMix64 outputs, layouts, shapes."""
import os

import numpy as np
import pytest

import f2gen


def test_splitmix64_reference_outputs():
    with open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")) as f:
        want = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    got = [int(x) for x in f2gen.draws(0, 0, len(want))]
    assert got == want
    assert f2gen.mix64_int(0x9E3779B97F4A7C15) == want[0]


@pytest.mark.parametrize("n,m", [(1, 1), (7, 64), (65, 65), (100, 130), (3, 200)])
def test_uniform_shape_padding_determinism(n, m):
    a = f2gen.uniform(n, m, 7)
    b = f2gen.uniform(n, m, 7)
    assert a.shape == (n, (m + 63) // 64) and a.dtype == np.uint64
    assert np.array_equal(a, b)
    assert not np.array_equal(a, f2gen.uniform(n, m, 8)) or n * m < 4
    if m % 64:
        assert not (a[:, -1] & ~f2gen.pad_mask(m)).any()


def test_densities():
    a = f2gen.unpack_bits(f2gen.uniform(300, 300, 1), 300)
    assert abs(a.mean() - 0.5) < 0.01
    b = f2gen.unpack_bits(f2gen.bernoulli(300, 300, 0.1, 1), 300)
    assert abs(b.mean() - 0.1) < 0.01
    s = f2gen.unpack_bits(f2gen.sparse_rows(200, 300, 7, 1), 300)
    assert (s.sum(axis=1) == 7).all()


def test_layouts_round_trip():
    a = f2gen.uniform(37, 200, 3)
    cb = f2gen.to_colblocks(a, ld=40)
    assert cb.shape == (4, 40)
    assert int(cb[2, 5]) == int(a[5, 2])
    assert np.array_equal(f2gen.from_colblocks(cb, 37), a)
    bits = f2gen.unpack_bits(a, 200)
    assert np.array_equal(f2gen.pack_bits(bits), a)
    for b in (1, 3, 8, 33):
        assert np.array_equal(f2gen.unpack_bits(f2gen.pack_bits(bits, b), 200, b), bits)


def test_fixed_rank_factor_shapes():
    X, Y = f2gen.fixed_rank_factors(50, 70, 20, 1)
    assert X.shape == (50, 1) and Y.shape == (20, 2)
    assert not (Y[:, -1] & ~f2gen.pad_mask(70)).any()

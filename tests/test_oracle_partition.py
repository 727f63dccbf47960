"""Pins of the oracle's sample-sort partition (Section 2's sample sorts with
regularly chosen splitters; the routing is one stable count-sort round on the
key's range). Checked against numpy (searchsorted for the ranges, a stable
argsort for the routing), against invariants, on ties with splitters and
repeated splitters, and a planted mistake (strict comparison) must fail."""
import numpy as np
import pytest

import gen
import oracle


def expected(keys, vals, sample, parts):
    m = sample.size
    spl = np.array([sample[(j * m) // parts] for j in range(1, parts)], dtype=keys.dtype)
    rng = np.searchsorted(spl, keys, side="right")
    order = np.argsort(rng, kind="stable")
    counts = np.bincount(rng, minlength=parts).astype(np.uint64)
    return keys[order], (None if vals is None else vals[order]), counts, spl


@pytest.mark.parametrize("dtype,bits", [(np.uint32, 32), (np.uint64, 64), (np.uint32, 12)])
@pytest.mark.parametrize("parts,m", [(1, 0), (2, 1), (2, 64), (3, 100), (8, 512), (256, 4096), (7, 5)])
def test_partition_matches_numpy(dtype, bits, parts, m):
    n = 20_011
    keys = (gen.uniform_u32(n, bits, 41, 0) if dtype == np.uint32 else gen.uniform_u64(n, bits, 41, 0))
    vals = np.arange(n, dtype=np.uint32)
    sample = np.sort(keys[np.random.default_rng(3).integers(0, n, m)]) if m else keys[:0]
    k, v, c = oracle.partition(keys, vals, sample, parts)
    ek, ev, ec, spl = expected(keys, vals, sample, parts)
    assert np.array_equal(k, ek) and np.array_equal(v, ev) and np.array_equal(c, ec)
    # invariants: counts add up; range r holds keys in [spl[r-1], spl[r])
    assert int(c.sum()) == n
    start = 0
    for r in range(parts):
        part = k[start:start + int(c[r])]
        if r > 0:
            assert np.all(part >= spl[r - 1])
        if r < parts - 1:
            assert np.all(part < spl[r])
        # stable within a range: payloads increase
        assert np.all(np.diff(v[start:start + int(c[r])].astype(np.int64)) > 0)
        start += int(c[r])


def test_ties_with_splitters_and_repeated_splitters():
    keys = np.array([5, 3, 5, 9, 5, 1, 7, 5], dtype=np.uint32)
    vals = np.arange(keys.size, dtype=np.uint32)
    sample = np.array([5, 5, 5, 5], dtype=np.uint32)  # every splitter is 5
    k, v, c = oracle.partition(keys, vals, sample, 4)
    # ranges: < 5 -> 0; >= 5 -> 3 (ranges 1 and 2 are empty); ties keep input order
    assert c.tolist() == [2, 0, 0, 6]
    assert k.tolist() == [3, 1, 5, 5, 9, 5, 7, 5] and v.tolist() == [1, 5, 0, 2, 3, 4, 6, 7]


def test_one_range_is_identity():
    keys = gen.uniform_u32(1000, 32, 42, 0)
    k, v, c = oracle.partition(keys, None, keys[:0], 1)
    assert np.array_equal(k, keys) and v is None and c.tolist() == [1000]


def test_bad_arguments():
    keys = np.arange(10, dtype=np.uint32)
    with pytest.raises(ValueError):
        oracle.partition(keys, None, keys[:0], 2)  # splitters need a sample
    with pytest.raises(ValueError):
        oracle.partition(keys, None, keys, 257)


def test_planted_strict_comparison_is_caught():
    keys = np.array([5, 3, 5, 9], dtype=np.uint32)
    sample = np.array([5, 5], dtype=np.uint32)
    good = oracle.partition(keys, None, sample, 2)
    bad = oracle.partition(keys, None, sample, 2, mutant=7)
    ek, _, ec, _ = expected(keys, None, sample, 2)
    assert np.array_equal(good[0], ek) and np.array_equal(good[2], ec)
    assert not np.array_equal(bad[2], ec)

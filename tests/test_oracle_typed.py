"""Pins for the oracle's typed-key sort (signed integers by value, floats by
IEEE 754 totalOrder): against numpy's stable argsort where the two orders
agree (integers; floats without zeros or NaNs); against the order of the
special encodings written out from the IEEE 754 binary formats; stability
among equal keys and among zeros of either sign."""
import numpy as np
import pytest

import oracle


def _stable(keys):
    idx = np.argsort(keys, kind="stable")
    return keys[idx], idx.astype(np.uint32)


@pytest.mark.parametrize("dt", [np.int32, np.int64])
@pytest.mark.parametrize("n", [0, 1, 2, 1000, 100_003])
def test_signed_integers_match_numpy(dt, n):
    r = np.random.default_rng(n)
    info = np.iinfo(dt)
    keys = r.integers(info.min, info.max, n, dtype=dt, endpoint=True)
    if n > 10:
        keys[::3] = keys[1]
        keys[:4] = [info.min, info.max, -1, 0]
    k, v = oracle.sort_typed(keys, np.arange(n, dtype=np.uint32))
    ek, ev = _stable(keys)
    assert np.array_equal(k, ek) and np.array_equal(v, ev)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_floats_without_zeros_or_nans_match_numpy(dt):
    r = np.random.default_rng(7)
    n = 50_001
    keys = (r.standard_normal(n) * np.exp(r.uniform(-40, 40, n))).astype(dt)
    keys[keys == 0] = 1
    keys[::4] = keys[9]
    keys[:2] = [np.inf, -np.inf]
    k, v = oracle.sort_typed(keys, np.arange(n, dtype=np.uint32))
    ek, ev = _stable(keys)
    assert np.array_equal(k, ek) and np.array_equal(v, ev)


F32_ORDER = [0xFFC00000, 0xFF800001, 0xFF800000, 0xFF7FFFFF, 0xBF800000, 0x80800000, 0x80000001, 0x80000000,
             0x00000000, 0x00000001, 0x00800000, 0x3F800000, 0x7F7FFFFF, 0x7F800000, 0x7F800001, 0x7FC00000]
F64_ORDER = [0xFFF8000000000000, 0xFFF0000000000001, 0xFFF0000000000000, 0xFFEFFFFFFFFFFFFF, 0xBFF0000000000000,
             0x8000000000000001, 0x8000000000000000, 0x0000000000000000, 0x0000000000000001, 0x3FF0000000000000,
             0x7FEFFFFFFFFFFFFF, 0x7FF0000000000000, 0x7FF0000000000001, 0x7FF8000000000000]


@pytest.mark.parametrize("order,ut,ft", [(F32_ORDER, np.uint32, np.float32), (F64_ORDER, np.uint64, np.float64)])
def test_special_encodings_in_total_order(order, ut, ft):
    """-qNaN < -sNaN < -Inf < -max < -1 < -min normal < -min subnormal < -0
    < +0 < +min subnormal < ... < +Inf < +sNaN < +qNaN."""
    bits = np.array(order, dtype=ut)
    r = np.random.default_rng(3)
    for _ in range(5):
        perm = r.permutation(bits.size)
        k, v = oracle.sort_typed(bits[perm].view(ft), np.arange(bits.size, dtype=np.uint32))
        assert np.array_equal(k.view(ut), bits)
        assert np.array_equal(perm[v], np.arange(bits.size))


def test_zeros_of_both_signs_are_stable():
    keys = np.array([0.0, -0.0, 0.0, -0.0, 1.0, -0.0], np.float32)
    k, v = oracle.sort_typed(keys, np.arange(6, dtype=np.uint32))
    assert np.array_equal(v, [1, 3, 5, 0, 2, 4])
    assert np.array_equal(np.signbit(k), [True, True, True, False, False, False])

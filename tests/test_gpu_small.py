"""GPU parity of BTN and OET against the oracle (bit-exact), including the
stage counts the paper states: lg p (lg p + 1)/2 merge-split stages for BTN and
p rounds for OET (Section 2)."""
import math

import numpy as np
import pytest

import gen
import oracle
from gen import workloads
from tests._util import to_dev, to_np

pytestmark = pytest.mark.gpu


def run(isort, fn, keys, vals, p=None):
    import torch

    tk = to_dev(keys)
    tv = None if vals is None else to_dev(vals)
    out = getattr(isort, fn)(tk, tv, p)
    torch.cuda.synchronize()
    stages = out[2] if p is not None else None
    return to_np(tk, np.uint32), (None if vals is None else to_np(tv, np.uint32)), stages


@pytest.mark.parametrize("fn", ["btn", "oet"])
def test_first_1024_of_small_uniform(cuda_lib, fn):
    keys = workloads.small_uniform()[: workloads.SMALL_BTN_N].copy()
    rk, _ = oracle.lsd(keys, None, 32, 8)
    ok, _, _ = run(cuda_lib, fn, keys, None)
    assert np.array_equal(ok, rk)
    vals = np.arange(keys.size, dtype=np.uint32)
    ok, ov, _ = run(cuda_lib, fn, keys, vals)
    rk, rv = oracle.lsd(keys, vals, 32, 8)
    assert np.array_equal(ok, rk) and np.array_equal(ov, rv)


@pytest.mark.parametrize("p", [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024])
def test_btn_stage_count_and_result(cuda_lib, p):
    lg = int(math.log2(p))
    for n in sorted({1, 2, p, p + 1, 3 * p - 1, min(8 * p, 16384), min(32 * p, 16384)}):
        if n > 32 * p or (p > 512 and n > 16 * p):
            continue
        keys = gen.uniform_u32(n, 6, n + p, 0)  # heavy ties: stability matters
        vals = np.arange(n, dtype=np.uint32)
        ok, ov, st = run(cuda_lib, "btn", keys, vals, p)
        rk, rv = oracle.lsd(keys, vals, 32, 8)
        assert np.array_equal(ok, rk) and np.array_equal(ov, rv), (p, n)
        assert st == lg * (lg + 1) // 2
        bk, bv, bst = oracle.btn(keys, vals, p)
        assert bst == st and np.array_equal(bk, ok) and np.array_equal(bv, ov)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 31, 32, 33, 100, 128, 256])
def test_oet_round_count_and_result(cuda_lib, p):
    for n in sorted({1, 2, p, p + 1, 4 * p - 3, min(16 * p, 16384)}):
        if n > 32 * p:
            continue
        keys = np.sort(gen.uniform_u32(n, 32, n + 3 * p, 0))[::-1].copy()  # reverse: transposition's worst case
        keys[: n // 3] = 77
        vals = np.arange(n, dtype=np.uint32)
        ok, ov, st = run(cuda_lib, "oet", keys, vals, p)
        rk, rv = oracle.lsd(keys, vals, 32, 8)
        assert np.array_equal(ok, rk) and np.array_equal(ov, rv), (p, n)
        assert st == p
        ek, ev, est = oracle.oet(keys, vals, p)
        assert est == st and np.array_equal(ek, ok)


@pytest.mark.parametrize("fn", ["btn", "oet"])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 33, 1000, 4096, 4097, 10_000, 16_384])
def test_default_p_sizes(cuda_lib, fn, n):
    keys = gen.uniform_u32(n, 32, 40 + n, 0) if n else np.zeros(0, np.uint32)
    if n > 2:
        keys[1] = 0xFFFFFFFF
    vals = np.arange(n, dtype=np.uint32)
    if n == 0:
        return
    ok, ov, _ = run(cuda_lib, fn, keys, vals)
    rk, rv = oracle.lsd(keys, vals, 32, 8)
    assert np.array_equal(ok, rk) and np.array_equal(ov, rv)


def test_too_large_is_unsupported(cuda_lib):
    tk = to_dev(np.zeros(16_385, np.uint32))
    with pytest.raises(cuda_lib.IsortError) as e:
        cuda_lib.btn(tk)
    assert e.value.code == cuda_lib.UNSUPPORTED

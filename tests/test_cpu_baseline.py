"""The multicore CPU baseline (parallel radix sort, BTN and OET on host
threads) against the serial oracle: the same stable result, bit for bit."""
import numpy as np
import pytest

import cpu_baseline
import gen
import oracle


@pytest.mark.parametrize("n,key_bits,rb,threads", [
    (1, 32, 8, 4), (2, 32, 8, 4), (1000, 32, 8, 3), (100_003, 32, 8, 8), (100_003, 32, 11, 5),
    (65_537, 20, 8, 4), (65_537, 20, 11, 7), (50_000, 32, 16, 4), (12_345, 7, 3, 16)])
def test_pr_sort_u32_matches_oracle(n, key_bits, rb, threads):
    keys = gen.uniform_u32(n, key_bits, 31, 0)
    keys[: n // 5] = keys[n // 3]  # ties: stability
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.lsd(keys, vals, key_bits, rb)
    k, v = keys.copy(), vals.copy()
    cpu_baseline.pr_sort(k, v, key_bits, rb, threads)
    assert np.array_equal(k, ek) and np.array_equal(v, ev)
    k = keys.copy()
    cpu_baseline.pr_sort(k, None, key_bits, rb, threads)
    assert np.array_equal(k, ek)


@pytest.mark.parametrize("n,key_bits,rb,threads", [(77_777, 64, 8, 6), (77_777, 48, 8, 3), (9_999, 40, 13, 4)])
def test_pr_sort_u64_matches_oracle(n, key_bits, rb, threads):
    keys = gen.uniform_u64(n, key_bits, 32, 0)
    keys[::7] = keys[5]
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.lsd(keys, vals, key_bits, rb)
    k, v = keys.copy(), vals.copy()
    cpu_baseline.pr_sort(k, v, key_bits, rb, threads)
    assert np.array_equal(k, ek) and np.array_equal(v, ev)


@pytest.mark.parametrize("fn,p", [(cpu_baseline.btn, 1), (cpu_baseline.btn, 2), (cpu_baseline.btn, 4),
                                  (cpu_baseline.btn, 8), (cpu_baseline.oet, 1), (cpu_baseline.oet, 3),
                                  (cpu_baseline.oet, 4), (cpu_baseline.oet, 7)])
@pytest.mark.parametrize("n", [1, 2, 5, 1000, 1024, 4099])
def test_block_networks_match_oracle(fn, p, n):
    keys = gen.uniform_u32(n, 32, 33, 0)
    keys[: n // 4] = 0xFFFFFFFF  # ties with the padding key
    vals = np.arange(100, 100 + n, dtype=np.uint32)  # payload is not the index
    ek, ev = oracle.lsd(keys, vals, 32, 8)
    k, v = keys.copy(), vals.copy()
    fn(k, v, p)
    assert np.array_equal(k, ek) and np.array_equal(v, ev)


def test_btn_rejects_non_power_of_two():
    k = np.arange(10, dtype=np.uint32)
    with pytest.raises(ValueError):
        cpu_baseline.btn(k, None, 3)

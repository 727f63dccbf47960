"""The allocation-free radix entry point (isort_radix_noalloc), called through
the C ABI.

Some callers cannot let a library allocate device memory (for example a
process whose device memory is reserved up front by another allocator). This
entry point takes its scratch from a fixed array the library declares in
device memory.
The tests check its output against the ordinary isort_radix and against the
serial oracle, bit for bit, on calls made one after another (the shared array
keeps the previous call's contents, so later calls also show that what must
start cleared is cleared), over every branch of the buffer plan (one round,
an odd and an even number of rounds), and that sizes beyond the array's
limit are refused. This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle
from tests._util import to_dev, to_np

pytestmark = pytest.mark.gpu

MAX_KEYS = 1 << 18


def reference_sort(lib, keys, vals, key_bits, rb, stream):
    tk = to_dev(keys)
    tv = None if vals is None else to_dev(vals)
    rc = lib.isort_radix(ctypes.c_void_p(tk.data_ptr()), None if tv is None else ctypes.c_void_p(tv.data_ptr()),
                         keys.size, key_bits, rb, stream)
    assert rc == 0
    return tk, tv


def noalloc_sort(cuda_lib, lib, keys, vals, key_bits, rb, stream):
    import torch

    tk = to_dev(keys)
    tv = None if vals is None else to_dev(vals)
    rc = lib.isort_radix_noalloc(ctypes.c_void_p(tk.data_ptr()),
                                 None if tv is None else ctypes.c_void_p(tv.data_ptr()), keys.size, key_bits, rb,
                                 stream)
    assert rc == 0, cuda_lib.STATUS.get(rc, rc)
    torch.cuda.synchronize()
    return tk, tv


# (n, key_bits, radix_bits, seed): 4 rounds, 4 rounds, then 3, 7 and 1 round
# (the odd-round ping-pong and the single-round copy back), at the array's
# maximum size and at odd sizes
CASES = [(MAX_KEYS, 32, 8, 81), (100_003, 20, 5, 82), (MAX_KEYS, 24, 8, 84), (77_777, 32, 5, 85),
         (MAX_KEYS, 8, 8, 86), (99_999, 8, 8, 87), (131_071, 24, 8, 88)]


def test_noalloc_matches_isort_radix_and_oracle(cuda_lib):
    import torch

    lib = cuda_lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, key_bits, rb, seed in CASES:  # calls one after another on the shared array
        keys = gen.uniform_u32(n, key_bits, seed, 0)
        keys[: n // 7] = keys[n // 2]  # ties: stability matters
        vals = np.arange(n, dtype=np.uint32)
        ok, ov = oracle.lsd(keys, vals, key_bits, rb)
        rk, rv = reference_sort(lib, keys, vals, key_bits, rb, stream)
        tk, tv = noalloc_sort(cuda_lib, lib, keys, vals, key_bits, rb, stream)
        gk, gv = to_np(tk, np.uint32), to_np(tv, np.uint32)
        assert np.array_equal(gk, ok) and np.array_equal(gv, ov), (n, key_bits, rb)
        assert np.array_equal(gk, to_np(rk, np.uint32)) and np.array_equal(gv, to_np(rv, np.uint32))


def test_noalloc_keys_only_and_limits(cuda_lib):
    import torch

    lib = cuda_lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, key_bits, rb, seed in [(5000, 32, 8, 83), (MAX_KEYS, 24, 8, 89)]:
        keys = gen.uniform_u32(n, key_bits, seed, 0)
        ok, _ = oracle.lsd(keys, None, key_bits, rb)
        tk, _ = noalloc_sort(cuda_lib, lib, keys, None, key_bits, rb, stream)
        rk, _ = reference_sort(lib, keys, None, key_bits, rb, stream)
        assert np.array_equal(to_np(tk, np.uint32), ok)
        assert np.array_equal(to_np(tk, np.uint32), to_np(rk, np.uint32))
    # beyond the fixed array's limits: refused before any work
    small = to_dev(np.zeros(5000, np.uint32))
    big = to_dev(np.zeros(MAX_KEYS + 1, np.uint32))
    assert lib.isort_radix_noalloc(ctypes.c_void_p(big.data_ptr()), None, MAX_KEYS + 1, 32, 8, stream) == 6
    assert lib.isort_radix_noalloc(ctypes.c_void_p(small.data_ptr()), None, 5000, 32, 11, stream) == 6


def test_noalloc_key_range_error_matches_isort_radix(cuda_lib):
    """A key above the declared range: the same status as isort_radix, buffers untouched."""
    import torch

    lib = cuda_lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    keys = gen.uniform_u32(10_001, 16, 90, 0)
    keys[5000] = 1 << 20
    tk = to_dev(keys)
    rc = lib.isort_radix_noalloc(ctypes.c_void_p(tk.data_ptr()), None, keys.size, 16, 8, stream)
    rk = to_dev(keys)
    rc_ref = lib.isort_radix(ctypes.c_void_p(rk.data_ptr()), None, keys.size, 16, 8, stream)
    torch.cuda.synchronize()
    assert rc == rc_ref == 2
    assert np.array_equal(to_np(tk, np.uint32), keys)

"""The allocation-free radix entry point (isort_radix_noalloc), called through
the C ABI.

Some callers cannot let a library allocate device memory (for example code
running while a global-mode stream capture is in progress, or a process whose
device memory is reserved up front by another allocator). This entry point
takes its scratch from a fixed array the library declares in device memory.
The test checks its output against the ordinary isort_radix on two calls in a
row (the shared array keeps the previous call's contents, so the second call
also shows that what must start cleared is cleared), and that sizes beyond
the array's limit are refused. This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import gen
from tests._util import to_dev, to_np

pytestmark = pytest.mark.gpu

MAX_KEYS = 1 << 18


def reference_sort(lib, keys, vals, key_bits, rb, stream):
    tk, tv = to_dev(keys), to_dev(vals)
    rc = lib.isort_radix(ctypes.c_void_p(tk.data_ptr()), ctypes.c_void_p(tv.data_ptr()), keys.size, key_bits, rb,
                         stream)
    assert rc == 0
    return tk, tv


def test_noalloc_matches_isort_radix_twice(cuda_lib):
    import torch

    lib = cuda_lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(MAX_KEYS, 32, 8, 81), (100_003, 20, 5, 82)]  # two calls in a row, different sizes and widths
    for n, key_bits, rb, seed in cases:
        keys = gen.uniform_u32(n, key_bits, seed, 0)
        keys[: n // 7] = keys[n // 2]  # ties: stability matters
        vals = np.arange(n, dtype=np.uint32)
        rk, rv = reference_sort(lib, keys, vals, key_bits, rb, stream)
        tk, tv = to_dev(keys), to_dev(vals)
        rc = lib.isort_radix_noalloc(ctypes.c_void_p(tk.data_ptr()), ctypes.c_void_p(tv.data_ptr()), n, key_bits,
                                     rb, stream)
        assert rc == 0, cuda_lib.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        assert np.array_equal(to_np(tk, np.uint32), to_np(rk, np.uint32))
        assert np.array_equal(to_np(tv, np.uint32), to_np(rv, np.uint32))


def test_noalloc_keys_only_and_limits(cuda_lib):
    import torch

    lib = cuda_lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = 5000
    keys = gen.uniform_u32(n, 32, 83, 0)
    tk = to_dev(keys)
    assert lib.isort_radix_noalloc(ctypes.c_void_p(tk.data_ptr()), None, n, 32, 8, stream) == 0
    torch.cuda.synchronize()
    assert np.array_equal(to_np(tk, np.uint32), np.sort(keys))
    # beyond the fixed array's limits: refused before any work
    big = to_dev(np.zeros(MAX_KEYS + 1, np.uint32))
    assert lib.isort_radix_noalloc(ctypes.c_void_p(big.data_ptr()), None, MAX_KEYS + 1, 32, 8, stream) == 6
    assert lib.isort_radix_noalloc(ctypes.c_void_p(tk.data_ptr()), None, n, 32, 11, stream) == 6

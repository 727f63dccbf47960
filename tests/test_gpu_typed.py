"""Typed keys on the GPU (signed integers, IEEE 754 floats) against the
oracle's merge sort by the type's order, bit for bit (payload = input index,
so stability is checked): random values of every magnitude, runs of equal
keys, zeros of both signs, infinities and NaNs with payload bits, ragged sizes
over several tiles, keys-only and pairs, radix 2^8, 2^11 and 2^16; and the
integer / float boundaries of each type."""
import numpy as np
import pytest

import gen
import oracle
from tests._util import to_np

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    a = np.ascontiguousarray(a)
    view = np.int32 if a.itemsize == 4 else np.int64
    return torch.from_numpy(a.view(view).copy()).cuda()


def _keys(kind, n, seed):
    r = np.random.default_rng(seed)
    if kind in ("i32", "i64"):
        dt = np.int32 if kind == "i32" else np.int64
        info = np.iinfo(dt)
        k = r.integers(info.min, info.max, n, dtype=dt, endpoint=True)
        k[::7] = k[min(3, n - 1)]
        k[1::11] = r.integers(-5, 5, k[1::11].size)
        k[:4] = np.array([info.min, info.max, -1, 0], dtype=dt)[: min(4, n)]
        return k
    dt, ut = (np.float32, np.uint32) if kind == "f32" else (np.float64, np.uint64)
    k = (r.standard_normal(n) * np.exp(r.uniform(-30, 30, n))).astype(dt)
    k[::9] = k[min(4, n - 1)]
    k[2::13] = 0.0
    k[3::13] = -0.0
    k[5::17] = np.inf
    k[6::17] = -np.inf
    bits = k.view(ut)
    nan = (0x7FC00000 if kind == "f32" else 0x7FF8000000000000)
    sign = (1 << 31) if kind == "f32" else (1 << 63)
    bits[7::19] = nan
    bits[8::19] = nan | sign
    bits[9::23] = nan | 12345  # a NaN with payload bits
    return k


@pytest.mark.parametrize("kind", ["i32", "f32", "i64", "f64"])
@pytest.mark.parametrize("n", [2, 1000, 3 * 4096 + 17, 200_003])
@pytest.mark.parametrize("rb", [8, 11, 16])
def test_typed_matches_oracle(cuda_lib, kind, n, rb):
    keys = _keys(kind, n, n + rb)
    vals = gen.iota_u32(n)
    ek, ev = oracle.sort_typed(keys, vals)
    dk, dv = _dev(keys), _dev(vals)
    cuda_lib.radix_typed(dk, kind, dv, rb)
    ut = np.uint32 if keys.itemsize == 4 else np.uint64
    assert np.array_equal(to_np(dk, ut), ek.view(ut))
    assert np.array_equal(to_np(dv, np.uint32), ev)
    dk = _dev(keys)
    cuda_lib.radix_typed(dk, kind, None, rb)
    assert np.array_equal(to_np(dk, ut), ek.view(ut))


@pytest.mark.parametrize("kind", ["u32", "u64"])
def test_unsigned_through_the_typed_call(cuda_lib, kind):
    n = 100_003
    keys = gen.uniform_u32(n, 32, 4, 0) if kind == "u32" else gen.uniform_u64(n, 64, 4, 0)
    vals = gen.iota_u32(n)
    ek, ev = oracle.lsd(keys, vals, 0, 8)
    dk, dv = _dev(keys), _dev(vals)
    cuda_lib.radix_typed(dk, kind, dv, 8)
    assert np.array_equal(to_np(dk, keys.dtype), ek) and np.array_equal(to_np(dv, np.uint32), ev)


def test_typed_large_f32_pairs(cuda_lib):
    """2^26 float32 keys of every magnitude and sign with payload = index."""
    n = 1 << 26
    keys = _keys("f32", n, 77)
    vals = gen.iota_u32(n)
    dk, dv = _dev(keys), _dev(vals)
    cuda_lib.radix_typed(dk, "f32", dv, 8)
    gk, gv = to_np(dk, np.uint32), to_np(dv, np.uint32)
    del dk, dv
    ek, ev = oracle.sort_typed(keys, vals)
    assert np.array_equal(gk, ek.view(np.uint32)) and np.array_equal(gv, ev)


def test_typed_rejects(cuda_lib):
    import torch

    k = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(TypeError):
        cuda_lib.radix_typed(k, "f64")
    with pytest.raises(ValueError):
        cuda_lib.radix_typed(k, "bf16")
    with pytest.raises(cuda_lib.IsortError):
        cuda_lib.radix_typed(k, "i32", None, 17)

"""GPU parity of the LSD radix path against the oracle (bit-exact).

Every case compares the CUDA result element by element with the serial oracle
on the same seeded input: sizes that span many tiles with a ragged tail, every
digit width the kernels take, known key ranges (fewer rounds), payloads, u64
keys, unaligned and host buffers, adversarial key sets, the error paths, and
the full-size large uniform workloads.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle
from gen import workloads
from tests._util import to_dev, to_np

pytestmark = pytest.mark.gpu

TILE = 4096


def run_radix(isort, keys, vals, key_bits, rb):
    import torch

    tk = to_dev(keys)
    tv = None if vals is None else to_dev(vals)
    isort.radix(tk, tv, key_bits, rb)
    torch.cuda.synchronize()
    ok = to_np(tk, keys.dtype)
    ov = None if vals is None else to_np(tv, np.uint32)
    return ok, ov


def check(isort, keys, vals, key_bits, rb):
    ok, ov = run_radix(isort, keys, vals, key_bits, rb)
    rk, rv = oracle.lsd(keys, vals, key_bits, rb)
    assert np.array_equal(ok, rk), f"keys differ (n={keys.size}, kb={key_bits}, rb={rb})"
    if vals is not None:
        assert np.array_equal(ov, rv), f"payload differs (n={keys.size}, kb={key_bits}, rb={rb})"


def test_small_uniform_keys_only(cuda_lib):
    """65,536 u32 keys uniform on [0,2^32), seed 1, radix 2^8: 4 rounds."""
    check(cuda_lib, workloads.small_uniform(), None, 32, 8)


SIZES = [2, 3, 31, 100, TILE - 1, TILE, TILE + 1, 3 * TILE + 17, 16 * TILE, 65537, 200_003]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("rb", [8, 11])
def test_sizes_pairs(cuda_lib, n, rb):
    keys = gen.uniform_u32(n, 32, 100 + n, 0)
    vals = np.arange(n, dtype=np.uint32)
    check(cuda_lib, keys, vals, 32, rb)


@pytest.mark.parametrize("rb", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16])
@pytest.mark.parametrize("key_bits", [32, 20, 13, 1])
def test_all_digit_widths(cuda_lib, rb, key_bits):
    n = 3 * TILE + 123
    keys = gen.uniform_u32(n, key_bits, 7 * rb + key_bits, 0)
    vals = np.arange(n, dtype=np.uint32)
    check(cuda_lib, keys, vals, key_bits, rb)
    check(cuda_lib, keys, None, key_bits, rb)


@pytest.mark.parametrize("key_bits,rb", [(64, 8), (48, 8), (64, 11), (40, 12), (33, 5), (64, 16), (48, 13)])
@pytest.mark.parametrize("n", [5000, 100_003])
def test_u64(cuda_lib, key_bits, rb, n):
    keys = gen.uniform_u64(n, key_bits, 5 + n, 0)
    keys[::7] = keys[3]  # duplicates
    vals = np.arange(n, dtype=np.uint32)
    check(cuda_lib, keys, vals, key_bits, rb)
    check(cuda_lib, keys, None, key_bits, rb)


def adversarial(n):
    r = np.random.default_rng(n)
    yield "all-equal", np.full(n, 12345, np.uint32)
    yield "all-max", np.full(n, 0xFFFFFFFF, np.uint32)
    yield "sorted", np.sort(gen.uniform_u32(n, 32, 1, 0))
    yield "reverse", np.sort(gen.uniform_u32(n, 32, 2, 0))[::-1].copy()
    yield "two-values", r.choice(np.array([0, 0xFFFFFFFF], np.uint32), n)
    yield "one-digit-differs", (np.uint32(0xABCDEF00) | (np.arange(n, dtype=np.uint32) & np.uint32(0xFF)))[::-1].copy()
    yield "zipf", gen.zipf_u32(n, 1.1, 3, 10)
    yield "lognormal", gen.lognormal_u32(n, 20.0, 2.0, 3, 11)


@pytest.mark.parametrize("rb", [8, 11])
def test_adversarial(cuda_lib, rb):
    n = 50_001
    for name, keys in adversarial(n):
        vals = np.arange(n, dtype=np.uint32)
        ok, ov = run_radix(cuda_lib, keys, vals, 32, rb)
        rk, rv = oracle.lsd(keys, vals, 32, rb)
        assert np.array_equal(ok, rk) and np.array_equal(ov, rv), name


def test_copy_keeps_inputs(cuda_lib):
    import torch

    n = 100_000
    keys = gen.uniform_u32(n, 32, 9, 0)
    vals = np.arange(n, dtype=np.uint32)
    for rb in (8, 11, 4):  # 4, 3 and 8 rounds: both buffer parities
        ki, vi = to_dev(keys), to_dev(vals)
        ko, vo = torch.empty_like(ki), torch.empty_like(vi)
        cuda_lib.radix_copy(ki, vi, ko, vo, 32, rb)
        torch.cuda.synchronize()
        rk, rv = oracle.lsd(keys, vals, 32, rb)
        assert np.array_equal(to_np(ko, np.uint32), rk) and np.array_equal(to_np(vo, np.uint32), rv)
        assert np.array_equal(to_np(ki, np.uint32), keys) and np.array_equal(to_np(vi, np.uint32), vals)


def test_unaligned_pointers(cuda_lib):
    """Buffers offset by one element take the non-bulk-copy path."""
    import torch

    n = 3 * TILE + 5
    keys = gen.uniform_u32(n + 1, 32, 11, 0)
    vals = np.arange(n + 1, dtype=np.uint32)
    tk, tv = to_dev(keys), to_dev(vals)
    lib = cuda_lib.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.isort_radix(ctypes.c_void_p(tk.data_ptr() + 4), ctypes.c_void_p(tv.data_ptr() + 4), n, 32, 8, s)
    assert rc == 0
    torch.cuda.synchronize()
    rk, rv = oracle.lsd(keys[1:], vals[1:], 32, 8)
    assert np.array_equal(to_np(tk, np.uint32)[1:], rk) and np.array_equal(to_np(tv, np.uint32)[1:], rv)
    assert to_np(tk, np.uint32)[0] == keys[0]


def test_host_buffers(cuda_lib):
    """Host (pageable numpy) buffers are staged through device memory."""
    lib = cuda_lib.load()
    n = 70_001
    keys = gen.uniform_u32(n, 32, 12, 0)
    vals = np.arange(n, dtype=np.uint32)
    k, v = keys.copy(), vals.copy()
    rc = lib.isort_radix(k.ctypes.data_as(ctypes.c_void_p), v.ctypes.data_as(ctypes.c_void_p), n, 32, 8, None)
    assert rc == 0
    rk, rv = oracle.lsd(keys, vals, 32, 8)
    assert np.array_equal(k, rk) and np.array_equal(v, rv)
    ko, vo = np.empty_like(keys), np.empty_like(vals)
    rc = lib.isort_radix_copy(keys.ctypes.data_as(ctypes.c_void_p), vals.ctypes.data_as(ctypes.c_void_p),
                              ko.ctypes.data_as(ctypes.c_void_p), vo.ctypes.data_as(ctypes.c_void_p), n, 32, 11, None)
    assert rc == 0
    assert np.array_equal(ko, rk) and np.array_equal(vo, rv)


def test_host_buffers_large_split_copies(cuda_lib):
    """Host buffers large enough for the staging copies to be cut into pieces
    on several streams: pinned (torch) and pageable (numpy), in place and out."""
    import torch

    lib = cuda_lib.load()
    n = (1 << 25) + 7
    keys = gen.uniform_u32(n, 32, 14, 0)
    vals = np.arange(n, dtype=np.uint32)
    rk, rv = oracle.lsd(keys, vals, 32, 8)
    hk = torch.from_numpy(keys.view(np.int32).copy()).pin_memory()
    hv = torch.from_numpy(vals.view(np.int32).copy()).pin_memory()
    rc = lib.isort_radix(ctypes.c_void_p(hk.data_ptr()), ctypes.c_void_p(hv.data_ptr()), n, 32, 8, None)
    assert rc == 0
    assert np.array_equal(hk.numpy().view(np.uint32), rk) and np.array_equal(hv.numpy().view(np.uint32), rv)
    ko, vo = np.empty_like(keys), np.empty_like(vals)
    rc = lib.isort_radix_copy(keys.ctypes.data_as(ctypes.c_void_p), vals.ctypes.data_as(ctypes.c_void_p),
                              ko.ctypes.data_as(ctypes.c_void_p), vo.ctypes.data_as(ctypes.c_void_p), n, 32, 8, None)
    assert rc == 0
    assert np.array_equal(ko, rk) and np.array_equal(vo, rv)


def test_host_buffers_asynchronous_calls_on_several_streams(cuda_lib):
    """Asynchronous status mode: host-to-host calls return after enqueueing,
    several are in flight on different streams (their copies and sorts
    overlap), each writes its own pinned output; all results are exact once
    the streams are done, and the device status stays clear."""
    import torch

    lib = cuda_lib.load()
    n = (1 << 24) + 3
    inputs = [gen.uniform_u32(n, 32, 40 + i, 0) for i in range(3)]
    vals = np.arange(n, dtype=np.uint32)
    hk = [torch.from_numpy(k.view(np.int32).copy()).pin_memory() for k in inputs]
    hv = torch.from_numpy(vals.view(np.int32).copy()).pin_memory()
    ko = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(6)]
    vo = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(6)]
    streams = [torch.cuda.Stream() for _ in range(3)]
    lib.isort_set_sync(0)
    try:
        for i in range(6):
            j = i % 3
            rc = lib.isort_radix_copy(ctypes.c_void_p(hk[j].data_ptr()), ctypes.c_void_p(hv.data_ptr()),
                                      ctypes.c_void_p(ko[i].data_ptr()), ctypes.c_void_p(vo[i].data_ptr()), n, 32, 8,
                                      ctypes.c_void_p(streams[j].cuda_stream))
            assert rc == 0
        torch.cuda.synchronize()
    finally:
        lib.isort_set_sync(1)
    assert lib.isort_device_status(1, None) == 0
    for j in range(3):
        rk, rv = oracle.lsd(inputs[j], vals, 32, 8)
        for i in (j, j + 3):
            assert np.array_equal(ko[i].numpy().view(np.uint32), rk)
            assert np.array_equal(vo[i].numpy().view(np.uint32), rv)


def test_key_range_violation_leaves_buffers(cuda_lib):
    import torch

    n = 20_000
    keys = gen.uniform_u32(n, 20, 13, 0)
    keys[12_345] = 1 << 20
    vals = np.arange(n, dtype=np.uint32)
    tk, tv = to_dev(keys), to_dev(vals)
    with pytest.raises(cuda_lib.IsortError) as e:
        cuda_lib.radix(tk, tv, 20, 8)
    assert e.value.code == cuda_lib.KEY_RANGE
    torch.cuda.synchronize()
    assert np.array_equal(to_np(tk, np.uint32), keys) and np.array_equal(to_np(tv, np.uint32), vals)
    # the same keys sort with the full width
    check(cuda_lib, keys, vals, 21, 8)


def test_invalid_args(cuda_lib):
    tk = to_dev(np.zeros(10, np.uint32))
    for kb, rb in ((33, 8), (32, 0), (32, 17), (-1, 8)):
        with pytest.raises(cuda_lib.IsortError) as e:
            cuda_lib.radix(tk, None, kb, rb)
        assert e.value.code == cuda_lib.INVALID_ARG


def test_tiny_n_noop(cuda_lib):
    for n in (0, 1):
        k = np.arange(n, dtype=np.uint32) + 5
        ok, _ = run_radix(cuda_lib, k, None, 32, 8)
        assert np.array_equal(ok, k)


def test_lookback_timeout_is_reported_and_recoverable(cuda_lib):
    """A tile that never publishes makes its successors' bounded waits run
    out: the call returns ISORT_ERR_TIMEOUT, and the next call works."""
    import torch

    n = 40 * TILE
    keys = gen.uniform_u32(n, 32, 14, 0)
    tk = to_dev(keys)
    cuda_lib.set_spin_limit(50_000)  # 50 ms
    try:
        cuda_lib.load().isort_debug_stall_tile(3)
        with pytest.raises(cuda_lib.IsortError) as e:
            cuda_lib.radix(tk, None, 32, 8)
        assert e.value.code == cuda_lib.TIMEOUT
    finally:
        cuda_lib.load().isort_debug_stall_tile(-1)
        cuda_lib.set_spin_limit(2_000_000)
    torch.cuda.synchronize()
    check(cuda_lib, keys, None, 32, 8)


def test_async_mode_collects_errors(cuda_lib):
    import torch

    n = 10_000
    keys = gen.uniform_u32(n, 16, 15, 0)
    keys[7] = 1 << 16
    tk = to_dev(keys)
    cuda_lib.device_status(clear=True)
    cuda_lib.set_sync(False)
    try:
        cuda_lib.radix(tk, None, 16, 8)  # returns after enqueueing
        assert cuda_lib.device_status(clear=True) == cuda_lib.KEY_RANGE
        assert cuda_lib.device_status(clear=True) == cuda_lib.OK
        t2 = to_dev(gen.uniform_u32(n, 32, 16, 0))
        cuda_lib.radix(t2, None, 32, 8)
        assert cuda_lib.device_status(clear=True) == cuda_lib.OK
    finally:
        cuda_lib.set_sync(True)
    torch.cuda.synchronize()


# ----------------------------------------------------------------- primitives


@pytest.mark.parametrize("key_bits,rb,width", [(32, 8, 32), (32, 11, 32), (20, 8, 32), (48, 8, 64), (64, 11, 64)])
def test_digit_hist(cuda_lib, key_bits, rb, width):
    n = 123_457
    keys = gen.uniform_u32(n, key_bits, 21, 0) if width == 32 else gen.uniform_u64(n, key_bits, 21, 0)
    keys[:5000] = keys[5000]  # one heavy digit
    h = cuda_lib.digit_hist(to_dev(keys), key_bits, rb)
    ref = oracle.digit_hist(keys, key_bits, rb)
    assert np.array_equal(to_np(h, np.uint32).astype(np.uint64), ref)


@pytest.mark.parametrize("shift,width", [(0, 8), (8, 8), (24, 8), (21, 11), (3, 5), (31, 1), (20, 12)])
def test_count_round(cuda_lib, shift, width):
    n = 5 * TILE + 99
    keys = gen.uniform_u32(n, 32, 22 + shift, 0)
    vals = gen.uniform_u32(n, 32, 23 + shift, 0)
    ko, vo = cuda_lib.count_round(to_dev(keys), to_dev(vals), shift, width)
    rk, rv = oracle.count_round(keys, vals, shift, width)
    assert np.array_equal(to_np(ko, np.uint32), rk) and np.array_equal(to_np(vo, np.uint32), rv)


def test_count_round_u64(cuda_lib):
    n = 3 * TILE + 1
    keys = gen.uniform_u64(n, 64, 24, 0)
    vals = np.arange(n, dtype=np.uint32)
    ko, vo = cuda_lib.count_round(to_dev(keys), to_dev(vals), 40, 8)
    rk, rv = oracle.count_round(keys, vals, 40, 8)
    assert np.array_equal(to_np(ko, np.uint64), rk) and np.array_equal(to_np(vo, np.uint32), rv)


# ----------------------------------------------------------------- full size


@pytest.fixture(scope="module")
def large_uniform():
    keys, vals = workloads.large_uniform()  # 2^28 u32 keys, seed 2, payload = index
    ref_k, ref_v = oracle.lsd(keys, vals, 32, 8)  # the stable order is unique: one oracle run serves every radix
    return keys, vals, ref_k, ref_v


@pytest.mark.parametrize("rb", [8, 11])
def test_full_size_uniform(cuda_lib, large_uniform, rb):
    """n = 2^28 u32 keys + payload through the out-of-place call the benchmark
    times; bit-exact against the oracle, plus the invariants."""
    import torch

    keys, vals, ref_k, ref_v = large_uniform
    ki, vi = to_dev(keys), to_dev(vals)
    ko, vo = torch.empty_like(ki), torch.empty_like(vi)
    cuda_lib.radix_copy(ki, vi, ko, vo, 32, rb)
    torch.cuda.synchronize()
    gk, gv = to_np(ko, np.uint32), to_np(vo, np.uint32)
    del ki, vi, ko, vo
    assert np.array_equal(gk, ref_k) and np.array_equal(gv, ref_v)
    assert oracle.is_sorted(gk) and oracle.is_stable(gk, gv)


@pytest.mark.parametrize("rb", [8, 11])
def test_full_size_range20(cuda_lib, rb):
    """n = 2^28 keys on [0,2^20) (seed 3): 3 rounds at radix 2^8, 2 at 2^11."""
    import torch

    keys, vals = workloads.large_range20()
    ki, vi = to_dev(keys), to_dev(vals)
    ko, vo = torch.empty_like(ki), torch.empty_like(vi)
    cuda_lib.radix_copy(ki, vi, ko, vo, 20, rb)
    torch.cuda.synchronize()
    gk, gv = to_np(ko, np.uint32), to_np(vo, np.uint32)
    del ki, vi, ko, vo
    assert oracle.is_sorted(gk) and oracle.is_stable(gk, gv)
    assert oracle.multiset_hash(gk, gv) == oracle.multiset_hash(keys, vals)
    assert np.array_equal(oracle.digit_hist(gk, 20, rb), oracle.digit_hist(keys, 20, rb))
    if rb == 11:
        rk, rv = oracle.lsd(keys, vals, 20, rb)
        assert np.array_equal(gk, rk) and np.array_equal(gv, rv)


@pytest.mark.parametrize("bits", [64, 48])
def test_full_size_u64(cuda_lib, bits):
    """n = 2^27 u64 keys on [0, 2^bits) + payload (seed 5): 8 or 6 rounds at
    radix 2^8, in place, bit-exact against the oracle."""
    keys, vals = workloads.wide_u64(bits=bits)
    ki, vi = to_dev(keys), to_dev(vals)
    cuda_lib.radix(ki, vi, bits, 8)
    gk, gv = to_np(ki, np.uint64), to_np(vi, np.uint32)
    del ki, vi
    ref_k, ref_v = oracle.lsd(keys, vals, bits, 8)
    assert np.array_equal(gk, ref_k) and np.array_equal(gv, ref_v)


def test_autotune_picks_a_shape_and_caches_it(cuda_lib, tmp_path):
    """With autotuning on, the sort stays bit-exact, the choice is written to
    the cache file, and a second process-level enable reads it back."""
    path = str(tmp_path / "isort_tune.txt")
    n = (1 << 21) + 3
    keys = gen.uniform_u32(n, 32, 31, 0)
    vals = np.arange(n, dtype=np.uint32)
    try:
        cuda_lib.autotune(True, path)
        check(cuda_lib, keys, vals, 32, 8)
        lines = open(path).read().split("\n")
        rows = [list(map(int, ln.split())) for ln in lines if ln.strip()]
        assert rows and rows[0][:4] == [4, 1, 0, 21]
        cuda_lib.autotune(True, path)  # reads the cache: no new line for the same kind
        check(cuda_lib, keys, vals, 32, 8)
        assert len([ln for ln in open(path).read().split("\n") if ln.strip()]) == len(rows)
    finally:
        cuda_lib.autotune(False)


@pytest.mark.parametrize("rb", [16, 13])
def test_wide_radix_against_the_paper_radix_rounds(cuda_lib, rb):
    """Radix 2^16 (and 2^13): the GPU runs each round as two stable passes
    over the halves of the digit; the oracle runs the paper's 2^16-way (2^13)
    count-sort rounds directly. Several chunks and a ragged tail."""
    n = (1 << 22) + 4097
    keys = gen.uniform_u32(n, 32, 1600 + rb, 0)
    keys[::5] = keys[11]
    vals = np.arange(n, dtype=np.uint32)
    check(cuda_lib, keys, vals, 32, rb)


def _repeated_key_sets(n):
    """Inputs with repeated keys: every round heavy (hashed Zipf ranks), only
    the upper rounds heavy (three hot upper halves over uniform lower halves),
    and long runs of one key (warps whose keys share every digit)."""
    zipf = gen.zipf_u32(n, 1.1, 21, 3)
    lo = gen.uniform_u32(n, 16, 22, 0)
    hot = np.array([0x0000, 0x7A31, 0xFFFF], np.uint32)[gen.uniform_u32(n, 32, 22, 1) % 3]
    upper = (hot << np.uint32(16)) | lo
    runs = np.repeat(gen.uniform_u32(n // 100 + 1, 32, 23, 0), 100)[:n].copy()
    return [("zipf", zipf), ("hot upper halves", upper), ("runs of 100", runs)]


@pytest.mark.parametrize("payload", [True, False])
def test_repeated_keys_both_round_forms(cuda_lib, payload):
    """Pairs at the default shape launch two forms of each round and the
    round's digit counts pick one (a digit over four times the mean: the
    per-warp form); keys only take the per-warp form, whose warps with one
    shared digit skip the mask atomics. Ragged tail, against the oracle."""
    n = 3 * (1 << 20) + 4097
    for name, keys in _repeated_key_sets(n):
        vals = np.arange(n, dtype=np.uint32) if payload else None
        ok, ov = run_radix(cuda_lib, keys, vals, 32, 8)
        rk, rv = oracle.lsd(keys, vals, 32, 8)
        assert np.array_equal(ok, rk), name
        if payload:
            assert np.array_equal(ov, rv), name


def test_round_form_choice_at_scale(cuda_lib):
    """2^26 + 4,321 pairs: on hashed Zipf(1.1) ranks every round has a heavy
    digit and the per-warp form does the rounds' work; on uniform keys the
    half-warp form does. Both against the oracle; the library's launch
    profile shows which form worked (the other returns at once)."""
    import torch

    n = (1 << 26) + 4321
    vals = np.arange(n, dtype=np.uint32)
    for name, keys, heavy in (("zipf", gen.zipf_u32(n, 1.1, 31, 0), True),
                              ("uniform", gen.uniform_u32(n, 32, 32, 0), False)):
        tk, tv = to_dev(keys), to_dev(vals)
        cuda_lib.profile_read()
        cuda_lib.profile_enable(True)
        cuda_lib.radix(tk, tv, 32, 8)
        torch.cuda.synchronize()
        cuda_lib.profile_enable(False)
        prof = cuda_lib.profile_read()
        rk, rv = oracle.lsd(keys, vals, 32, 8)
        assert np.array_equal(to_np(tk, np.uint32), rk), name
        assert np.array_equal(to_np(tv, np.uint32), rv), name
        del tk, tv
        half_ms, per_warp_ms = prof["downsweep"][1], prof["downsweep_heavy"][1]
        assert prof["downsweep"][0] == prof["downsweep_heavy"][0] == 4, name
        if heavy:
            assert per_warp_ms > 5 * half_ms, (name, prof)
        else:
            assert half_ms > 5 * per_warp_ms, (name, prof)

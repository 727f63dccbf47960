"""The sample-sort steps on the GPU against the oracle, bit for bit:
isort_sample (SplitMix64-chosen indices) and isort_partition[_u64] (stable
routing into the ranges of regularly chosen splitters, with range counts), on
ragged sizes, 1..256 ranges, ties and repeated splitters, keys only and with
payloads; argument errors; and the whole sort over one process (NCCL, world
size 1) through the library's kernels."""
import ctypes
import os
import socket

import numpy as np
import pytest

import gen
import oracle
from tests._util import to_dev, to_np

pytestmark = pytest.mark.gpu


def _keys(n, bits, u64, seed, dup=False):
    k = gen.uniform_u64(n, bits, seed, 0) if u64 else gen.uniform_u32(n, bits, seed, 0)
    if dup:
        k = k % k.dtype.type(11)
    return k


@pytest.mark.parametrize("u64", [False, True])
@pytest.mark.parametrize("n,m,seed", [(1, 5, 1), (4097, 64, 2), (1_000_003, 4096, 0x5EED5EED5EED)])
def test_sample_matches_oracle(cuda_lib, u64, n, m, seed):
    keys = _keys(n, 64 if u64 else 32, u64, 61)
    got = cuda_lib.sample(to_dev(keys), m, seed)
    ref = keys[oracle.sample_indices(n, m, seed)]
    assert np.array_equal(to_np(got, keys.dtype), ref)


@pytest.mark.parametrize("u64", [False, True])
@pytest.mark.parametrize("n,parts,bits,dup", [
    (1, 2, 32, False), (5, 3, 32, False), (4097, 8, 32, False), (100_003, 1, 32, False), (100_003, 2, 20, False),
    (100_003, 7, 32, True), (333_333, 64, 32, False), (1_000_003, 256, 32, False), (1_000_003, 8, 12, True)])
@pytest.mark.parametrize("payload", [True, False])
def test_partition_matches_oracle(cuda_lib, u64, n, parts, bits, dup, payload):
    keys = _keys(n, bits, u64, 62, dup)
    vals = np.arange(n, dtype=np.uint32) if payload else None
    smp = np.sort(keys[oracle.sample_indices(n, 64 * parts, 7)])
    ek, ev, ec = oracle.partition(keys, vals, smp, parts)
    ko, vo, c = cuda_lib.partition(to_dev(keys), None if vals is None else to_dev(vals), to_dev(smp), parts)
    assert np.array_equal(to_np(ko, keys.dtype), ek)
    if payload:
        assert np.array_equal(to_np(vo, np.uint32), ev)
    assert np.array_equal(c.cpu().numpy().astype(np.uint64), ec)


def test_partition_full_size(cuda_lib):
    n = 1 << 26
    keys = gen.uniform_u32(n, 32, 63, 0)
    vals = np.arange(n, dtype=np.uint32)
    smp = np.sort(keys[oracle.sample_indices(n, 8 * 256, 9)])
    ek, ev, ec = oracle.partition(keys, vals, smp, 8)
    ko, vo, c = cuda_lib.partition(to_dev(keys), to_dev(vals), to_dev(smp), 8)
    assert np.array_equal(to_np(ko, np.uint32), ek) and np.array_equal(to_np(vo, np.uint32), ev)
    assert np.array_equal(c.cpu().numpy().astype(np.uint64), ec)


def test_partition_argument_errors(cuda_lib):
    import torch

    lib = cuda_lib.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    k = to_dev(np.arange(100, dtype=np.uint32))
    o = torch.empty_like(k)
    smp = to_dev(np.arange(10, dtype=np.uint32))
    cnt = torch.empty(300, dtype=torch.int64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.isort_partition(p(k), None, p(o), None, 100, p(smp), 10, 0, p(cnt), s) == 1
    assert lib.isort_partition(p(k), None, p(o), None, 100, p(smp), 10, 257, p(cnt), s) == 1
    assert lib.isort_partition(p(k), None, p(o), None, 100, p(smp), 0, 4, p(cnt), s) == 1
    assert lib.isort_partition(p(k), None, p(k), None, 100, p(smp), 10, 4, p(cnt), s) == 1  # aliased output
    host = np.zeros(4, np.uint64)
    assert lib.isort_partition(p(k), None, p(o), None, 100, p(smp), 10, 4,
                               ctypes.c_void_p(host.ctypes.data), s) == 1  # host counts
    assert lib.isort_sample(p(k), 16, 100, 4, 1, p(o), s) == 1


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_sample_sort_one_process_through_the_kernels(cuda_lib):
    import torch
    import torch.distributed as dist

    from paper_1708_09495_gb300 import dist as idist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        n = 3_000_017
        keys = gen.uniform_u32(n, 32, 64, 0)
        vals = np.arange(n, dtype=np.uint32)
        rk, rv, sent = idist.sample_sort(to_dev(keys), to_dev(vals))
        torch.cuda.synchronize()
        ek, ev = oracle.lsd(keys, vals, 32, 8)
        assert np.array_equal(to_np(rk, np.uint32), ek) and np.array_equal(to_np(rv, np.uint32), ev)
        assert sent.cpu().tolist() == [n]
    finally:
        dist.destroy_process_group()

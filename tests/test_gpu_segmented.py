"""GPU parity of the batched segmented sort against the oracle (bit-exact):
every routing class (OET, warp BTN, CTA BTN, clusters of 1/2/4/8 CTAs, and the
long-segment path), empty and one-key segments, key ranges, payloads, graph
reuse, error paths, and the full 200,000-length workload capped at 2^28 keys."""
import os

import numpy as np
import pytest

import gen
import oracle
from gen import workloads
from tests._util import to_dev, to_np

pytestmark = pytest.mark.gpu

CLASS_EDGES = [0, 1, 2, 3, 31, 32, 33, 255, 256, 257, 4095, 4096, 4097, 8191, 8192, 8193, 16384, 16385,
               32768, 32769, 65535, 65536]


def make(lengths, seed, bits=32):
    lengths = np.asarray(lengths, dtype=np.uint64)
    off = np.zeros(lengths.size + 1, np.uint64)
    off[1:] = np.cumsum(lengths)
    n = int(off[-1])
    keys = gen.uniform_u32(n, bits, seed, 0) if n else np.zeros(0, np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    return keys, vals, off


def run(isort, keys, vals, off, key_bits=32):
    import torch

    tk = to_dev(keys)
    tv = None if vals is None else to_dev(vals)
    to = to_dev(off)
    isort.segmented(tk, tv, to, key_bits)
    torch.cuda.synchronize()
    return to_np(tk, np.uint32), (None if vals is None else to_np(tv, np.uint32))


def check(isort, keys, vals, off, key_bits=32):
    gk, gv = run(isort, keys, vals, off, key_bits)
    rk, rv = oracle.segmented(keys, vals, off, key_bits, 8)
    assert np.array_equal(gk, rk)
    if vals is not None:
        assert np.array_equal(gv, rv)


def test_every_class_edge(cuda_lib):
    lengths = CLASS_EDGES + CLASS_EDGES[::-1]
    keys, vals, off = make(lengths, 5)
    keys[::3] = keys[7]  # ties across and within segments
    check(cuda_lib, keys, vals, off)
    check(cuda_lib, keys, None, off)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_lengths(cuda_lib, seed):
    r = np.random.default_rng(seed)
    lengths = np.concatenate([r.integers(0, 40, 300), r.integers(30, 300, 100), r.integers(250, 5000, 40),
                              r.integers(4000, 66000, 12)])
    r.shuffle(lengths)
    keys, vals, off = make(lengths, 10 + seed)
    check(cuda_lib, keys, vals, off)


@pytest.mark.parametrize("span", [1, 7, 300, 5000, 1 << 20])
def test_long_segments_narrow_key_ranges(cuda_lib, span):
    """Segments of 8193..65536 keys whose keys fall in a narrow range, so that
    the MSD digit groups stay large and are split again (several levels)."""
    lengths = [8193, 12000, 16385, 30000, 32769, 50000, 65536]
    keys, vals, off = make(lengths, 40 + span % 97)
    keys = (np.uint32(123456789) + keys % np.uint32(span)).astype(np.uint32)
    check(cuda_lib, keys, vals, off)
    check(cuda_lib, keys, None, off)


@pytest.mark.parametrize("key_bits", [8, 16, 20, 31])
def test_key_bits(cuda_lib, key_bits):
    lengths = [17, 200, 3000, 9000, 20000, 40000, 70000]
    keys, vals, off = make(lengths, 30 + key_bits, key_bits)
    check(cuda_lib, keys, vals, off, key_bits)


def test_skewed_keys(cuda_lib):
    lengths = [31, 250, 4000, 8000, 30000, 60000]
    keys, vals, off = make(lengths, 4)
    keys[:] = gen.zipf_u32(keys.size, 1.1, 9, 10)
    check(cuda_lib, keys, vals, off)


def test_long_segments_host_path(cuda_lib):
    lengths = [5, 70000, 3, 200001, 66000]
    keys, vals, off = make(lengths, 41)
    check(cuda_lib, keys, vals, off)


def test_graph_reuse_different_buffers(cuda_lib):
    for seed, lengths in ((51, [10, 300, 5000, 20000]), (52, [40000, 1, 33, 257]), (53, [10, 300, 5000, 20000])):
        keys, vals, off = make(lengths, seed)
        check(cuda_lib, keys, vals, off)


def test_key_range_segment_left_unchanged(cuda_lib):
    import torch

    lengths = [20, 100, 1000, 10000, 50000]
    keys, vals, off = make(lengths, 61, 16)
    bad_seg = [1, 3]  # a warp-BTN segment and a cluster segment
    for s in bad_seg:
        keys[int(off[s]) + 5] = 1 << 16
    tk, tv, to = to_dev(keys), to_dev(vals), to_dev(off)
    with pytest.raises(cuda_lib.IsortError) as e:
        cuda_lib.segmented(tk, tv, to, 16)
    assert e.value.code == cuda_lib.KEY_RANGE
    torch.cuda.synchronize()
    gk, gv = to_np(tk, np.uint32), to_np(tv, np.uint32)
    for s in range(len(lengths)):
        a, b = int(off[s]), int(off[s + 1])
        if s in bad_seg:
            assert np.array_equal(gk[a:b], keys[a:b]) and np.array_equal(gv[a:b], vals[a:b])
        else:
            rk, rv = oracle.lsd(keys[a:b], vals[a:b], 16, 8)
            assert np.array_equal(gk[a:b], rk) and np.array_equal(gv[a:b], rv)


def test_decreasing_offsets_rejected(cuda_lib):
    keys, vals, off = make([10, 10, 10], 71)
    off[2] = 5
    with pytest.raises(cuda_lib.IsortError) as e:
        run(cuda_lib, keys, vals, off)
    assert e.value.code == cuda_lib.INVALID_ARG


def test_async_mode_long_segment_unsupported(cuda_lib):
    import torch

    keys, vals, off = make([100, 70000], 72)
    tk, tv, to = to_dev(keys), to_dev(vals), to_dev(off)
    cuda_lib.device_status(clear=True)
    cuda_lib.set_sync(False)
    try:
        cuda_lib.segmented(tk, tv, to, 32)
        assert cuda_lib.device_status(clear=True) == cuda_lib.UNSUPPORTED
    finally:
        cuda_lib.set_sync(True)
    torch.cuda.synchronize()
    gk = to_np(tk, np.uint32)
    rk, _ = oracle.lsd(keys[:100], None, 32, 8)
    assert np.array_equal(gk[:100], rk)  # the short segment is still sorted


def test_full_segmented_workload(cuda_lib):
    """200,000 log-uniform lengths on [2, 65,536] (seed 4) capped at 2^28 keys,
    u32 keys + payload: bit-exact against the oracle."""
    keys, vals, off = workloads.segmented()
    gk, gv = run(cuda_lib, keys, vals, off)
    rk, rv = oracle.segmented(keys, vals, off, 32, 8)
    assert np.array_equal(gk, rk) and np.array_equal(gv, rv)


def _router_lines(path):
    out = {}
    if os.path.exists(path):
        for ln in open(path):
            p = ln.split()
            if p and p[0] == "router":
                out.setdefault(int(p[1]), []).append(tuple(int(x) for x in p[2:5]))
    return out


def test_router_autotune_cache_and_parity(cuda_lib, tmp_path):
    """The router's cut-offs measured on this GPU: written to the cache once per
    kind, read back after a reset instead of measured again, within the
    kernels' limits; and the sort bit-exact against the oracle with the tuned
    cut-offs and with planted ones."""
    lengths = [2, 7, 20, 32, 33, 60, 128, 255, 300, 700, 1500, 3000, 4096, 5000, 8192, 9000, 20000] * 3
    keys, vals, off = make(lengths, 97)
    path = str(tmp_path / "tune.txt")
    try:
        cuda_lib.autotune(True, path)
        check(cuda_lib, keys, vals, off)  # payload: measures and appends "router 1 ..."
        check(cuda_lib, keys, None, off)  # keys only: "router 0 ..."
        lines = _router_lines(path)
        assert sorted(lines) == [0, 1] and all(len(v) == 1 for v in lines.values())
        for oet, bw, bc in (lines[0][0], lines[1][0]):
            assert 0 <= oet <= 32 and oet <= bw <= 256 and bw <= bc <= 4096
        cuda_lib.autotune(True, path)  # reset: the cut-offs now come from the file
        check(cuda_lib, keys, vals, off)
        assert _router_lines(path) == lines
        planted = str(tmp_path / "planted.txt")
        with open(planted, "w") as f:  # every segment to the on-chip count-sort rounds / to the networks
            f.write("router 1 0 0 0\nrouter 0 32 256 4096\n")
        cuda_lib.autotune(True, planted)
        check(cuda_lib, keys, vals, off)
        check(cuda_lib, keys, None, off)
        assert _router_lines(planted) == {1: [(0, 0, 0)], 0: [(32, 256, 4096)]}
    finally:
        cuda_lib.autotune(False)


def _fine_segments(seed):
    """Segments of 4,097..8,192 keys (the one-CTA class) that drive every path
    of the fine finish: uniform keys (short runs), clusters of 10 / 20 / 300
    distinct keys under a far outlier (insertion, warp network), clusters of
    600 and 7,000 (runs too long: handed to the other kernel), all keys equal,
    ranges of 200 and 4,096 values (one or two passes, no runs)."""
    r = np.random.default_rng(seed)
    segs = []

    def uni(n, hi=2**32):
        return r.integers(0, hi, n, dtype=np.uint64).astype(np.uint32)

    segs.append(uni(8192))
    segs.append(uni(4097))
    for c in (10, 20, 300, 600):
        x = uni(5000 - c - 1)
        x = np.concatenate([x, (100 + r.permutation(c)).astype(np.uint32), np.array([2**32 - 1], np.uint32)])
        segs.append(r.permutation(x).astype(np.uint32))
    x = np.concatenate([(1000 + r.permutation(7000)).astype(np.uint32), uni(100), np.array([2**32 - 1], np.uint32)])
    segs.append(r.permutation(x).astype(np.uint32))
    segs.append(np.full(5000, 123456789, np.uint32))
    segs.append(uni(6000, 200))
    segs.append(uni(7000, 4096))
    dup = uni(6500)
    dup[::3] = dup[1]  # many equal keys spread through the segment
    segs.append(dup)
    keys = np.concatenate(segs)
    off = np.zeros(len(segs) + 1, np.uint64)
    off[1:] = np.cumsum([len(x) for x in segs])
    return keys, np.arange(keys.size, dtype=np.uint32), off


@pytest.mark.parametrize("payload", [True, False])
def test_fine_finish_every_path(cuda_lib, payload):
    keys, vals, off = _fine_segments(98)
    check(cuda_lib, keys, vals if payload else None, off)

"""ORACLE — test infrastructure only.

Python access to the serial C oracle (``isort_oracle.c``). Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this
package; the library under test never does, and the two share no code.

Every function returns new arrays (inputs are copied first) and follows the
passage of Gerbessiotis, arXiv:1708.09495, cited in the C source: the LSD sort
is the paper's serial radix-r count-sort rounds (Section 3, eq. Ts), BTN and OET
its block networks (Section 2; Section 3 eqs. Tb, To).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isort_oracle.c")
_lock = threading.Lock()
_handles: dict = {}


def so_path(mutant: int = 0) -> str:
    return os.path.join(_HERE, "libisort_oracle.so" if mutant == 0 else f"libisort_oracle_m{mutant}.so")


def build(force: bool = False, mutant: int = 0) -> str:
    """Compile the oracle (gcc, -O2). ``mutant`` > 0 builds a deliberately
    broken variant used by the tests to show that the pins catch mistakes."""
    so = so_path(mutant)
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-Wall", "-ffp-contract=off", _SRC, "-o", tmp]
        if mutant:
            cmd.insert(1, f"-DORACLE_MUTANT={int(mutant)}")
        subprocess.check_call(cmd)
        os.replace(tmp, so)
    return so


def _lib(mutant: int = 0):
    with _lock:
        h = _handles.get(mutant)
        if h is None:
            h = ctypes.CDLL(build(mutant=mutant))
            vp, sz, i32, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64
            for nm in ("oracle_lsd_u32", "oracle_lsd_u64"):
                getattr(h, nm).argtypes = [vp, vp, sz, i32, i32]
            for nm in ("oracle_count_round_u32", "oracle_count_round_u64"):
                getattr(h, nm).argtypes = [vp, vp, vp, vp, sz, i32, i32]
            for nm in ("oracle_digit_hist_u32", "oracle_digit_hist_u64"):
                getattr(h, nm).argtypes = [vp, sz, i32, i32, vp]
            for nm in ("oracle_insertion_u32", "oracle_insertion_u64"):
                getattr(h, nm).argtypes = [vp, vp, sz]
                getattr(h, nm).restype = None
            h.oracle_btn_u32.argtypes = [vp, vp, sz, i32, vp]
            h.oracle_oet_u32.argtypes = [vp, vp, sz, i32, vp]
            h.oracle_segmented_u32.argtypes = [vp, vp, vp, sz, i32, i32]
            for nm in ("oracle_partition_u32", "oracle_partition_u64"):
                getattr(h, nm).argtypes = [vp, vp, vp, vp, sz, vp, sz, i32, vp]
            for nm in ("oracle_is_sorted_u32", "oracle_is_sorted_u64"):
                getattr(h, nm).argtypes = [vp, sz]
            for nm in ("oracle_is_stable_u32", "oracle_is_stable_u64"):
                getattr(h, nm).argtypes = [vp, vp, sz]
            for nm in ("oracle_multiset_hash_u32", "oracle_multiset_hash_u64"):
                getattr(h, nm).argtypes = [vp, vp, sz]
                getattr(h, nm).restype = u64
            h.oracle_sample_indices.argtypes = [u64, ctypes.c_uint32, u64, vp]
            h.oracle_sample_indices.restype = None
            h.oracle_bucket_of.argtypes = [vp, vp, i32, i32, i32, u64]
            h.oracle_bucket_of.restype = ctypes.c_uint32
            h.oracle_splitters.argtypes = [vp, vp, i32, i32, i32, vp]
            h.oracle_splitters.restype = None
            h.oracle_bucket_ids.argtypes = [vp, i32, sz, i32, vp, vp, i32, vp]
            h.oracle_bucket_ids.restype = None
            h.oracle_cdf_knots.argtypes = [vp, vp, vp]
            h.oracle_cdf_knots.restype = None
            h.oracle_cdf_loss_grad.argtypes = [vp, ctypes.c_uint32, vp, vp]
            h.oracle_cdf_loss_grad.restype = ctypes.c_double
            h.oracle_sort_typed.argtypes = [vp, i32, vp, sz]
            h.oracle_sort_typed.restype = i32
            h.oracle_mlp_cdf.argtypes = [vp, ctypes.c_double]
            h.oracle_mlp_cdf.restype = ctypes.c_double
            h.oracle_mlp_loss_grad.argtypes = [vp, ctypes.c_uint32, vp, vp]
            h.oracle_mlp_loss_grad.restype = ctypes.c_double
            _handles[mutant] = h
    return h


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _kind(keys: np.ndarray) -> str:
    if keys.dtype == np.uint32:
        return "u32"
    if keys.dtype == np.uint64:
        return "u64"
    raise TypeError(f"keys must be uint32 or uint64, got {keys.dtype}")


def _copy(keys, vals):
    k = np.array(keys, copy=True, order="C")
    v = None if vals is None else np.array(vals, dtype=np.uint32, copy=True, order="C")
    if v is not None and v.shape != k.shape:
        raise ValueError("vals must match keys")
    return k, v


def lsd(keys, vals=None, key_bits: int = 0, radix_bits: int = 8, mutant: int = 0):
    """Stable LSD radix sort (Section 3, SR4 generalised). Returns (keys, vals)."""
    k, v = _copy(keys, vals)
    rc = getattr(_lib(mutant), f"oracle_lsd_{_kind(k)}")(_p(k), _p(v), k.size, key_bits, radix_bits)
    if rc != 0:
        raise ValueError("oracle_lsd: invalid arguments")
    return k, v


def count_round(keys, vals, shift: int, width: int, mutant: int = 0):
    """One stable count-sort round on digit (key >> shift) & (2^width - 1)."""
    k, v = _copy(keys, vals)
    ko = np.empty_like(k)
    vo = None if v is None else np.empty_like(v)
    rc = getattr(_lib(mutant), f"oracle_count_round_{_kind(k)}")(_p(k), _p(v), _p(ko), _p(vo), k.size, shift, width)
    if rc != 0:
        raise MemoryError("oracle_count_round")
    return ko, vo


def digit_hist(keys, key_bits: int = 0, radix_bits: int = 8):
    """Per-round digit histograms, shape (rounds, 2^radix_bits), uint64."""
    k = np.ascontiguousarray(keys)
    kb = key_bits or (32 if k.dtype == np.uint32 else 64)
    P = -(-kb // radix_bits)
    h = np.zeros((P, 1 << radix_bits), np.uint64)
    rc = getattr(_lib(), f"oracle_digit_hist_{_kind(k)}")(_p(k), k.size, key_bits, radix_bits, _p(h))
    if rc != P:
        raise ValueError("oracle_digit_hist: invalid arguments")
    return h


def insertion(keys, vals=None):
    """Brute-force stable insertion sort (a pin)."""
    k, v = _copy(keys, vals)
    getattr(_lib(), f"oracle_insertion_{_kind(k)}")(_p(k), _p(v), k.size)
    return k, v


def btn(keys, vals=None, p: int = 4, mutant: int = 0):
    """BTN on p blocks (Section 2, eq. Tb). Returns (keys, vals, stages)."""
    k, v = _copy(keys, vals)
    st = np.zeros(1, np.uint64)
    rc = _lib(mutant).oracle_btn_u32(_p(k), _p(v), k.size, p, _p(st))
    if rc != 0:
        raise ValueError("oracle_btn: p must be a power of two")
    return k, v, int(st[0])


def oet(keys, vals=None, p: int = 4, mutant: int = 0):
    """OET on p blocks (Section 2, eq. To). Returns (keys, vals, rounds)."""
    k, v = _copy(keys, vals)
    rd = np.zeros(1, np.uint64)
    rc = _lib(mutant).oracle_oet_u32(_p(k), _p(v), k.size, p, _p(rd))
    if rc != 0:
        raise ValueError("oracle_oet: invalid arguments")
    return k, v, int(rd[0])


def segmented(keys, vals, offsets, key_bits: int = 0, radix_bits: int = 8):
    """Each CSR segment [off[s], off[s+1]) sorted on its own."""
    k, v = _copy(keys, vals)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    rc = _lib().oracle_segmented_u32(_p(k), _p(v), _p(off), off.size - 1, key_bits, radix_bits)
    if rc != 0:
        raise ValueError("oracle_segmented: invalid arguments")
    return k, v


def partition(keys, vals, sorted_sample, parts: int, mutant: int = 0):
    """Sample-sort routing: splitter j = sorted_sample[floor(j m / parts)]
    (1 <= j < parts), range of a key = number of splitters <= key, keys routed
    stably by range. Returns (keys, vals, counts)."""
    k = np.ascontiguousarray(keys)
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32)
    smp = np.ascontiguousarray(sorted_sample, dtype=k.dtype)
    ko = np.empty_like(k)
    vo = None if v is None else np.empty_like(v)
    counts = np.zeros(max(parts, 1), np.uint64)
    rc = getattr(_lib(mutant), f"oracle_partition_{_kind(k)}")(_p(k), _p(v), _p(ko), _p(vo), k.size, _p(smp),
                                                                 smp.size, parts, _p(counts))
    if rc != 0:
        raise ValueError("oracle_partition: invalid arguments")
    return ko, vo, counts


def is_sorted(keys) -> bool:
    k = np.ascontiguousarray(keys)
    return bool(getattr(_lib(), f"oracle_is_sorted_{_kind(k)}")(_p(k), k.size))


def is_stable(keys, vals) -> bool:
    """With payload = original index: strictly increasing payloads within equal keys."""
    k = np.ascontiguousarray(keys)
    v = np.ascontiguousarray(vals, dtype=np.uint32)
    return bool(getattr(_lib(), f"oracle_is_stable_{_kind(k)}")(_p(k), _p(v), k.size))


def multiset_hash(keys, vals=None, mutant: int = 0) -> int:
    """Commutative 64-bit hash of the (key, payload) multiset."""
    k = np.ascontiguousarray(keys)
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32)
    return int(getattr(_lib(mutant), f"oracle_multiset_hash_{_kind(k)}")(_p(k), _p(v), k.size))


def key_range_ok(keys, key_bits: int) -> bool:
    """True iff every key is < 2^key_bits (key_bits 0 = full width)."""
    k = np.ascontiguousarray(keys)
    width = 32 if k.dtype == np.uint32 else 64
    if key_bits in (0, width):
        return True
    return bool(k.size == 0 or int(k.max()) >> key_bits == 0)


# ----------------------------------------------------------------------------- learned buckets

SAMPLE_SEED = 0x5EED5EED5EED
SAMPLE_SIZE = 1 << 16


def sample_indices(n: int, m: int = SAMPLE_SIZE, seed: int = SAMPLE_SEED):
    """index_j = floor(r_j * n / 2^64), r_j = SplitMix64 output j from state seed."""
    idx = np.empty(m, np.uint64)
    _lib().oracle_sample_indices(n, m, seed, _p(idx))
    return idx


def bucket_of(X, Y, key: int, key_width: int = 32, key_bits: int = 32, nbuckets: int = 4096) -> int:
    """The model's bucket of one key."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    return int(_lib().oracle_bucket_of(_p(X), _p(Y), key_width, key_bits, nbuckets, int(key)))


def splitters(X, Y, key_width: int = 32, key_bits: int = 32, nbuckets: int = 4096):
    """The splitter table: the first key of each bucket (uint64, nbuckets
    entries; entry 0 is 0)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    s = np.zeros(nbuckets, np.uint64)
    _lib().oracle_splitters(_p(X), _p(Y), key_width, key_bits, nbuckets, _p(s))
    return s


def bucket_ids(keys, X, Y, key_bits: int = 0, nbuckets: int = 4096):
    """The model's bucket of every key (uint32)."""
    k = np.ascontiguousarray(keys)
    w = 32 if k.dtype == np.uint32 else 64
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    ids = np.empty(k.size, np.uint32)
    _lib().oracle_bucket_ids(_p(k), w, k.size, key_bits or w, _p(X), _p(Y), nbuckets, _p(ids))
    return ids


def cdf_knots(theta):
    t = np.ascontiguousarray(theta, dtype=np.float64)
    X = np.empty(257, np.float64)
    Y = np.empty(257, np.float64)
    _lib().oracle_cdf_knots(_p(t), _p(X), _p(Y))
    return X, Y


def cdf_loss_grad(u, theta, with_grad: bool = True):
    """(loss, dloss/dtheta) of the CDF model in double precision."""
    uu = np.ascontiguousarray(u, dtype=np.float64)
    t = np.ascontiguousarray(theta, dtype=np.float64)
    g = np.zeros(512, np.float64) if with_grad else None
    loss = _lib().oracle_cdf_loss_grad(_p(uu), uu.size, _p(t), _p(g))
    return float(loss), g


MLP_HIDDEN = 32
MLP_PARAMS = 3 * MLP_HIDDEN + 1


def mlp_cdf(params, u: float) -> float:
    """F(u) of the 1-32-1 monotone MLP model (double)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    return float(_lib().oracle_mlp_cdf(_p(p), float(u)))


def mlp_loss_grad(u, params, with_grad: bool = True):
    """(loss, dloss/dparams) of the MLP model in double precision."""
    uu = np.ascontiguousarray(u, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    g = np.zeros(MLP_PARAMS, np.float64) if with_grad else None
    loss = _lib().oracle_mlp_loss_grad(_p(uu), uu.size, _p(p), _p(g))
    return float(loss), g


KEY_TYPES = {"i32": (1, np.int32), "f32": (2, np.float32), "i64": (4, np.int64), "f64": (5, np.float64)}


def sort_typed(keys, vals=None):
    """Stable sort of int32/float32/int64/float64 keys by the order of their
    type (floats: IEEE 754 totalOrder, on the bits); returns (keys, vals)."""
    name = {np.dtype(t): n for n, (_, t) in KEY_TYPES.items()}.get(np.asarray(keys).dtype)
    if name is None:
        raise TypeError(f"keys must be int32, float32, int64 or float64, got {np.asarray(keys).dtype}")
    k = np.array(keys, copy=True)
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    rc = _lib().oracle_sort_typed(_p(k), KEY_TYPES[name][0], _p(v), k.size)
    if rc != 0:
        raise RuntimeError(f"oracle_sort_typed failed ({rc})")
    return k, v

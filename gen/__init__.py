"""Seeded synthetic inputs for the integer-sort workloads.

This module only produces inputs (keys, payloads, segment lengths). It holds no
sorting arithmetic, so both the oracle and the CUDA library can consume its
output without sharing any of the method's code. The C source
(``isort_gen.c``) documents the counter-based SplitMix64 streams and each
distribution; ``workloads`` names the concrete benchmark inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isort_gen.c")
_SO = os.path.join(_HERE, "libisort_gen.so")
_lock = threading.Lock()
_handle = None


def build(force: bool = False) -> str:
    """Compile ``libisort_gen.so`` next to its source (host C, gcc)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE", "-Wall", _SRC, "-o", tmp,
             "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            build()
            h = ctypes.CDLL(_SO)
            u64, sz, i32, dbl, vp = ctypes.c_uint64, ctypes.c_size_t, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            h.isort_gen_uniform_u32.argtypes = [u64, u64, sz, i32, vp]
            h.isort_gen_uniform_u64.argtypes = [u64, u64, sz, i32, vp]
            h.isort_gen_iota_u32.argtypes = [sz, vp]
            h.isort_gen_iota_u32.restype = None
            h.isort_gen_loguniform_lengths.argtypes = [u64, u64, sz, dbl, dbl, vp]
            h.isort_gen_zipf_u32.argtypes = [u64, u64, sz, dbl, vp]
            h.isort_gen_lognormal_u32.argtypes = [u64, u64, sz, dbl, dbl, vp]
            h.isort_gen_gmm_u32.argtypes = [u64, u64, sz, i32, dbl, vp]
            h.isort_gen_fnv1a.argtypes = [vp, sz]
            h.isort_gen_fnv1a.restype = u64
            h.isort_gen_draw.argtypes = [u64, u64, u64]
            h.isort_gen_draw.restype = u64
            h.isort_gen_splitmix_raw.argtypes = [u64, u64]
            h.isort_gen_splitmix_raw.restype = u64
            h.isort_gen_mix32.argtypes = [ctypes.c_uint32]
            h.isort_gen_mix32.restype = ctypes.c_uint32
            h.isort_gen_set_threads.argtypes = [i32]
            h.isort_gen_set_threads.restype = None
            _handle = h
    return _handle


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed (rc={rc})")


def set_threads(t: int) -> None:
    """Threads used by the generators (0 = all online CPUs)."""
    _lib().isort_gen_set_threads(int(t))


def draw(seed: int, stream: int, i: int) -> int:
    """The i-th raw 64-bit SplitMix64 draw of (seed, stream)."""
    return int(_lib().isort_gen_draw(seed, stream, i))


def splitmix_raw(state: int, i: int) -> int:
    """The i-th output of plain SplitMix64 started from ``state``."""
    return int(_lib().isort_gen_splitmix_raw(state, i))


def uniform_u32(n: int, bits: int = 32, seed: int = 0, stream: int = 0, out: np.ndarray | None = None):
    """n keys uniform on [0, 2^bits) (top bits of each draw)."""
    a = np.empty(n, np.uint32) if out is None else out
    _check(_lib().isort_gen_uniform_u32(seed, stream, n, bits, _ptr(a)), "uniform_u32")
    return a


def uniform_u64(n: int, bits: int = 64, seed: int = 0, stream: int = 0, out: np.ndarray | None = None):
    """n keys uniform on [0, 2^bits)."""
    a = np.empty(n, np.uint64) if out is None else out
    _check(_lib().isort_gen_uniform_u64(seed, stream, n, bits, _ptr(a)), "uniform_u64")
    return a


def iota_u32(n: int, out: np.ndarray | None = None):
    """Payload = original index."""
    a = np.empty(n, np.uint32) if out is None else out
    _lib().isort_gen_iota_u32(n, _ptr(a))
    return a


def loguniform_lengths(nseg: int, lo: float, hi: float, seed: int, stream: int = 1):
    """Segment lengths round(exp(U(ln lo, ln hi)))."""
    a = np.empty(nseg, np.uint64)
    _check(_lib().isort_gen_loguniform_lengths(seed, stream, nseg, lo, hi, _ptr(a)), "loguniform_lengths")
    return a


def zipf_u32(n: int, s: float, seed: int, stream: int = 0, out: np.ndarray | None = None):
    """Zipf(s) ranks on 1..2^32-1 mapped through a bijective 32-bit mixer."""
    a = np.empty(n, np.uint32) if out is None else out
    _check(_lib().isort_gen_zipf_u32(seed, stream, n, s, _ptr(a)), "zipf_u32")
    return a


def lognormal_u32(n: int, mu: float, sigma: float, seed: int, stream: int = 0, out: np.ndarray | None = None):
    """floor(exp(mu + sigma Z)); draws >= 2^32 redrawn."""
    a = np.empty(n, np.uint32) if out is None else out
    _check(_lib().isort_gen_lognormal_u32(seed, stream, n, mu, sigma, _ptr(a)), "lognormal_u32")
    return a


def gmm_u32(n: int, ncomp: int, sigma: float, seed: int, stream: int = 0, out: np.ndarray | None = None):
    """Equal-weight Gaussian mixture, means uniform on [0, 2^32), clipped to uint32."""
    a = np.empty(n, np.uint32) if out is None else out
    _check(_lib().isort_gen_gmm_u32(seed, stream, n, ncomp, sigma, _ptr(a)), "gmm_u32")
    return a


def mix32(x: int) -> int:
    """The bijective 32-bit mixer used to hash Zipf ranks."""
    return int(_lib().isort_gen_mix32(x))


def fnv1a(a: np.ndarray) -> int:
    """FNV-1a digest of an array's bytes (golden fixtures)."""
    a = np.ascontiguousarray(a)
    return int(_lib().isort_gen_fnv1a(_ptr(a), a.nbytes))

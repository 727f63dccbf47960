"""Multicore CPU baseline (the paper's parallel radix-r sort and its BTN / OET
block networks on std::thread workers), built from ``pr_sort.cpp`` with the
host C++ compiler and loaded through ctypes.

It is a reported baseline for the benchmark, timed on the host cores beside
the GPU path; it shares no code with the serial checker or the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pr_sort.cpp")
LIB = os.path.join(HERE, "libpr_sort.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the library (g++, -O3, C++20) if it is missing or stale."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O3", "-std=c++20", "-fPIC", "-shared", "-pthread", SRC, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"g++ failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, sz = ctypes.c_void_p, ctypes.c_size_t
            for name in ("cpu_pr_sort_u32", "cpu_pr_sort_u64"):
                fn = getattr(lib, name)
                fn.restype = ctypes.c_int
                fn.argtypes = [vp, vp, sz, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            for name in ("cpu_btn_u32", "cpu_oet_u32"):
                fn = getattr(lib, name)
                fn.restype = ctypes.c_int
                fn.argtypes = [vp, vp, sz, ctypes.c_int]
            lib.cpu_hardware_threads.restype = ctypes.c_int
            lib.cpu_hardware_threads.argtypes = []
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def hardware_threads() -> int:
    return int(_load().cpu_hardware_threads())


def pr_sort(keys, vals=None, key_bits: int = 0, radix_bits: int = 8, threads: int = 0):
    """Stable parallel radix sort in place on numpy arrays (u32 or u64 keys)."""
    lib = _load()
    t = threads or hardware_threads()
    fn = lib.cpu_pr_sort_u32 if keys.dtype == np.uint32 else lib.cpu_pr_sort_u64
    if not keys.flags.c_contiguous or (vals is not None and not vals.flags.c_contiguous):
        raise ValueError("contiguous arrays only")
    if fn(_p(keys), _p(vals), keys.size, key_bits, radix_bits, t) != 0:
        raise ValueError("cpu_pr_sort: invalid arguments")


def btn(keys, vals=None, p: int = 4):
    """BTN on p workers (p a power of two), in place (u32 keys)."""
    if _load().cpu_btn_u32(_p(keys), _p(vals), keys.size, p) != 0:
        raise ValueError("cpu_btn: invalid arguments")


def oet(keys, vals=None, p: int = 4):
    """OET on p workers, in place (u32 keys)."""
    if _load().cpu_oet_u32(_p(keys), _p(vals), keys.size, p) != 0:
        raise ValueError("cpu_oet: invalid arguments")


def cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo; Arm cores report implementer and part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    for key in ("model name", "Model name", "cpu model"):
        for ln in info:
            if ln.lower().startswith(key.lower()) and ":" in ln:
                return ln.split(":", 1)[1].strip()
    impl = part = None
    for ln in info:
        if ln.startswith("CPU implementer") and impl is None:
            impl = ln.split(":", 1)[1].strip()
        if ln.startswith("CPU part") and part is None:
            part = ln.split(":", 1)[1].strip()
    names = {("0x41", "0xd4f"): "Arm Neoverse V2"}
    if impl and part:
        return names.get((impl, part), f"implementer {impl} part {part}")
    return "unknown"

"""GB300 integer sorting: Python binding of ``libisort.so``.

The library implements, in hand-written CUDA for sm_103a, the count-sort
rounds of LSD radix sort and the BTN / OET block networks of Gerbessiotis,
"Integer sorting on multicores: some (experiments and) observations"
(arXiv:1708.09495, Sections 2 and 3). This module only marshals arguments:
every step of every sort runs in the library's kernels. PyTorch provides
device memory and streams.

Two layers:
  * ``isort_*`` functions with the C ABI's names and arguments (raw pointers
    as ints, sizes, a stream handle) — see ``include/isort.h``;
  * tensor helpers (``radix``, ``radix_copy``, ``btn``, ``oet``, ``digit_hist``,
    ``count_round``) that take torch tensors and raise ``IsortError``.

There is no fallback: if the library is missing or fails to load, ``load()``
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libisort.so")

STATUS = {
    0: "ISORT_OK",
    1: "ISORT_ERR_INVALID_ARG",
    2: "ISORT_ERR_KEY_RANGE",
    3: "ISORT_ERR_NO_MEMORY",
    4: "ISORT_ERR_CUDA",
    5: "ISORT_ERR_TIMEOUT",
    6: "ISORT_ERR_UNSUPPORTED",
}
OK, INVALID_ARG, KEY_RANGE, NO_MEMORY, CUDA_ERROR, TIMEOUT, UNSUPPORTED = range(7)

# Every symbol include/isort.h declares: (name, restype, argtypes).
_vp, _sz, _i32, _u64, _i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64


class LearnedStats(ctypes.Structure):
    _fields_ = [("imbalance_max_over_mean", ctypes.c_double), ("overflow_fraction", ctypes.c_double),
                ("fixups", ctypes.c_uint64), ("overflow_buckets", ctypes.c_uint64),
                ("fell_back_to_lsd", ctypes.c_int), ("train_steps", ctypes.c_int),
                ("train_loss_initial", ctypes.c_float), ("train_loss", ctypes.c_float), ("nbuckets", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


SIGNATURES = [
    ("isort_status_string", ctypes.c_char_p, [_i32]),
    ("isort_radix", _i32, [_vp, _vp, _sz, _i32, _i32, _vp]),
    ("isort_radix_u64", _i32, [_vp, _vp, _sz, _i32, _i32, _vp]),
    ("isort_radix_copy", _i32, [_vp, _vp, _vp, _vp, _sz, _i32, _i32, _vp]),
    ("isort_radix_copy_u64", _i32, [_vp, _vp, _vp, _vp, _sz, _i32, _i32, _vp]),
    ("isort_digit_hist", _i32, [_vp, _i32, _sz, _i32, _i32, _vp, _vp]),
    ("isort_count_round", _i32, [_vp, _vp, _vp, _vp, _sz, _i32, _i32, _vp]),
    ("isort_count_round_u64", _i32, [_vp, _vp, _vp, _vp, _sz, _i32, _i32, _vp]),
    ("isort_btn", _i32, [_vp, _vp, _sz, _vp]),
    ("isort_oet", _i32, [_vp, _vp, _sz, _vp]),
    ("isort_btn_p", _i32, [_vp, _vp, _sz, _i32, _vp, _vp]),
    ("isort_oet_p", _i32, [_vp, _vp, _sz, _i32, _vp, _vp]),
    ("isort_segmented", _i32, [_vp, _vp, _vp, _sz, _i32, _vp]),
    ("isort_radix_noalloc", _i32, [_vp, _vp, _sz, _i32, _i32, _vp]),
    ("isort_sample", _i32, [_vp, _i32, _sz, ctypes.c_uint32, ctypes.c_uint64, _vp, _vp]),
    ("isort_partition", _i32, [_vp, _vp, _vp, _vp, _sz, _vp, _sz, _i32, _vp, _vp]),
    ("isort_partition_u64", _i32, [_vp, _vp, _vp, _vp, _sz, _vp, _sz, _i32, _vp, _vp]),
    ("isort_learned", _i32, [_vp, _vp, _sz, _i32, _i32, _i32, _vp, _vp]),
    ("isort_learned_u64", _i32, [_vp, _vp, _sz, _i32, _i32, _i32, _vp, _vp]),
    ("isort_cdf_train", _i32, [_vp, ctypes.c_uint32, _i32, _vp, _vp, _vp, _vp, _vp]),
    ("isort_cdf_loss_grad", _i32, [_vp, ctypes.c_uint32, _vp, _vp, _vp, _vp]),
    ("isort_radix_typed", _i32, [_vp, _i32, _vp, ctypes.c_size_t, _i32, _vp]),
    ("isort_mlp_train", _i32, [_vp, ctypes.c_uint32, _i32, _vp, _vp, _vp, _vp, _vp]),
    ("isort_mlp_loss_grad", _i32, [_vp, ctypes.c_uint32, _vp, _vp, _vp, _vp]),
    ("isort_cdf_splitters", _i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    ("isort_bucket_ids", _i32, [_vp, _i32, _sz, _i32, _vp, _vp, _i32, _vp, _vp]),
    ("isort_autotune", _i32, [_i32, ctypes.c_char_p]),
    ("isort_set_sync", _i32, [_i32]),
    ("isort_device_status", _i32, [_i32, _vp]),
    ("isort_set_spin_limit", _i32, [_u64]),
    ("isort_debug_stall_tile", _i32, [_i64]),
    ("isort_launch_count", _u64, []),
    ("isort_last_error_string", ctypes.c_char_p, []),
    ("isort_profile_enable", _i32, [_i32]),
    ("isort_profile_read", _i32, [ctypes.POINTER(KernelTime), _i32]),
]

_lock = threading.Lock()
_lib = None


class IsortError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        detail = ""
        try:
            if _lib is not None:
                detail = (_lib.isort_last_error_string() or b"").decode()
        except Exception:
            detail = ""
        msg = f"{where}: {STATUS.get(code, code)}" if where else STATUS.get(code, str(code))
        super().__init__(f"{msg} ({detail})" if detail else msg)


def load(path: str | None = None):
    """Loads the CUDA library (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"{p} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(p)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def lib():
    return load()


def __getattr__(name):
    # isort_* raw entry points, resolved from the loaded library
    if name.startswith("isort_"):
        return getattr(load(), name)
    raise AttributeError(name)


# --------------------------------------------------------------------------- helpers


def _stream(stream):
    import torch

    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _check(code: int, where: str):
    if code != OK:
        raise IsortError(code, where)


def _key_width(t) -> int:
    import torch

    if t.dtype in (torch.uint32, torch.int32):
        return 32
    if t.dtype in (torch.uint64, torch.int64):
        return 64
    raise TypeError(f"keys must be 32- or 64-bit integers, got {t.dtype}")


def radix(keys, vals=None, key_bits: int = 0, radix_bits: int = 8, stream=None):
    """Stable in-place LSD radix sort of ``keys`` (uint32/uint64 bit patterns;
    int32/int64 tensors are sorted as their unsigned bit patterns) with an
    optional uint32 payload ``vals`` that moves with its key."""
    w = _key_width(keys)
    fn = load().isort_radix if w == 32 else load().isort_radix_u64
    _check(fn(_ptr(keys), _ptr(vals), keys.numel(), key_bits, radix_bits, _stream(stream)), "isort_radix")
    return keys, vals


def radix_copy(keys_in, vals_in, keys_out, vals_out, key_bits: int = 0, radix_bits: int = 8, stream=None):
    """Stable out-of-place LSD radix sort: inputs read, result in the outputs."""
    w = _key_width(keys_in)
    fn = load().isort_radix_copy if w == 32 else load().isort_radix_copy_u64
    _check(fn(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), keys_in.numel(), key_bits, radix_bits,
              _stream(stream)), "isort_radix_copy")
    return keys_out, vals_out


def digit_hist(keys, key_bits: int = 0, radix_bits: int = 8, stream=None):
    """Per-round digit counts, shape (rounds, 2^radix_bits), as a uint32 tensor."""
    import torch

    w = _key_width(keys)
    kb = key_bits or w
    rounds = -(-kb // radix_bits)
    hist = torch.empty((rounds, 1 << radix_bits), dtype=torch.uint32, device=keys.device)
    _check(load().isort_digit_hist(_ptr(keys), w, keys.numel(), key_bits, radix_bits, _ptr(hist), _stream(stream)),
           "isort_digit_hist")
    return hist


def count_round(keys_in, vals_in, shift: int, width: int, stream=None):
    """One stable count-sort round on digit (key >> shift) & (2^width - 1)."""
    import torch

    w = _key_width(keys_in)
    ko = torch.empty_like(keys_in)
    vo = None if vals_in is None else torch.empty_like(vals_in)
    fn = load().isort_count_round if w == 32 else load().isort_count_round_u64
    _check(fn(_ptr(keys_in), _ptr(vals_in), _ptr(ko), _ptr(vo), keys_in.numel(), shift, width, _stream(stream)),
           "isort_count_round")
    return ko, vo


def btn(keys, vals=None, p: int | None = None, stream=None):
    """In-place BTN sort (uint32 keys). With ``p`` given, returns the number
    of merge-split stages executed as well."""
    if p is None:
        _check(load().isort_btn(_ptr(keys), _ptr(vals), keys.numel(), _stream(stream)), "isort_btn")
        return keys, vals
    st = ctypes.c_uint64(0)
    _check(load().isort_btn_p(_ptr(keys), _ptr(vals), keys.numel(), p, ctypes.byref(st), _stream(stream)),
           "isort_btn_p")
    return keys, vals, int(st.value)


def oet(keys, vals=None, p: int | None = None, stream=None):
    """In-place OET sort (uint32 keys). With ``p`` given, also returns rounds."""
    if p is None:
        _check(load().isort_oet(_ptr(keys), _ptr(vals), keys.numel(), _stream(stream)), "isort_oet")
        return keys, vals
    st = ctypes.c_uint64(0)
    _check(load().isort_oet_p(_ptr(keys), _ptr(vals), keys.numel(), p, ctypes.byref(st), _stream(stream)),
           "isort_oet_p")
    return keys, vals, int(st.value)


def segmented(keys, vals, offsets, key_bits: int = 0, stream=None):
    """Sorts each CSR segment [offsets[s], offsets[s+1]) of keys (and vals) in
    place; offsets is a uint64/int64 device tensor of nseg + 1 entries."""
    if offsets.element_size() != 8:
        raise TypeError("offsets must be 64-bit")
    _check(load().isort_segmented(_ptr(keys), _ptr(vals), _ptr(offsets), offsets.numel() - 1, key_bits,
                                  _stream(stream)), "isort_segmented")
    return keys, vals


def learned(keys, vals=None, key_bits: int = 0, nbuckets: int = 0, model: int = 0, stream=None):
    """Learned-bucket stable sort of uint32 or uint64 keys (in place). Returns
    the stats dict. nbuckets 0 lets the library choose (4096 up to 32768 with n);
    model 0 = the piecewise-linear CDF, 1 = the MLP CDF."""
    st = LearnedStats()
    fn = load().isort_learned if _key_width(keys) == 32 else load().isort_learned_u64
    _check(fn(_ptr(keys), _ptr(vals), keys.numel(), key_bits, nbuckets, model, ctypes.byref(st), _stream(stream)),
           "isort_learned")
    return st.as_dict()


def cdf_train(sorted_sample, key_bits: int = 32, stream=None):
    """Trains the CDF model on a sorted uint32 sample; returns (theta, X, Y, losses) tensors."""
    import torch

    dev = sorted_sample.device
    theta = torch.empty(512, dtype=torch.float32, device=dev)
    X = torch.empty(257, dtype=torch.float32, device=dev)
    Y = torch.empty(257, dtype=torch.float32, device=dev)
    losses = torch.empty(66, dtype=torch.float32, device=dev)
    _check(load().isort_cdf_train(_ptr(sorted_sample), sorted_sample.numel(), key_bits, _ptr(theta), _ptr(X), _ptr(Y),
                                  _ptr(losses), _stream(stream)), "isort_cdf_train")
    return theta, X, Y, losses


def cdf_loss_grad(u, theta, stream=None):
    """(loss, grad) of the CDF model at theta on normalised sorted sample values u."""
    import torch

    grad = torch.empty(512, dtype=torch.float32, device=u.device)
    loss = torch.empty(1, dtype=torch.float32, device=u.device)
    _check(load().isort_cdf_loss_grad(_ptr(u), u.numel(), _ptr(theta), _ptr(grad), _ptr(loss), _stream(stream)),
           "isort_cdf_loss_grad")
    return loss, grad


KEY_TYPES = {"u32": 0, "i32": 1, "f32": 2, "u64": 3, "i64": 4, "f64": 5}


def radix_typed(keys, key_type: str, vals=None, radix_bits: int = 8, stream=None):
    """Stable in-place sort of typed keys (a 4- or 8-byte device tensor whose
    bits are key_type: u32, i32, f32, u64, i64 or f64); floats by IEEE 754
    totalOrder. Returns (keys, vals)."""
    if key_type not in KEY_TYPES:
        raise ValueError(f"key_type must be one of {sorted(KEY_TYPES)}")
    want = 4 if key_type.endswith("32") else 8
    if keys.element_size() != want:
        raise TypeError(f"{key_type} keys need {want}-byte elements, got {keys.element_size()}")
    _check(load().isort_radix_typed(_ptr(keys), KEY_TYPES[key_type], _ptr(vals), keys.numel(), radix_bits,
                                    _stream(stream)), "isort_radix_typed")
    return keys, vals


def mlp_train(sorted_sample, key_bits: int = 32, stream=None):
    """Trains the MLP CDF model on a sorted uint32 sample; returns (params, X, Y, losses) tensors."""
    import torch

    dev = sorted_sample.device
    params = torch.empty(97, dtype=torch.float32, device=dev)
    X = torch.empty(257, dtype=torch.float32, device=dev)
    Y = torch.empty(257, dtype=torch.float32, device=dev)
    losses = torch.empty(66, dtype=torch.float32, device=dev)
    _check(load().isort_mlp_train(_ptr(sorted_sample), sorted_sample.numel(), key_bits, _ptr(params), _ptr(X), _ptr(Y),
                                  _ptr(losses), _stream(stream)), "isort_mlp_train")
    return params, X, Y, losses


def mlp_loss_grad(u, params, stream=None):
    """(loss, grad) of the MLP CDF model at params on normalised sorted sample values u."""
    import torch

    grad = torch.empty(97, dtype=torch.float32, device=u.device)
    loss = torch.empty(1, dtype=torch.float32, device=u.device)
    _check(load().isort_mlp_loss_grad(_ptr(u), u.numel(), _ptr(params), _ptr(grad), _ptr(loss), _stream(stream)),
           "isort_mlp_loss_grad")
    return loss, grad


def cdf_splitters(X, Y, key_width: int = 32, key_bits: int = 0, nbuckets: int = 4096, stream=None):
    import torch

    dt = torch.int32 if key_width == 32 else torch.int64
    out = torch.empty(nbuckets, dtype=dt, device=X.device)
    _check(load().isort_cdf_splitters(_ptr(X), _ptr(Y), key_width, key_bits, nbuckets, _ptr(out), _stream(stream)),
           "isort_cdf_splitters")
    return out


def bucket_ids(keys, X, Y, nbuckets: int = 4096, key_bits: int = 0, stream=None):
    """The learned model's bucket of every key (int32 tensor of bucket ids)."""
    import torch

    w = _key_width(keys)
    ids = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device)
    _check(load().isort_bucket_ids(_ptr(keys), w, keys.numel(), key_bits, _ptr(X), _ptr(Y), nbuckets, _ptr(ids),
                                   _stream(stream)), "isort_bucket_ids")
    return ids


def sample(keys, m: int, seed: int, stream=None):
    """m keys drawn at SplitMix64-chosen indices (a new device tensor)."""
    import torch

    out = torch.empty(m, dtype=keys.dtype, device=keys.device)
    _check(load().isort_sample(_ptr(keys), _key_width(keys), keys.numel(), m, seed & (2**64 - 1), _ptr(out),
                               _stream(stream)), "isort_sample")
    return out


def partition(keys, vals, sorted_sample, parts: int, stream=None):
    """Stable routing of keys (and payloads) into the ranges of `parts - 1`
    splitters chosen regularly from `sorted_sample`; returns (keys_out,
    vals_out, counts) with counts an int64 device tensor of `parts` entries."""
    import torch

    ko = torch.empty_like(keys)
    vo = None if vals is None else torch.empty_like(vals)
    counts = torch.empty(parts, dtype=torch.int64, device=keys.device)
    fn = load().isort_partition if _key_width(keys) == 32 else load().isort_partition_u64
    _check(fn(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), keys.numel(), _ptr(sorted_sample), sorted_sample.numel(),
              parts, _ptr(counts), _stream(stream)), "isort_partition")
    return ko, vo, counts


def autotune(enable: bool, cache_path: str | None = None):
    """Turn the launch-shape autotuner on (with an optional cache file) or off."""
    _check(load().isort_autotune(1 if enable else 0, cache_path.encode() if cache_path else None), "isort_autotune")


def set_sync(on: bool):
    _check(load().isort_set_sync(1 if on else 0), "isort_set_sync")


def device_status(clear: bool = True, stream=None) -> int:
    return int(load().isort_device_status(1 if clear else 0, _stream(stream)))


def set_spin_limit(microseconds: int):
    _check(load().isort_set_spin_limit(int(microseconds)), "isort_set_spin_limit")


def launch_count() -> int:
    return int(load().isort_launch_count())


def profile_enable(on: bool):
    _check(load().isort_profile_enable(1 if on else 0), "isort_profile_enable")


def profile_read(max_entries: int = 64):
    """{kernel name: (launches, total_ms)} recorded since the last read."""
    buf = (KernelTime * max_entries)()
    k = load().isort_profile_read(buf, max_entries)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(k)}

"""Learned-bucket sort on the GPU against the oracle.

The sort's output is compared bit for bit with the oracle's stable LSD sort
(payload = input index, so stability is checked too). The model's pieces are
checked one by one on inputs the test makes itself: the gradient against the
oracle's double-precision chain rule, the splitter table and the bucket ids
bit for bit against the oracle's (same fp32 operations in the same order),
and the training record against the oracle's loss at the trained parameters.
"""
import numpy as np
import pytest

import gen
import gen.workloads
import oracle
from tests._util import to_dev, to_np

pytestmark = pytest.mark.gpu

N = 1 << 22


def _keys(kind, n=N, seed=6):
    if kind == "uniform":
        return gen.uniform_u32(n, 32, seed, 0)
    if kind == "range20":
        return gen.uniform_u32(n, 20, seed, 2)
    if kind == "zipf":
        return gen.zipf_u32(n, 1.1, seed, 10)
    if kind == "lognormal":
        return gen.lognormal_u32(n, 20.0, 2.0, seed, 11)
    if kind == "gmm":
        return gen.gmm_u32(n, 16, float(1 << 20), seed, 12)
    raise ValueError(kind)


def _learned_vs_oracle(isort, keys, vals=True, key_bits=0, nbuckets=4096):
    v = gen.iota_u32(keys.size) if vals else None
    dk = to_dev(keys)
    dv = to_dev(v) if vals else None
    st = isort.learned(dk, dv, key_bits=key_bits, nbuckets=nbuckets)
    ek, ev = oracle.lsd(keys, v, key_bits=key_bits, radix_bits=8)
    assert np.array_equal(to_np(dk, np.uint32), ek)
    if vals:
        assert np.array_equal(to_np(dv, np.uint32), ev)
    return st


@pytest.mark.parametrize("kind", ["uniform", "zipf", "lognormal", "gmm"])
def test_learned_matches_oracle(cuda_lib, kind):
    st = _learned_vs_oracle(cuda_lib, _keys(kind))
    assert st["nbuckets"] == 4096 and st["train_steps"] == 64
    # the returned model is never worse than the initial one (the two losses
    # come from separate float reductions: allow their rounding)
    assert np.isfinite(st["train_loss"]) and st["train_loss"] <= st["train_loss_initial"] * (1 + 1e-5)
    if kind == "uniform":
        assert not st["fell_back_to_lsd"]
        assert st["imbalance_max_over_mean"] < 2.0


@pytest.mark.parametrize("kind", ["lognormal", "zipf"])
def test_learned_full_size_keys_only(cuda_lib, kind):
    """The benchmark's learned workload: 2^28 skewed u32 keys, keys only,
    bucket count chosen by the library, against the oracle's sort."""
    keys = gen.workloads.skewed(kind, 1 << 28)
    dk = to_dev(keys)
    st = cuda_lib.learned(dk, None)
    got = to_np(dk, np.uint32)
    del dk
    ek, _ = oracle.lsd(keys, None, 0, 8)
    assert np.array_equal(got, ek)
    if kind == "lognormal":
        assert st["nbuckets"] == 16384 and not st["fell_back_to_lsd"]


def _u64_vs_oracle(isort, keys, vals=True, key_bits=0):
    v = gen.iota_u32(keys.size) if vals else None
    dk = to_dev(keys)
    dv = to_dev(v) if vals else None
    st = isort.learned(dk, dv, key_bits=key_bits)
    ek, ev = oracle.lsd(keys, v, key_bits=key_bits, radix_bits=8)
    assert np.array_equal(to_np(dk, np.uint64), ek)
    if vals:
        assert np.array_equal(to_np(dv, np.uint32), ev)
    return st


@pytest.mark.parametrize("bits", [64, 48])
def test_learned_u64_uniform(cuda_lib, bits):
    keys = gen.uniform_u64((1 << 22) + 99, bits, 5, 0 if bits == 64 else 2)
    st = _u64_vs_oracle(cuda_lib, keys, key_bits=bits)
    assert not st["fell_back_to_lsd"] and st["imbalance_max_over_mean"] < 2.0
    # the fit starts from the sorted sample's quantiles: a small loss only if
    # the sample came out sorted (an unsorted sample puts it near 0.1)
    assert st["train_loss_initial"] < 1e-5


def test_learned_u64_skewed_and_keys_only(cuda_lib):
    """u64 keys whose high half is lognormal and low half uniform, plus runs of
    equal keys: narrow buckets split again on chip."""
    n = 1 << 22
    hi = gen.lognormal_u32(n, 20.0, 2.0, 14, 11).astype(np.uint64)
    lo = gen.uniform_u32(n, 32, 14, 1).astype(np.uint64)
    keys = (hi << np.uint64(32)) | lo
    keys[: n // 8] = keys[7]
    _u64_vs_oracle(cuda_lib, keys)
    _u64_vs_oracle(cuda_lib, keys, vals=False)


def test_learned_u64_full_size(cuda_lib):
    """The 64-bit workload: 2^27 u64 keys uniform on [0, 2^64), payload = index."""
    keys, vals = gen.workloads.wide_u64()
    dk, dv = to_dev(keys), to_dev(vals)
    st = cuda_lib.learned(dk, dv)
    gk, gv = to_np(dk, np.uint64), to_np(dv, np.uint32)
    del dk, dv
    ek, ev = oracle.lsd(keys, vals, 0, 8)
    assert np.array_equal(gk, ek) and np.array_equal(gv, ev)
    assert not st["fell_back_to_lsd"]


def test_learned_keys_only_and_key_bits(cuda_lib):
    keys = _keys("range20", (1 << 20) + 12345, seed=7)
    st = _learned_vs_oracle(cuda_lib, keys, vals=False, key_bits=20)
    assert not st["fell_back_to_lsd"]


@pytest.mark.parametrize("n,nb", [(1 << 18, 4096), ((1 << 18) + 1, 64), ((1 << 21) + 777, 256), (3_000_001, 16384),
                                  ((1 << 18) - 1, 4096)])
def test_learned_sizes_and_bucket_counts(cuda_lib, n, nb):
    st = _learned_vs_oracle(cuda_lib, _keys("gmm", n, seed=8), nbuckets=nb)
    assert st["fell_back_to_lsd"] == (1 if n < (1 << 18) else 0)


def test_learned_auto_bucket_count(cuda_lib):
    """nbuckets = 0: 4096 doubled while n / nbuckets > 16384."""
    keys = _keys("gmm", (1 << 26) + 5, seed=13)
    st = _learned_vs_oracle(cuda_lib, keys, vals=False, nbuckets=0)
    assert st["nbuckets"] == 8192 and not st["fell_back_to_lsd"]


def test_learned_one_key_value_falls_back(cuda_lib):
    keys = np.full(1 << 19, 0xDEADBEEF, np.uint32)
    st = _learned_vs_oracle(cuda_lib, keys)
    assert st["fell_back_to_lsd"] == 1 and st["overflow_fraction"] > 0.5


def test_learned_heavy_buckets_finish_by_plain_rounds(cuda_lib):
    """A tenth of the keys on one value and a tenth in a narrow band: some
    buckets exceed the on-chip capacity but not half of the keys."""
    n = 1 << 21
    keys = gen.uniform_u32(n, 32, 9, 0)
    keys[: n // 10] = 12345678
    keys[n // 10: n // 5] = (12345678 + (gen.uniform_u32(n // 10, 32, 9, 1) % 4096)).astype(np.uint32)
    st = _learned_vs_oracle(cuda_lib, keys)
    assert not st["fell_back_to_lsd"]


def test_learned_overflow_buckets_apart_are_sorted_together(cuda_lib):
    """Two narrow bands far apart, each a fifth of the keys: several buckets
    over the on-chip capacity in separate places, gathered, sorted by one call
    of the plain rounds and scattered back (payload = index checks stability)."""
    n = (1 << 21) + 77
    keys = gen.uniform_u32(n, 32, 21, 0)
    band = gen.uniform_u32(n, 12, 21, 1)
    keys[: n // 5] = (100_000_000 + band[: n // 5]).astype(np.uint32)
    keys[n // 5: 2 * n // 5] = (3_000_000_000 + band[n // 5: 2 * n // 5]).astype(np.uint32)
    st = _learned_vs_oracle(cuda_lib, keys)
    assert st["overflow_buckets"] >= 2 and not st["fell_back_to_lsd"]
    _learned_vs_oracle(cuda_lib, keys, vals=False)


def test_learned_rejects(cuda_lib):
    import torch

    k = torch.zeros(1 << 19, dtype=torch.int32, device="cuda")
    with pytest.raises(cuda_lib.IsortError, match="INVALID|invalid"):
        cuda_lib.learned(k, model=3)
    with pytest.raises(cuda_lib.IsortError):
        cuda_lib.learned(k, nbuckets=65536)
    big = torch.full((1 << 19,), 1 << 21, dtype=torch.int32, device="cuda")
    with pytest.raises(cuda_lib.IsortError, match="RANGE|range"):
        cuda_lib.learned(big, key_bits=20)
    assert int(big[0]) == 1 << 21 and int(big[-1]) == 1 << 21  # untouched


# ------------------------------------------------------------------ the model's pieces

def _random_theta(seed):
    r = np.random.default_rng(seed)
    return r.normal(0.0, 0.8, 512)


def _sample_u(seed, m=1 << 16):
    keys = np.sort(gen.lognormal_u32(m, 20.0, 2.0, seed, 11))
    return keys.astype(np.float32) * np.float32(2.0 ** -32)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_oracle(cuda_lib, seed):
    import torch

    u = _sample_u(seed)
    theta = _random_theta(seed)
    loss, g = cuda_lib.cdf_loss_grad(torch.from_numpy(u).cuda(), torch.from_numpy(theta.astype(np.float32)).cuda())
    eloss, eg = oracle.cdf_loss_grad(u.astype(np.float64), theta.astype(np.float32).astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - eloss) <= 1e-4 * eloss + 1e-9
    scale = np.abs(eg).max()
    assert np.all(np.abs(gg - eg) <= 2e-3 * scale + 1e-3 * np.abs(eg)), np.abs(gg - eg).max() / scale


def _test_knots(seed):
    X, Y = oracle.cdf_knots(_random_theta(seed))
    return X.astype(np.float32), Y.astype(np.float32)


@pytest.mark.parametrize("width,kb,B", [(32, 32, 4096), (32, 20, 1000), (32, 32, 65536), (64, 64, 4096),
                                        (64, 40, 2)])
def test_splitters_bit_exact(cuda_lib, width, kb, B):
    import torch

    X, Y = _test_knots(width + kb + B)
    s = cuda_lib.cdf_splitters(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), key_width=width, key_bits=kb,
                               nbuckets=B)
    got = to_np(s, np.uint32 if width == 32 else np.uint64).astype(np.uint64)
    exp = oracle.splitters(X, Y, width, kb, B)
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("width,kb,B", [(32, 32, 4096), (32, 32, 16384), (32, 20, 1000), (64, 64, 4096),
                                        (32, 32, 3), (32, 32, 65536)])
def test_bucket_ids_bit_exact(cuda_lib, width, kb, B):
    import torch

    X, Y = _test_knots(100 + B + kb)
    split = oracle.splitters(X, Y, width, kb, B)
    n = 1_000_003
    if width == 32:
        keys = gen.uniform_u32(n, kb, 10, 0)
        keys[:1000] = split[B // 2].astype(np.uint32)  # the first keys of buckets and their predecessors
        keys[1000:2000] = (np.maximum(split[B // 2], 1) - 1).astype(np.uint32)
    else:
        keys = gen.uniform_u64(n, 64, 10, 0)
        keys[:1000] = split[B // 2]
        keys[1000:2000] = np.maximum(split[B // 2], 1) - 1
    ids = cuda_lib.bucket_ids(to_dev(keys), torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), B, kb)
    got = to_np(ids, np.uint32)
    assert np.array_equal(got, oracle.bucket_ids(keys, X, Y, kb, B))
    # and the GPU's own splitter table bounds the GPU's buckets
    s = cuda_lib.cdf_splitters(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), key_width=width, key_bits=kb,
                               nbuckets=B)
    gs = to_np(s, np.uint32 if width == 32 else np.uint64).astype(np.uint64)
    assert np.array_equal(got, np.searchsorted(gs[1:], keys.astype(np.uint64), side="right").astype(np.uint32))


def test_training_reduces_loss_and_reports_it(cuda_lib):
    import torch

    keys = np.sort(gen.lognormal_u32(1 << 16, 20.0, 2.0, 12, 11))
    theta, X, Y, losses = cuda_lib.cdf_train(to_dev(keys))
    L = losses.cpu().numpy()
    assert np.all(np.isfinite(L))
    # the returned model is the best seen: no worse than any step, and
    # training improved on the quantile initialisation
    assert L[64] <= L[:64].min() and L[64] < L[65]
    u = keys.astype(np.float32) * np.float32(2.0 ** -32)
    eloss, _ = oracle.cdf_loss_grad(u.astype(np.float64), theta.cpu().numpy().astype(np.float64), with_grad=False)
    assert abs(L[64] - eloss) <= 1e-3 * eloss + 1e-9
    # the knots the call returns are the ones theta defines
    eX, eY = oracle.cdf_knots(theta.cpu().numpy().astype(np.float64))
    assert np.allclose(X.cpu().numpy(), eX, atol=2e-6) and np.allclose(Y.cpu().numpy(), eY, atol=2e-6)


@pytest.mark.parametrize("kind", ["lognormal", "gmm"])
def test_model_beats_equal_width_buckets(cuda_lib, kind):
    """The point of the model: on skewed keys its buckets are far better
    balanced than 4096 equal-width key ranges (the MSD split with no model).
    Measured at 2^22 keys: lognormal well over 8x, the 16-component mixture
    about 5x (a 256-segment model cannot follow 16 narrow peaks bucket by
    bucket)."""
    keys = _keys(kind)
    counts = np.bincount(keys >> 20, minlength=4096)
    plain = counts.max() / (keys.size / 4096)
    st = cuda_lib.learned(to_dev(keys), None)
    assert st["imbalance_max_over_mean"] * 4 < plain, (st["imbalance_max_over_mean"], plain)


# ------------------------------------------------------------------ without the model

@pytest.mark.parametrize("kind", ["lognormal", "gmm"])
def test_regular_sampling_matches_oracle(cuda_lib, kind):
    """model 2: the untrained quantile table (regular sampling)."""
    keys = _keys(kind, (1 << 21) + 5)
    v = gen.iota_u32(keys.size)
    dk, dv = to_dev(keys), to_dev(v)
    st = cuda_lib.learned(dk, dv, model=2)
    ek, ev = oracle.lsd(keys, v, 0, 8)
    assert np.array_equal(to_np(dk, np.uint32), ek) and np.array_equal(to_np(dv, np.uint32), ev)
    assert st["train_steps"] == 0 and st["train_loss"] == st["train_loss_initial"]


def _equal_width_imbalance(keys, nbuckets):
    """max / mean bucket size of the plain MSD split (top bits of the key: the
    bucketing without any CDF model)."""
    counts = np.bincount(keys >> np.uint32(32 - int(np.log2(nbuckets))), minlength=nbuckets)
    return counts.max() / (keys.size / nbuckets)


@pytest.mark.parametrize("kind", ["lognormal", "gmm"])
def test_trained_model_vs_the_method_without_it(cuda_lib, kind):
    """What training buys, measured: the fit lowers the sample loss of its
    regular-sampling start (it can fail to: the assertion is strict); the
    model's buckets are far better balanced than the plain MSD split by the
    top bits of the key; and against regular sampling itself (Section 2) the
    trained model is no worse balanced. All three sorts are exact."""
    keys = _keys(kind)
    ek, _ = oracle.lsd(keys, None, 0, 8)
    res = {}
    for model in (2, 0, 1):
        dk = to_dev(keys)
        res[model] = cuda_lib.learned(dk, None, model=model)
        assert np.array_equal(to_np(dk, np.uint32), ek)
    B = res[0]["nbuckets"]
    plain = _equal_width_imbalance(keys, B)
    print(kind, "equal-width", plain, {m: (r["train_loss_initial"], r["train_loss"], r["imbalance_max_over_mean"],
                                           r["overflow_fraction"]) for m, r in res.items()})
    # each fit makes progress from its start (the piecewise-linear model starts
    # from the regular-sampling table itself)
    assert res[0]["train_loss"] < 0.99 * res[0]["train_loss_initial"]
    assert res[0]["train_loss_initial"] == pytest.approx(res[2]["train_loss"], rel=1e-6)
    assert res[1]["train_loss"] < 0.5 * res[1]["train_loss_initial"]
    # the CDF model (trained or regular) against no model at all
    for m in (0, 1, 2):
        assert res[m]["imbalance_max_over_mean"] < plain
    # trained against regular sampling: not worse balanced (measured: the
    # piecewise-linear fit leaves the balance where its quantile start has it;
    # the MLP is 2-11 % better balanced)
    for m in (0, 1):
        assert res[m]["imbalance_max_over_mean"] <= res[2]["imbalance_max_over_mean"] * 1.05
        assert res[m]["overflow_fraction"] <= res[2]["overflow_fraction"] + 0.01

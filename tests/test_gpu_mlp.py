"""The MLP CDF model (learned sort with model = 1) on the GPU against the oracle.

The sort's output is compared bit for bit with the oracle's stable LSD sort.
The model's pieces are checked on inputs the test makes itself: the loss and
gradient of the cluster fit against the oracle's double-precision chain rule
(ragged point counts included); the training record against the oracle's
loss at the returned parameters; the table against the oracle's F at the
sample's quantile keys, made non-decreasing.
"""
import numpy as np
import pytest

import gen
import oracle
from tests._util import to_dev, to_np

pytestmark = pytest.mark.gpu

H = oracle.MLP_HIDDEN


def _keys(kind, n, seed):
    if kind == "uniform":
        return gen.uniform_u32(n, 32, seed, 0)
    if kind == "lognormal":
        return gen.lognormal_u32(n, 20.0, 2.0, seed, 11)
    if kind == "gmm":
        return gen.gmm_u32(n, 16, float(1 << 20), seed, 12)
    if kind == "zipf":
        return gen.zipf_u32(n, 1.1, seed, 10)
    raise ValueError(kind)


def _u(kind, m, seed):
    return np.sort(_keys(kind, m, seed)).astype(np.float32) * np.float32(2.0 ** -32)


def _params_near_quantiles(u, seed):
    """Parameters shaped like the library's start (units on the sample's
    quantiles), perturbed: the region the fit works in."""
    r = np.random.default_rng(seed)
    q = np.quantile(u.astype(np.float64), np.arange(H + 1) / H)
    c = np.quantile(u.astype(np.float64), (np.arange(H) + 0.5) / H)
    w1 = np.minimum(4.0 / np.maximum(np.diff(q), 4e-6), 1e6) * np.exp(r.normal(0, 0.3, H))
    a1 = np.where(w1 > 20, w1, np.log(np.expm1(np.minimum(w1, 20))))
    b1 = -w1 * c + r.normal(0, 0.5, H)
    a2 = np.log(np.expm1(1.0 / H)) + r.normal(0, 0.5, H)
    return np.concatenate([a1, b1, a2, [0.25]]).astype(np.float32)


@pytest.mark.parametrize("kind,m,seed", [("lognormal", 4096, 1), ("gmm", 3001, 2), ("uniform", 65536, 3),
                                         ("zipf", 777, 4)])
def test_mlp_gradient_matches_oracle(cuda_lib, kind, m, seed):
    import torch

    u = _u(kind, m, seed)
    p = _params_near_quantiles(u, seed)
    loss, g = cuda_lib.mlp_loss_grad(torch.from_numpy(u).cuda(), torch.from_numpy(p).cuda())
    eloss, eg = oracle.mlp_loss_grad(u.astype(np.float64), p.astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - eloss) <= 1e-4 * eloss + 1e-9, (float(loss.item()), eloss)
    assert gg[-1] == 0.0 and eg[-1] == 0.0
    scale = np.abs(eg).max()
    assert np.all(np.abs(gg - eg) <= 2e-3 * scale + 1e-3 * np.abs(eg)), np.abs(gg - eg).max() / scale


@pytest.mark.parametrize("kind", ["lognormal", "gmm", "uniform"])
def test_mlp_training_record_and_table(cuda_lib, kind):
    m = 1 << 16
    keys = np.sort(_keys(kind, m, 12))
    params, X, Y, losses = cuda_lib.mlp_train(to_dev(keys))
    L = losses.cpu().numpy()
    p = params.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(L)) and np.all(np.isfinite(p))
    # the returned parameters are the best seen, the start included
    assert L[64] <= L[:64].min() and L[64] <= L[65]
    if kind != "uniform":
        assert L[64] < L[65]
    u = keys.astype(np.float32) * np.float32(2.0 ** -32)
    eloss, _ = oracle.mlp_loss_grad(u.astype(np.float64), p, with_grad=False)
    assert abs(L[64] - eloss) <= 1e-3 * eloss + 1e-9
    # the table: quantile knots, F there made non-decreasing
    gX, gY = X.cpu().numpy(), Y.cpu().numpy()
    eX = np.ones(257, np.float32)
    eX[0] = 0.0
    idx = (np.arange(1, 256, dtype=np.uint64) * np.uint64(m)) // np.uint64(256)
    eX[1:256] = np.minimum(keys[idx].astype(np.float32) * np.float32(2.0 ** -32), np.float32(1.0))
    assert np.array_equal(gX, eX)
    F = np.array([oracle.mlp_cdf(p, float(x)) for x in eX])
    F[0], F[-1] = 0.0, 1.0
    eY = np.maximum.accumulate(np.clip(F, 0.0, 1.0))
    assert np.all(np.diff(gY) >= 0) and gY[0] == 0.0 and gY[-1] == 1.0
    assert np.abs(gY - eY).max() < 2e-5, np.abs(gY - eY).max()


def _mlp_vs_oracle(isort, keys, vals=True, key_bits=0, nbuckets=4096, dtype=np.uint32):
    v = gen.iota_u32(keys.size) if vals else None
    dk = to_dev(keys)
    dv = to_dev(v) if vals else None
    st = isort.learned(dk, dv, key_bits=key_bits, nbuckets=nbuckets, model=1)
    ek, ev = oracle.lsd(keys, v, key_bits=key_bits, radix_bits=8)
    assert np.array_equal(to_np(dk, dtype), ek)
    if vals:
        assert np.array_equal(to_np(dv, np.uint32), ev)
    return st


@pytest.mark.parametrize("kind", ["uniform", "zipf", "lognormal", "gmm"])
def test_learned_mlp_matches_oracle(cuda_lib, kind):
    st = _mlp_vs_oracle(cuda_lib, _keys(kind, (1 << 22) + 31, 6))
    assert st["nbuckets"] == 4096 and st["train_steps"] == 64
    assert np.isfinite(st["train_loss"]) and st["train_loss"] <= st["train_loss_initial"] * (1 + 1e-5)
    if kind == "uniform":
        assert not st["fell_back_to_lsd"] and st["imbalance_max_over_mean"] < 2.0


def test_learned_mlp_keys_only_key_bits_and_bucket_counts(cuda_lib):
    keys = gen.uniform_u32((1 << 20) + 12345, 20, 7, 2)
    st = _mlp_vs_oracle(cuda_lib, keys, vals=False, key_bits=20)
    assert not st["fell_back_to_lsd"]
    _mlp_vs_oracle(cuda_lib, _keys("gmm", (1 << 21) + 777, 8), nbuckets=256)
    _mlp_vs_oracle(cuda_lib, _keys("gmm", 3_000_001, 8), nbuckets=16384)


def test_learned_mlp_u64(cuda_lib):
    n = 1 << 22
    hi = gen.lognormal_u32(n, 20.0, 2.0, 14, 11).astype(np.uint64)
    lo = gen.uniform_u32(n, 32, 14, 1).astype(np.uint64)
    keys = (hi << np.uint64(32)) | lo
    st = _mlp_vs_oracle(cuda_lib, keys, dtype=np.uint64)
    assert not st["fell_back_to_lsd"]
    keys = gen.uniform_u64(n + 99, 48, 5, 2)
    _mlp_vs_oracle(cuda_lib, keys, vals=False, key_bits=48, dtype=np.uint64)


def test_mlp_beats_equal_width_buckets(cuda_lib):
    keys = _keys("lognormal", 1 << 22, 6)
    counts = np.bincount(keys >> 20, minlength=4096)
    plain = counts.max() / (keys.size / 4096)
    st = cuda_lib.learned(to_dev(keys), None, model=1)
    assert st["imbalance_max_over_mean"] * 4 < plain, (st["imbalance_max_over_mean"], plain)

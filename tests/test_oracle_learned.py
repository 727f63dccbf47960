"""Pins for the oracle's learned-bucket functions (CPU): the sample index rule
against SplitMix64's published outputs; the bucket model of the identity knots
against numpy's float32 arithmetic; the bucket model's monotonicity and its
agreement with the piecewise-linear CDF in double precision; the splitter
table as the buckets' boundaries (numpy.searchsorted); the loss against its
closed form for the identity model; and the analytic gradient against central
finite differences of the loss."""
import numpy as np
import pytest

import oracle

PUBLISHED = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
             16408922859458223821]


def test_sample_indices_follow_splitmix64():
    # with n = 2^64 - 1, floor(r * n / 2^64) = r - 1 for r > 0
    idx = oracle.sample_indices(2**64 - 1, 5, 1234567)
    assert [int(i) + 1 for i in idx] == PUBLISHED
    # and with n = 2^63 the index is r >> 1
    idx = oracle.sample_indices(2**63, 5, 1234567)
    assert [int(i) for i in idx] == [r >> 1 for r in PUBLISHED]


def identity_knots():
    return np.arange(257, dtype=np.float32) / np.float32(256)


def _f32_bucket_identity(key, B, kb=32):
    u = np.float32(np.float32(key) * np.float32(2.0 ** -kb))
    return min(B - 1, int(np.float32(u * np.float32(B))))


@pytest.mark.parametrize("B", [2, 16, 1000, 4096])
def test_identity_model_buckets_are_scaled_keys(B):
    """With X = Y = j/256 the model is F(u) = u exactly (slope 1, exact
    subtraction), so the bucket is trunc(u B) in float32."""
    X = identity_knots()
    r = np.random.default_rng(B)
    keys = np.concatenate([r.integers(0, 2**32, 2000, dtype=np.uint64),
                           np.array([0, 1, 2**32 - 1, 2**31, 2**24 + 1], np.uint64)])
    for k in keys[:300]:
        assert oracle.bucket_of(X, X, int(k), 32, 32, B) == _f32_bucket_identity(int(k), B), k
    ids = oracle.bucket_ids(keys.astype(np.uint32), X, X, 32, B)
    assert [int(i) for i in ids] == [_f32_bucket_identity(int(k), B) for k in keys]


@pytest.mark.parametrize("B", [2, 16, 4096])
def test_identity_model_splitters_by_bisection(B):
    X = identity_knots()
    s = oracle.splitters(X, X, 32, 32, B)
    assert s[0] == 0 and np.all(np.diff(s.astype(np.int64)) >= 0)
    for b in list(range(1, min(B, 30))) + [B - 1]:
        lo, hi = 0, 2**32 - 1
        while lo < hi:
            mid = (lo + hi) // 2
            if _f32_bucket_identity(mid, B) >= b:
                hi = mid
            else:
                lo = mid + 1
        assert int(s[b]) == lo, b


def _random_knots(seed):
    X, Y = oracle.cdf_knots(np.random.default_rng(seed).normal(0.0, 1.0, 512))
    return X.astype(np.float32), Y.astype(np.float32)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bucket_model_is_monotone(seed):
    """The bucket never decreases as the key grows: over sorted random keys,
    and over every key in a window around each knot (where rounding between
    neighbouring segments could otherwise step back)."""
    X, Y = _random_knots(seed)
    r = np.random.default_rng(seed)
    keys = np.sort(r.integers(0, 2**32, 200_000, dtype=np.uint64)).astype(np.uint32)
    assert np.all(np.diff(oracle.bucket_ids(keys, X, Y, 32, 4096).astype(np.int64)) >= 0)
    for j in range(1, 256, 5):
        c = int(np.float64(X[j]) * 2**32)
        win = np.arange(max(0, c - 600), min(2**32, c + 600), dtype=np.uint64).astype(np.uint32)
        assert np.all(np.diff(oracle.bucket_ids(win, X, Y, 32, 4096).astype(np.int64)) >= 0)


@pytest.mark.parametrize("seed", [4, 5])
def test_bucket_model_matches_pwl_cdf_within_rounding(seed):
    """Against the piecewise-linear CDF in double precision: floor(F(u) B) is
    the bucket up to one step at most (float32 rounding near a boundary)."""
    X, Y = _random_knots(seed)
    r = np.random.default_rng(seed)
    keys = r.integers(0, 2**32, 50_000, dtype=np.uint64).astype(np.uint32)
    u = keys.astype(np.float64) / 2**32
    F = np.interp(u, X.astype(np.float64), Y.astype(np.float64))
    exact = np.minimum(np.floor(F * 4096), 4095)
    got = oracle.bucket_ids(keys, X, Y, 32, 4096).astype(np.float64)
    assert np.max(np.abs(got - exact)) <= 1
    assert np.mean(got == exact) > 0.99


@pytest.mark.parametrize("width,kb", [(32, 32), (32, 20), (64, 64), (64, 40)])
def test_splitters_are_the_bucket_boundaries(width, kb):
    """bucket(k) = #{b >= 1 : s_b <= k}: at random keys and on both sides of
    every splitter."""
    X, Y = _random_knots(kb + width)
    B = 1024
    s = oracle.splitters(X, Y, width, kb, B)
    dt = np.uint32 if width == 32 else np.uint64
    r = np.random.default_rng(kb)
    top = 2**kb
    keys = r.integers(0, top - 1, 20_000, dtype=np.uint64, endpoint=True)
    edges = np.concatenate([s[1:], np.maximum(s[1:], 1) - 1]).astype(np.uint64)
    keys = np.concatenate([keys, edges[edges < np.uint64(top - 1) + np.uint64(1)] if kb < 64 else edges]).astype(dt)
    ids = oracle.bucket_ids(keys, X, Y, kb, B)
    ref = np.searchsorted(s[1:], keys.astype(np.uint64), side="right")
    assert np.array_equal(ids, ref.astype(np.uint32))


def test_knots_of_equal_increments_are_uniform():
    X, Y = oracle.cdf_knots(np.full(512, 0.3))
    assert np.allclose(X, np.arange(257) / 256, atol=1e-15) and np.allclose(Y, X)


def test_identity_model_loss_closed_form():
    r = np.random.default_rng(2)
    u = np.sort(r.random(5000))
    loss, g = oracle.cdf_loss_grad(u, np.zeros(512))
    m = u.size
    ref = np.mean((u - (np.arange(m) + 0.5) / m) ** 2)
    assert abs(loss - ref) < 1e-12 * max(1.0, ref)


@pytest.mark.parametrize("seed", [3, 4])
def test_gradient_matches_finite_differences(seed):
    r = np.random.default_rng(seed)
    u = np.sort(r.lognormal(-2.0, 0.7, 3000) % 1.0)
    theta = r.normal(0.0, 0.6, 512)
    loss, g = oracle.cdf_loss_grad(u, theta)
    h = 1e-6
    for i in list(r.choice(512, 24, replace=False)) + [0, 255, 256, 511]:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (oracle.cdf_loss_grad(u, tp, False)[0] - oracle.cdf_loss_grad(u, tm, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (i, fd, g[i])

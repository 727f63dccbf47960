"""Pins for the oracle's learned-bucket functions (CPU): the sample index rule
against SplitMix64's published outputs, the splitter table of the identity
model against numpy's float32 rounding, bucket ids against numpy.searchsorted,
the loss against its closed form for the identity model, and the analytic
gradient against central finite differences of the loss."""
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


@pytest.mark.parametrize("B", [2, 16, 4096])
def test_identity_model_splitters_match_float32_rounding(B):
    """F(u) = u for X = Y = j/256, so s_b is the first key whose float32 value
    times 2^-32 reaches b/B; found here by bisection on numpy's float32."""
    X = identity_knots()
    s = oracle.splitters(X, X, 32, 32, B)
    assert s[0] == 0 and np.all(np.diff(s.astype(np.int64)) >= 0)
    for b in list(range(1, min(B, 40))) + [B - 1]:
        t = np.float32(b) / np.float32(B)
        lo, hi = 0, 2**32 - 1
        while lo < hi:
            mid = (lo + hi) // 2
            if np.float32(mid) * np.float32(2.0**-32) >= t:
                hi = mid
            else:
                lo = mid + 1
        assert int(s[b]) == lo, b


def test_bucket_ids_match_searchsorted():
    r = np.random.default_rng(1)
    split = np.sort(r.integers(0, 2**32, 4096, dtype=np.uint64))
    split[0] = 0
    split[100:140] = split[100]  # empty buckets
    keys = r.integers(0, 2**32, 200_000, dtype=np.uint64).astype(np.uint32)
    keys[:1000] = np.uint32(split[100])
    ids = oracle.bucket_ids(keys, split)
    ref = np.searchsorted(split[1:], keys.astype(np.uint64), side="right")
    assert np.array_equal(ids, ref.astype(np.uint32))
    k64 = (keys.astype(np.uint64) << np.uint64(20))
    s64 = split << np.uint64(20)
    assert np.array_equal(oracle.bucket_ids(k64, s64), np.searchsorted(s64[1:], k64, side="right").astype(np.uint32))


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

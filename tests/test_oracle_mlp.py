"""Pins for the oracle's alternative CDF model, the 1-32-1 monotone MLP
(softplus weights, sigmoid hidden units, normalised to F(0)=0 and F(1)=1): the end
points and monotonicity for random parameters; the linear limit F(u) -> u for
small centred weights; the staircase limit for steep units, which counts the
unit centres below u (a dropped or misindexed unit moves a stair); the mirror
symmetry of units centred at 1/2; invariance under a permutation of the units
and under the output bias; and the analytic gradient against central finite
differences of the loss."""
import numpy as np
import pytest

import oracle

H = oracle.MLP_HIDDEN


def _pack(a1, b1, a2, b2=0.0):
    return np.concatenate([a1, b1, a2, [b2]]).astype(np.float64)


def _inv_softplus(w):
    w = np.asarray(w, dtype=np.float64)
    return w + np.log(-np.expm1(-w))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_end_points_and_monotone(seed):
    r = np.random.default_rng(seed)
    p = r.normal(0.0, 1.5, oracle.MLP_PARAMS)
    assert oracle.mlp_cdf(p, 0.0) == 0.0
    assert abs(oracle.mlp_cdf(p, 1.0) - 1.0) < 1e-15
    f = np.array([oracle.mlp_cdf(p, u) for u in np.linspace(0, 1, 2001)])
    assert np.all(np.diff(f) >= -1e-15)


def test_linear_limit_of_small_weights():
    # W1 = eps with the units centred on 1/2: sigma is linear to O(eps^3), F(u) = u + O(eps^2)
    eps = 1e-3
    p = _pack(np.full(H, _inv_softplus(eps)), np.full(H, -eps / 2), np.zeros(H))
    for u in np.linspace(0, 1, 11):
        assert abs(oracle.mlp_cdf(p, u) - u) < 1e-6


def test_steep_units_count_centres_below_u():
    r = np.random.default_rng(5)
    c = np.sort(r.uniform(0.05, 0.95, H))
    w = 2.0e4
    p = _pack(np.full(H, _inv_softplus(w)), -w * c, np.full(H, _inv_softplus(1.0 / H)))
    for u in r.uniform(0, 1, 64):
        if np.min(np.abs(u - c)) < 1e-3:
            continue
        # each unit contributes a step of height 1/H at its centre
        assert abs(oracle.mlp_cdf(p, u) - np.count_nonzero(c < u) / H) < 1e-6, u


def test_units_centred_at_half_are_symmetric():
    r = np.random.default_rng(6)
    w = r.uniform(0.5, 12.0, H)
    p = _pack(_inv_softplus(w), -w / 2, r.normal(0, 1, H), 3.0)
    for u in r.uniform(0, 1, 20):
        assert abs(oracle.mlp_cdf(p, 1 - u) - (1 - oracle.mlp_cdf(p, u))) < 1e-12


def test_unit_permutation_and_output_bias_do_not_matter():
    r = np.random.default_rng(7)
    a1, b1, a2 = r.normal(0, 1, H), r.normal(0, 2, H), r.normal(0, 1, H)
    perm = r.permutation(H)
    p = _pack(a1, b1, a2, 0.0)
    q = _pack(a1[perm], b1[perm], a2[perm], -7.5)
    u = np.sort(r.random(500))
    for x in u[::50]:
        assert abs(oracle.mlp_cdf(p, x) - oracle.mlp_cdf(q, x)) < 1e-12
    lp, gp = oracle.mlp_loss_grad(u, p)
    lq, gq = oracle.mlp_loss_grad(u, q)
    assert abs(lp - lq) < 1e-12
    assert np.allclose(gq[:H], gp[:H][perm], atol=1e-12)
    assert gp[-1] == 0.0


def test_loss_of_a_near_identity_model_on_midpoints():
    m = 4000
    u = (np.arange(m) + 0.5) / m
    eps = 1e-3
    p = _pack(np.full(H, _inv_softplus(eps)), np.full(H, -eps / 2), np.zeros(H))
    loss, _ = oracle.mlp_loss_grad(u, p, False)
    assert loss < 1e-12


@pytest.mark.parametrize("seed", [3, 4])
def test_gradient_matches_finite_differences(seed):
    r = np.random.default_rng(seed)
    u = np.sort(r.lognormal(-2.0, 0.7, 2000) % 1.0)
    c = np.quantile(u, (np.arange(H) + 0.5) / H)
    p = _pack(r.normal(2.0, 0.5, H), -np.exp(2.0) * c + r.normal(0, 0.3, H), r.normal(-3.0, 0.5, H))
    loss, g = oracle.mlp_loss_grad(u, p)
    h = 1e-6
    for i in list(r.choice(3 * H, 20, replace=False)) + [0, H, 2 * H, 3 * H - 1, 3 * H]:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(u, pp, False)[0] - oracle.mlp_loss_grad(u, pm, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10, (i, fd, g[i])

"""The MBSP cost model (Section 3) against the closed forms the paper derives
with g = 5G (eqs. TsG, Tp4, Tp2, ToG, TbG) and against the values it prints
from them in Observations 7-9 (tests/golden/mbsp_observations.json)."""
import json
import math
import os

import pytest

from paper_1708_09495_gb300 import mbsp

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mbsp_observations.json")))


@pytest.mark.parametrize("N", [1e3, 1e6, 2.0 ** 28])
def test_serial_closed_form(N):
    G = 1.0
    assert math.isclose(mbsp.Ts(N, 5 * G, G, 256), 68 * N * G)


@pytest.mark.parametrize("n,p", [(1e6, 4), (2.0 ** 20, 16), (5e5, 2)])
def test_parallel_closed_forms(n, p):
    G = 1.0
    assert math.isclose(mbsp.Tp(n / p, 5 * G, G, p, 256), (88 * n / p + 40 * 256 * p) * G)
    assert math.isclose(mbsp.Tp(n / p, 5 * G, G, p, 256 ** 2), (44 * n / p + 20 * 256 ** 2 * p) * G)
    assert math.isclose(mbsp.To(n, 5 * G, G, p), (68 * n / p + 20 * n) * G)
    lg = math.log2(p)
    assert math.isclose(mbsp.Tb(n, 5 * G, G, p), (68 * n / p + 10 * n * lg * (lg + 1) / p) * G)


def test_observation7_bounds():
    o = GOLD["obs7"]
    for p, b in zip(o["p"], o["bound"]):
        assert abs(mbsp.obs7_speedup_bound(p) - b) <= o["tol"], p
        # the finite-n ratio approaches the bound from below
        assert mbsp.obs7_speedup_bound(p, 1e6) < mbsp.obs7_speedup_bound(p) < 0.78 * p


def test_observation8_ratios():
    o = GOLD["obs8"]
    worst_small = max(mbsp.obs8_ratio(p) - 1 for p in o["p_small"])
    assert abs(worst_small - o["up_to_small"]) <= o["tol"]
    assert abs((mbsp.obs8_ratio(o["p_large"]) - 1) - o["up_to_large"]) <= o["tol"]
    for p in o["p_small"] + [o["p_large"]]:
        # the equations' form is below the observation's lg^2 form
        assert 1 < mbsp.obs8_ratio(p, approx=False) <= mbsp.obs8_ratio(p)


@pytest.mark.parametrize("key", ["obs9_amd", "obs9_intel"])
def test_observation9_speedups(key):
    o = GOLD[key]
    for p, s in zip(o["p"], o["speedup"]):
        assert abs(mbsp.obs9_speedup(p) - s) <= o["tol"], (p, mbsp.obs9_speedup(p))


def test_gb300_hbm_term_counts_bytes():
    # radix 2^8, u32 pairs: 4 rounds x (4 + 2 x 8) B = 80 B per key
    assert math.isclose(mbsp.gb300_lsd_hbm_seconds(1000, 8, True, 1.0), 80 * 1000 / 1e9)
    assert math.isclose(mbsp.gb300_lsd_hbm_seconds(1000, 16, False, 1.0), 2 * 12 * 1000 / 1e9)

"""Generator checks (CPU): the published SplitMix64 test vector, golden digests
of the integer-only streams, thread-count independence, and the shape of each
distribution."""
import json
import math
import os

import numpy as np
import pytest

import gen
from gen import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gen_digests.json")


def test_splitmix64_published_vector():
    # SplitMix64 (Steele, Lea & Flood 2014) from state 1234567: the first five
    # outputs of the authors' reference sequence.
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    assert [gen.splitmix_raw(1234567, i) for i in range(5)] == want


def test_golden_digests():
    with open(GOLDEN) as f:
        cases = json.load(f)
    for c in cases:
        a = getattr(gen, c["fn"])(c["n"], **c["kw"])
        assert gen.fnv1a(a) == c["fnv1a"], c
        assert int(a[0]) == c["first"]


@pytest.mark.parametrize("fn,args", [
    ("uniform_u32", (300_000, 32, 9, 0)),
    ("uniform_u64", (300_000, 48, 9, 0)),
    ("zipf_u32", (200_000, 1.1, 9, 0)),
    ("lognormal_u32", (200_000, 20.0, 2.0, 9, 0)),
    ("gmm_u32", (200_000, 16, float(1 << 20), 9, 0)),
])
def test_thread_count_independent(fn, args):
    gen.set_threads(1)
    a = getattr(gen, fn)(*args)
    gen.set_threads(7)
    b = getattr(gen, fn)(*args)
    gen.set_threads(0)
    assert np.array_equal(a, b)


def test_uniform_range_and_bits():
    a = gen.uniform_u32(1 << 16, 20, 3)
    assert int(a.max()) < (1 << 20) and int(a.max()) > (1 << 20) - 200
    b = gen.uniform_u64(1 << 16, 48, 5)
    assert int(b.max()) < (1 << 48)
    c = gen.uniform_u32(1 << 16, 32, 1)
    assert abs(float(c.mean()) / 2**32 - 0.5) < 0.01


def test_zipf_top_rank_mass():
    """P(rank 1) = 1 / sum_{k<=N} k^-1.1 with N = 2^32-1 (truncated Zipf)."""
    zeta = pytest.importorskip("scipy.special").zeta
    s, N = 1.1, 2**32 - 1
    # tail sum_{k>N} k^-s by Euler-Maclaurin: N^(1-s)/(s-1) - N^-s/2
    HN = zeta(s) - (N ** (1 - s) / (s - 1) - N ** (-s) / 2)
    n = 1 << 20
    a = gen.zipf_u32(n, s, 6, 10)
    top = np.count_nonzero(a == gen.mix32(1)) / n
    assert abs(top - 1 / HN) < 0.003
    two = np.count_nonzero(a == gen.mix32(2)) / n
    assert abs(two - 2 ** -s / HN) < 0.003


def test_lognormal_truncated_median():
    """Truncation at 2^32 removes P(Z > (ln 2^32 - 20)/2); the median of what
    remains is exp(20 + 2 * Phi^-1(q / 2)) with q the kept mass."""
    stats = pytest.importorskip("scipy.stats")
    q = stats.norm.cdf((32 * math.log(2) - 20) / 2)
    med = math.exp(20 + 2 * stats.norm.ppf(q / 2))
    a = gen.lognormal_u32(1 << 20, 20.0, 2.0, 6, 11)
    assert abs(float(np.median(a)) / med - 1) < 0.02


def test_gmm_clusters():
    a = gen.gmm_u32(1 << 18, 16, float(1 << 20), 6, 12).astype(np.float64)
    means = np.array([gen.draw(6, 13, c) >> 11 for c in range(16)], np.float64) / 2**53 * 2**32
    d = np.min(np.abs(a[:, None] - means[None, :]), axis=1)
    assert np.mean(d < 5 * 2**20) > 0.999


def test_segment_offsets():
    L = gen.loguniform_lengths(200_000, 2, 65536, 4)
    assert int(L.min()) >= 2 and int(L.max()) <= 65536
    assert abs(np.mean(np.log(L.astype(np.float64))) - (math.log(2) + math.log(65536)) / 2) < 0.05
    off = workloads.segment_offsets()
    assert int(off[-1]) <= workloads.SEG_CAP
    nxt = int(off[-1]) + int(L[off.size - 1])
    assert nxt > workloads.SEG_CAP  # longest prefix under the cap
    assert 30_000 < off.size - 1 < 60_000

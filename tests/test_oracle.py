"""Pins for the oracle (CPU only).

The oracle is checked against things other than itself: brute force on tiny
inputs (exhaustively for n <= 5 over an adversarial value set), the library's
own stable sort (numpy ``argsort(kind="stable")`` and Python ``sorted``, the
textbook special case), digit counts taken by ``numpy.bincount``, the stage
counts the paper states for BTN (lg p (lg p + 1) / 2, Section 2) and OET (p
rounds, Section 2), and invariants. ``test_mutants_are_caught`` builds
deliberately broken oracles and shows that these pins fail on each of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

VALUES4 = np.array([0, 1, 2, 0xFFFFFFFF], np.uint32)


def ref_stable(keys, vals=None):
    """Library special case: numpy's stable argsort."""
    order = np.argsort(keys, kind="stable")
    return keys[order], (None if vals is None else vals[order])


def rng(seed):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------- LSD


@pytest.mark.parametrize("rb", [1, 3, 8, 11, 16])
def test_lsd_exhaustive_tiny(rb):
    """Every array of length <= 5 over {0, 1, 2, 2^32-1}, payload = index,
    equals brute-force insertion sort and Python's stable ``sorted``."""
    for n in range(0, 6):
        for tup in itertools.product(range(4), repeat=n):
            k = VALUES4[list(tup)] if n else np.zeros(0, np.uint32)
            v = np.arange(n, dtype=np.uint32)
            ok, ov = oracle.lsd(k, v, 32, rb)
            bk, bv = oracle.insertion(k, v)
            pairs = sorted(zip(k.tolist(), v.tolist()), key=lambda t: t[0])
            assert ok.tolist() == bk.tolist() == [a for a, _ in pairs]
            assert ov.tolist() == bv.tolist() == [b for _, b in pairs]


@pytest.mark.parametrize("seed", range(40))
def test_lsd_small_random_vs_bruteforce(seed):
    r = rng(seed)
    n = int(r.integers(0, 65))
    key_bits = int(r.choice([1, 5, 8, 11, 20, 31, 32]))
    rb = int(r.integers(1, 17))
    mode = seed % 4
    if mode == 0:
        k = r.integers(0, 1 << key_bits, n, dtype=np.uint64).astype(np.uint32)
    elif mode == 1:
        k = r.choice(np.array([0, (1 << key_bits) - 1], np.uint64), n).astype(np.uint32)
    elif mode == 2:
        k = np.sort(r.integers(0, 1 << key_bits, n, dtype=np.uint64)).astype(np.uint32)[::-1].copy()
    else:
        k = np.full(n, (1 << key_bits) - 1, np.uint32)
    v = np.arange(n, dtype=np.uint32)
    ok, ov = oracle.lsd(k, v, key_bits, rb)
    bk, bv = oracle.insertion(k, v)
    rk, rv = ref_stable(k, v)
    assert np.array_equal(ok, bk) and np.array_equal(ov, bv)
    assert np.array_equal(ok, rk) and np.array_equal(ov, rv)


@pytest.mark.parametrize("rb,key_bits", [(8, 32), (11, 32), (8, 20), (11, 20), (16, 32), (5, 32), (13, 26)])
def test_lsd_large_vs_numpy(rb, key_bits):
    r = rng(rb * 100 + key_bits)
    n = 1 << 18
    k = r.integers(0, 1 << key_bits, n, dtype=np.uint64).astype(np.uint32)
    v = np.arange(n, dtype=np.uint32)
    ok, ov = oracle.lsd(k, v, key_bits, rb)
    rk, rv = ref_stable(k, v)
    assert np.array_equal(ok, rk) and np.array_equal(ov, rv)
    ok2, none = oracle.lsd(k, None, key_bits, rb)
    assert none is None and np.array_equal(ok2, rk)


@pytest.mark.parametrize("key_bits,rb", [(64, 8), (48, 8), (64, 11), (37, 16), (1, 1)])
def test_lsd_u64_vs_numpy(key_bits, rb):
    r = rng(key_bits + rb)
    n = 50_000
    hi = (1 << key_bits) - 1
    k = (r.integers(0, 1 << 62, n, dtype=np.uint64) * np.uint64(4) + r.integers(0, 4, n, dtype=np.uint64))
    k &= np.uint64(hi)
    k[: n // 10] = k[n // 10: 2 * (n // 10)]  # duplicates
    v = np.arange(n, dtype=np.uint32)
    ok, ov = oracle.lsd(k, v, key_bits, rb)
    rk, rv = ref_stable(k, v)
    assert np.array_equal(ok, rk) and np.array_equal(ov, rv)


def test_lsd_u64_exhaustive_tiny():
    vals = np.array([0, 1, 1 << 40, (1 << 64) - 1], np.uint64)
    for n in range(5):
        for tup in itertools.product(range(4), repeat=n):
            k = vals[list(tup)] if n else np.zeros(0, np.uint64)
            v = np.arange(n, dtype=np.uint32)
            ok, ov = oracle.lsd(k, v, 64, 8)
            bk, bv = oracle.insertion(k, v)
            assert np.array_equal(ok, bk) and np.array_equal(ov, bv)


def test_lsd_rounds_follow_key_bits():
    """Keys >= 2^key_bits are outside the sort's contract: only the low key_bits
    bits decide the order (the round count is ceil(key_bits / rb))."""
    k = np.array([1 << 20, 1, 0], np.uint32)
    ok, _ = oracle.lsd(k, None, 20, 8)
    assert ok.tolist() == [1 << 20, 0, 1]  # bit 20 is ignored: 0,0,1 by low bits, stable
    assert not oracle.key_range_ok(k, 20) and oracle.key_range_ok(k, 21)


def test_lsd_rejects_bad_args():
    with pytest.raises(ValueError):
        oracle.lsd(np.zeros(4, np.uint32), None, 33, 8)
    with pytest.raises(ValueError):
        oracle.lsd(np.zeros(4, np.uint32), None, 32, 17)
    with pytest.raises(ValueError):
        oracle.lsd(np.zeros(4, np.uint32), None, 32, 0)


# ----------------------------------------------------------------- hist / round


@pytest.mark.parametrize("key_bits,rb", [(32, 8), (32, 11), (20, 8), (20, 11), (64, 8), (48, 8)])
def test_digit_hist_vs_bincount(key_bits, rb):
    r = rng(7)
    n = 100_000
    dt = np.uint32 if key_bits <= 32 else np.uint64
    k = (r.integers(0, 1 << min(key_bits, 63), n, dtype=np.uint64) << np.uint64(max(0, key_bits - 63))).astype(dt)
    h = oracle.digit_hist(k, key_bits, rb)
    P = math.ceil(key_bits / rb)
    assert h.shape == (P, 1 << rb)
    k64 = k.astype(np.uint64)
    for d in range(P):
        w = min(rb, key_bits - d * rb)
        dig = (k64 >> np.uint64(d * rb)) & np.uint64((1 << w) - 1)
        ref = np.bincount(dig.astype(np.int64), minlength=1 << rb)
        assert np.array_equal(h[d], ref)
        assert int(h[d].sum()) == n


@pytest.mark.parametrize("shift,width", [(0, 8), (8, 8), (24, 8), (22, 10), (0, 16), (31, 1)])
def test_count_round_vs_stable_argsort(shift, width):
    r = rng(shift * 17 + width)
    n = 70_000
    k = r.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    v = r.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    ko, vo = oracle.count_round(k, v, shift, width)
    dig = (k >> np.uint32(shift)) & np.uint32((1 << width) - 1)
    order = np.argsort(dig, kind="stable")
    assert np.array_equal(ko, k[order]) and np.array_equal(vo, v[order])


# ----------------------------------------------------------------- BTN / OET


@pytest.mark.parametrize("p", [1, 2, 4, 8, 16, 32, 64, 128])
def test_btn_sorts_and_counts_stages(p):
    lg = int(math.log2(p))
    for n in [0, 1, 2, 3, p - 1, p, p + 1, 7 * p + 3, 1024, 1000]:
        if n < 0:
            continue
        r = rng(n * 31 + p)
        k = r.integers(0, 16, n, dtype=np.uint64).astype(np.uint32)  # many ties
        k[: n // 3] = 0xFFFFFFFF
        v = np.arange(n, dtype=np.uint32)
        ok, ov, st = oracle.btn(k, v, p)
        rk, rv = ref_stable(k, v)
        assert np.array_equal(ok, rk) and np.array_equal(ov, rv)
        if n:
            assert st == lg * (lg + 1) // 2  # Section 2: lg p (lg p + 1)/2 stages


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 8, 13, 32, 128])
def test_oet_sorts_and_counts_rounds(p):
    for n in [0, 1, 2, p, p + 1, 5 * p - 1, 1024, 999]:
        r = rng(n * 7 + p)
        k = r.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        k = np.sort(k)[::-1].copy()  # reverse order: the worst case for transposition
        k[: n // 4] = 5
        v = np.arange(n, dtype=np.uint32)
        ok, ov, rd = oracle.oet(k, v, p)
        rk, rv = ref_stable(k, v)
        assert np.array_equal(ok, rk) and np.array_equal(ov, rv)
        if n:
            assert rd == p  # Section 2: p rounds over p blocks


def test_btn_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.btn(np.zeros(8, np.uint32), None, 3)


# ----------------------------------------------------------------- segmented


def test_segmented_vs_per_segment_numpy():
    r = rng(3)
    lens = r.integers(0, 300, 200)
    off = np.zeros(lens.size + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    n = int(off[-1])
    k = r.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    k[::5] = 7
    v = np.arange(n, dtype=np.uint32)
    ok, ov = oracle.segmented(k, v, off)
    for s in range(lens.size):
        a, b = int(off[s]), int(off[s + 1])
        rk, rv = ref_stable(k[a:b], v[a:b])
        assert np.array_equal(ok[a:b], rk) and np.array_equal(ov[a:b], rv)


# ----------------------------------------------------------------- invariants


def test_invariant_checkers_detect_damage():
    r = rng(11)
    n = 5000
    k = r.integers(0, 50, n, dtype=np.uint64).astype(np.uint32)
    v = np.arange(n, dtype=np.uint32)
    sk, sv = ref_stable(k, v)
    assert oracle.is_sorted(sk) and oracle.is_stable(sk, sv)
    h0 = oracle.multiset_hash(k, v)
    assert oracle.multiset_hash(sk, sv) == h0  # permutation-invariant
    bad = sk.copy(); i = int(np.nonzero(np.diff(sk.astype(np.int64)) > 0)[0][0])
    bad[i], bad[i + 1] = bad[i + 1], bad[i]
    assert not oracle.is_sorted(bad)
    j = int(np.nonzero(np.diff(sk.astype(np.int64)) == 0)[0][0])
    bv = sv.copy(); bv[j], bv[j + 1] = bv[j + 1], bv[j]
    assert not oracle.is_stable(sk, bv)
    assert oracle.multiset_hash(sk, bv) == h0  # same multiset, different order
    # payloads swapped between two different keys: a different multiset
    a, b = 0, n - 1
    bv2 = sv.copy(); bv2[a], bv2[b] = bv2[b], bv2[a]
    assert oracle.multiset_hash(sk, bv2) != h0
    bk = sk.copy(); bk[0] += 1
    assert oracle.multiset_hash(bk, sv) != h0
    # u64 flavour
    k64 = k.astype(np.uint64) << np.uint64(20)
    assert oracle.multiset_hash(k64, v) == oracle.multiset_hash(k64[::-1].copy(), v[::-1].copy())


# ----------------------------------------------------------------- planted mistakes


def _pins_pass(mutant: int) -> bool:
    """Run a compact set of the pins above against a (possibly broken) oracle."""
    try:
        r = rng(5)
        for n in (0, 3, 17, 64, 3000):
            k = r.integers(0, 40, n, dtype=np.uint64).astype(np.uint32) * np.uint32(97)
            v = np.arange(n, dtype=np.uint32)
            rk, rv = ref_stable(k, v)
            for rb, kb in ((8, 32), (11, 32), (5, 13)):
                ok, ov = oracle.lsd(k, v, kb, rb, mutant=mutant)
                if not (np.array_equal(ok, rk) and np.array_equal(ov, rv)):
                    return False
            for p in (2, 4, 8):
                ok, ov, st = oracle.btn(k, v, p, mutant=mutant)
                if not (np.array_equal(ok, rk) and np.array_equal(ov, rv)):
                    return False
            for p in (3, 5, 8):
                rev = np.sort(k)[::-1].copy()
                ok, ov, rd = oracle.oet(rev, v, p, mutant=mutant)
                rk2, rv2 = ref_stable(rev, v)
                if not (np.array_equal(ok, rk2) and np.array_equal(ov, rv2)):
                    return False
        k = r.integers(0, 50, 4000, dtype=np.uint64).astype(np.uint32)
        v = np.arange(4000, dtype=np.uint32)
        sk, sv = ref_stable(k, v)
        bv = sv.copy(); bv[0], bv[-1] = bv[-1], bv[0]
        if oracle.multiset_hash(sk, bv, mutant=mutant) == oracle.multiset_hash(sk, sv, mutant=mutant):
            return False
        return True
    except ValueError:
        return False


def test_pins_pass_on_the_real_oracle():
    assert _pins_pass(0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6])
def test_mutants_are_caught(mutant):
    """Each planted mistake (unstable tie order, payload not moved, short last
    digit dropped, bitonic direction ignored, one OET round short, hash blind to
    the payload) makes at least one pin fail."""
    assert not _pins_pass(mutant)

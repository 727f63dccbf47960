"""The benchmark's own output checks (bench.check_pairs / check_keys) accept
the stable sort and reject planted mistakes: an inversion, an unstable tie, a
duplicated payload, a key that does not match its payload, a key moved across
segments, a changed key in a keys-only result."""
import numpy as np

import bench


def _stable_sort(keys):
    order = np.argsort(keys, kind="stable").astype(np.uint32)
    return keys[order], order


def test_accepts_the_stable_sort():
    r = np.random.default_rng(1)
    keys = r.integers(0, 50, 10_000).astype(np.uint32)
    k, v = _stable_sort(keys)
    assert bench.check_pairs(keys, k, v)["ok"]
    assert bench.check_keys(keys, k)["ok"]


def test_rejects_planted_mistakes():
    r = np.random.default_rng(2)
    keys = r.integers(0, 50, 10_000).astype(np.uint32)
    k, v = _stable_sort(keys)
    i = int(np.nonzero(k[1:] > k[:-1])[0][0])
    k2, v2 = k.copy(), v.copy()  # an inversion
    k2[[i, i + 1]], v2[[i, i + 1]] = k2[[i + 1, i]], v2[[i + 1, i]]
    assert not bench.check_pairs(keys, k2, v2)["non_decreasing"]
    j = int(np.nonzero(k[1:] == k[:-1])[0][0])
    v3 = v.copy()  # an unstable tie
    v3[[j, j + 1]] = v3[[j + 1, j]]
    res = bench.check_pairs(keys, k, v3)
    assert not res["stable"] and not res["ok"]
    v4 = v.copy()  # a duplicated payload
    v4[5] = v4[6]
    assert not bench.check_pairs(keys, k, v4)["payload_permutation"]
    k5 = k.copy()  # a key that is not the input key its payload names
    k5[-1] = k5[-1] + 1
    assert not bench.check_pairs(keys, k5, v)["keys_match_payload"]
    k6 = k.copy()  # keys only: a changed key keeps the order but not the multiset
    k6[-1] = k6[-1] + 1
    res = bench.check_keys(keys, k6)
    assert res["non_decreasing"] and not res["multiset_hash_equal"]


def test_segments():
    off = np.array([0, 3, 7, 10])
    keys = np.array([5, 1, 3, 9, 2, 2, 0, 4, 4, 1], dtype=np.uint32)
    seg = np.repeat(np.arange(3, dtype=np.uint32), np.diff(off))
    out_k, out_v = [], []
    for s in range(3):
        part = keys[off[s]:off[s + 1]]
        o = np.argsort(part, kind="stable")
        out_k.append(part[o])
        out_v.append((o + off[s]).astype(np.uint32))
    k, v = np.concatenate(out_k), np.concatenate(out_v)
    assert bench.check_pairs(keys, k, v, seg)["ok"]
    # a key from segment 0 swapped into segment 1 keeps the keys matching
    # their payloads, but crosses a segment
    k2, v2 = k.copy(), v.copy()
    k2[[2, 3]], v2[[2, 3]] = k2[[3, 2]], v2[[3, 2]]
    assert not bench.check_pairs(keys, k2, v2, seg)["ok"]

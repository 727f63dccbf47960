"""Writes gen_digests.json: FNV-1a digests of the first 1024 outputs of the
integer-only generators (uniform u32/u64, payload index). Calls only ``gen``.

Run from the repository root:  python tests/golden/make_gen_digests.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

CASES = [
    ("uniform_u32", dict(bits=32, seed=1, stream=0)),
    ("uniform_u32", dict(bits=32, seed=2, stream=0)),
    ("uniform_u32", dict(bits=20, seed=3, stream=0)),
    ("uniform_u32", dict(bits=32, seed=4, stream=0)),
    ("uniform_u64", dict(bits=64, seed=5, stream=0)),
    ("uniform_u64", dict(bits=48, seed=5, stream=2)),
]


def digests():
    out = []
    for fn, kw in CASES:
        a = getattr(gen, fn)(1024, **kw)
        out.append({"fn": fn, "kw": kw, "n": 1024, "fnv1a": gen.fnv1a(a), "first": int(a[0])})
    out.append({"fn": "iota_u32", "kw": {}, "n": 1024, "fnv1a": gen.fnv1a(gen.iota_u32(1024)), "first": 0})
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gen_digests.json")
    with open(path, "w") as f:
        json.dump(digests(), f, indent=1)
    print("wrote", path)

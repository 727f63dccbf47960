"""The paper's MBSP cost model of its sorts (Section 3) and the ratios it reads
from it (Section 4, Observations 7-9), in the paper's notation, plus the
model's HBM term instantiated for one GB300.

Notation (Section 3): N keys per processor (n in all, p processors), r the
radix, g the cost of one access to main memory per key word, G the cost of
one access to the fast (cache) memory; 32-bit keys take 32 / lg r rounds.

  Ts(N, g, G, r)    = (32 / lg r) (3 N g + 2 N G)                 serial LSD
  Tp(N, g, G, p, r) = (32 / lg r) (4 N g + 2 N G + 2 p r g)       parallel LSD
  To(n, g, G, p)    = Ts(n/p) + p (4 n/p) g                       OET
  Tb(n, g, G, p)    = Ts(n/p) + (lg p (lg p + 1) / 2) (4 n/p) g   BTN

With g = 5G and r = 2^8: Ts = 68 N G, Tp = (88 n/p + 40 * 256 p) G,
To = (68 n/p + 20 n) G, Tb = (68 n/p + 10 n lg p (lg p + 1) / p) G; with
r = 2^16: Tp = (44 n/p + 20 * 256^2 p) G.

Run as ``python -m paper_1708_09495_gb300.mbsp`` to print the tables. This is
analysis, not part of the sort path.
"""
import math

KEY_BITS = 32


def rounds(r: int, key_bits: int = KEY_BITS) -> float:
    """32 / lg r: the count-sort rounds of a key_bits-bit key (Section 3)."""
    return key_bits / math.log2(r)


def Ts(N, g, G, r=256):
    """Serial radix-r LSD: every round reads the keys to count (N g), reads and
    writes them to output (2 N g), and touches the count array twice per key
    (2 N G)."""
    return rounds(r) * (3 * N * g + 2 * N * G)


def Tp(N, g, G, p, r=256):
    """Parallel radix-r LSD (PR4: r = 2^8, PR2: r = 2^16): the output step
    costs one more access per key for the exchange (4 N g), and the counts'
    scatter and gather cost 2 p r g per round."""
    return rounds(r) * (4 * N * g + 2 * N * G + 2 * p * r * g)


def To(n, g, G, p, r=256):
    """Odd-even transposition: a local LSD sort of n/p keys, then p rounds of
    merge-split at 4 (n/p) g each."""
    return Ts(n / p, g, G, r) + p * (4 * n / p) * g


def Tb(n, g, G, p, r=256):
    """Bitonic: a local LSD sort of n/p keys, then lg p (lg p + 1) / 2
    merge-split stages at 4 (n/p) g each."""
    lg = math.log2(p)
    return Ts(n / p, g, G, r) + (lg * (lg + 1) / 2) * (4 * n / p) * g


def obs7_speedup_bound(p: int, n: float = float("inf")) -> float:
    """Observation 7: Ts(n) / Tp(n/p, p) with g = 5G, r = 2^8; as n grows it
    tends to 68 p / 88 (about 0.75 p)."""
    if math.isinf(n):
        return 68.0 * p / 88.0
    return 68.0 * n / (88.0 * n / p + 40.0 * 256 * p)


def obs8_ratio(p: int, approx: bool = True) -> float:
    """Observation 8: To / Tb with g = 5G. The observation writes the BTN term
    as 10 lg^2 p (approx = True, the form behind its printed 40 % / 70 %);
    the equations give 10 lg p (lg p + 1) (approx = False)."""
    lg = math.log2(p)
    btn = 10 * lg * lg if approx else 10 * lg * (lg + 1)
    return (68 + 20 * p) / (68 + btn)


def obs9_speedup(p: int) -> float:
    """Observation 9: Ts(n) / Tb(n, p) with g = 5G: 68 p / (68 + 10 lg p (lg p + 1))."""
    lg = math.log2(p)
    return 68.0 * p / (68 + 10 * lg * (lg + 1))


def gb300_lsd_hbm_seconds(n: int, radix_bits: int, payload: bool, hbm_gbs: float, key_bytes: int = 4) -> float:
    """The model's main-memory term on one GB300, with g = the bytes of one key
    (and payload) access over the measured copy bandwidth: each round reads the
    keys once to count (3 N g's first access, keys only) and reads and writes
    keys and payloads once to output. A lower bound for the chunked rounds; the
    count step's fast-memory term (2 N G) runs on chip."""
    r_rounds = math.ceil(key_bytes * 8 / radix_bits)
    per_key = r_rounds * (key_bytes + 2 * (key_bytes + (4 if payload else 0)))
    return n * per_key / (hbm_gbs * 1e9)


def _main():
    print("Observation 7: Ts / Tp bound (about 0.75 p)")
    for p in (4, 8, 16):
        print(f"  p = {p:2d}: {obs7_speedup_bound(p):.2f}")
    print("Observation 8: To / Tb (lg^2 form | equations)")
    for p in (2, 4, 8, 16):
        print(f"  p = {p:2d}: {obs8_ratio(p):.3f} | {obs8_ratio(p, approx=False):.3f}")
    print("Observation 9: Ts / Tb")
    for p in (2, 4, 8, 16):
        print(f"  p = {p:2d}: {obs9_speedup(p):.2f}")
    print("GB300 HBM term, 2^28 u32 pairs at 6788 GB/s")
    for rb in (8, 11, 16):
        print(f"  radix 2^{rb}: {gb300_lsd_hbm_seconds(1 << 28, rb, True, 6788.3) * 1e3:.2f} ms")


if __name__ == "__main__":
    _main()

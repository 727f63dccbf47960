"""The sample sort over several processes (paper_1708_09495_gb300.dist): its
exchange logic runs here in two CPU processes over gloo, with the local steps
(sampling, sorting the gathered sample, partition, local sort) done by the
oracle. The concatenation of the processes' ranges must equal the oracle's
stable sort of the concatenated input, payload = global index, for uneven
parts, heavy duplicates, an empty part and 64-bit keys."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

CASES = {
    "uniform_u32": dict(sizes=(30_001, 12_345), bits=32, dup=False, u64=False),
    "duplicates": dict(sizes=(20_000, 20_000), bits=32, dup=True, u64=False),
    "empty_part": dict(sizes=(0, 25_000), bits=32, dup=False, u64=False),
    "narrow_u64": dict(sizes=(17_000, 9_000), bits=40, dup=False, u64=True),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def make_input(case, rank):
    import gen

    c = CASES[case]
    lo = sum(c["sizes"][:rank])
    n = c["sizes"][rank]
    gen_fn = gen.uniform_u64 if c["u64"] else gen.uniform_u32
    keys = gen_fn(sum(c["sizes"]), c["bits"], 51, 0)[lo:lo + n].copy()
    if c["dup"]:
        keys = keys % (5 if c["u64"] else np.uint32(5))
    vals = np.arange(lo, lo + n, dtype=np.uint32)  # the global index
    return keys, vals


def cpu_ops():
    import oracle
    from paper_1708_09495_gb300.dist import LocalOps

    def t(a):  # numpy uint -> torch int view
        return torch.from_numpy(a.view(np.int64 if a.dtype == np.uint64 else np.int32).copy())

    def a(x, u64):
        return x.numpy().view(np.uint64 if u64 else np.uint32)

    def sample(k, m, seed):
        u64 = k.dtype == torch.int64
        kk = a(k, u64)
        return t(kk[oracle.sample_indices(kk.size, m, seed)])

    def sort_keys(k):
        u64 = k.dtype == torch.int64
        return t(oracle.lsd(a(k, u64), None)[0])

    def partition(k, v, smp, p):
        u64 = k.dtype == torch.int64
        ko, vo, c = oracle.partition(a(k, u64), None if v is None else a(v, False), a(smp, u64), p)
        return t(ko), (None if vo is None else t(vo)), torch.from_numpy(c.astype(np.int64))

    def sort_pairs(k, v, key_bits, rb):
        u64 = k.dtype == torch.int64
        ko, vo = oracle.lsd(a(k, u64), None if v is None else a(v, False), key_bits, rb)
        return t(ko), (None if vo is None else t(vo))

    return LocalOps(sample=sample, sort_keys=sort_keys, partition=partition, sort_pairs=sort_pairs)


def _worker(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_1708_09495_gb300 import dist as idist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        keys, vals = make_input(case, rank)
        u64 = keys.dtype == np.uint64
        kt = torch.from_numpy(keys.view(np.int64 if u64 else np.int32).copy())
        vt = torch.from_numpy(vals.view(np.int32).copy())
        rk, rv, sent = idist.sample_sort(kt, vt, key_bits=CASES[case]["bits"], oversample=64, ops=cpu_ops())
        out[rank] = (rk.numpy().view(np.uint64 if u64 else np.uint32).copy(), rv.numpy().view(np.uint32).copy(),
                     sent.numpy().copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_process_sample_sort_matches_oracle(case):
    import oracle

    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), case, out), nprocs=world, start_method="spawn",
                           join=True)
        res = dict(out)
    parts = [make_input(case, r) for r in range(world)]
    keys = np.concatenate([p[0] for p in parts])
    vals = np.concatenate([p[1] for p in parts])
    ek, ev = oracle.lsd(keys, vals, CASES[case]["bits"], 8)
    gk = np.concatenate([res[r][0] for r in range(world)])
    gv = np.concatenate([res[r][1] for r in range(world)])
    assert np.array_equal(gk, ek) and np.array_equal(gv, ev)
    # what each process sent adds up to its part; process r received range r
    for r in range(world):
        assert int(res[r][2].sum()) == parts[r][0].size
    assert sum(int(res[q][2][0]) for q in range(world)) == res[0][0].size
    if res[0][0].size and res[1][0].size:
        assert res[0][0].max() <= res[1][0].min()

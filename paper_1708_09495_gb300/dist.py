"""Sorting keys spread over p processes, one GPU each: the sample sort of
Section 2 (regular choice of splitters from a gathered sample) with one
exchange of keys, Section 3's routing of eq. Tp done once instead of once per
round.

Every process holds a part of the input; after ``sample_sort`` process r holds
the r-th range of the globally sorted sequence, and the concatenation over
r = 0..p-1 is the stable sort of the concatenated input (ties in the order of
(process, position)). Steps, on each process:
  1. draw ``oversample`` keys of its part (isort_sample; seed = base + rank);
  2. gather every process's sample (all-gather) and sort the gathered keys;
  3. route its keys into p ranges by the p - 1 splitters chosen regularly from
     that sorted sample (isort_partition: stable, with per-range counts);
  4. exchange the range sizes, then the keys and payloads (all-to-all-v):
     process r receives range r from every process, in process order;
  5. sort what it received (isort_radix, stable).
Steps 1, 2's sort, 3 and 5 run in the library's kernels; the collectives are
torch.distributed's (NCCL between GPUs, gloo between CPU processes).

The local steps are passed in as ``ops`` so that the exchange logic can be
exercised by CPU processes (tests use gloo and CPU stand-ins for the steps).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable


@dataclass
class LocalOps:
    """The four local steps (tensors on this process's device)."""
    sample: Callable  # (keys, m, seed) -> m sample keys
    sort_keys: Callable  # (keys) -> keys sorted ascending (in place or new)
    partition: Callable  # (keys, vals, sorted_sample, parts) -> (keys_out, vals_out, counts int64)
    sort_pairs: Callable  # (keys, vals, key_bits, radix_bits) -> stable (keys, vals)


def gpu_ops() -> LocalOps:
    """The library's kernels (keys as int32 / int64 tensors of unsigned bit patterns)."""
    import paper_1708_09495_gb300 as isort

    def sort_keys(k):
        isort.radix(k, None)
        return k

    def sort_pairs(k, v, key_bits, radix_bits):
        isort.radix(k, v, key_bits, radix_bits)
        return k, v

    return LocalOps(sample=lambda k, m, seed: isort.sample(k, m, seed), sort_keys=sort_keys,
                    partition=lambda k, v, smp, p: isort.partition(k, v, smp, p), sort_pairs=sort_pairs)


def sample_sort(keys, vals=None, group=None, key_bits: int = 0, radix_bits: int = 8, oversample: int = 256,
                seed: int = 0x5A5A, ops: LocalOps | None = None):
    """Sorts the keys (and payloads) held by the processes of ``group``; returns
    this process's range (keys, vals) and the per-process range sizes it sent."""
    import torch
    import torch.distributed as dist

    ops = ops or gpu_ops()
    p = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = keys.device
    n = keys.numel()
    # 1-2. samples of every process (empty parts contribute none), gathered and sorted
    s = oversample if n > 0 else 0
    mine = ops.sample(keys, s, seed + rank) if s else keys[:0]
    sizes = torch.tensor([s], dtype=torch.int64, device=dev)
    all_sizes = [torch.zeros_like(sizes) for _ in range(p)]
    dist.all_gather(all_sizes, sizes, group=group)
    all_sizes = [int(x.item()) for x in all_sizes]
    if sum(all_sizes) == 0:  # no keys anywhere
        return keys, vals, torch.zeros(p, dtype=torch.int64, device=dev)
    pad = torch.zeros(oversample, dtype=keys.dtype, device=dev)
    pad[:s] = mine
    gathered = [torch.empty_like(pad) for _ in range(p)]
    dist.all_gather(gathered, pad, group=group)
    smp = torch.cat([g[:c] for g, c in zip(gathered, all_sizes)]).contiguous()
    smp = ops.sort_keys(smp)
    # 3. route this process's keys into p ranges
    ko, vo, counts = ops.partition(keys, vals, smp, p)
    # 4. range sizes, then the ranges themselves
    recv_counts = torch.empty_like(counts)
    dist.all_to_all_single(recv_counts, counts, group=group)
    send = counts.tolist()
    recv = recv_counts.tolist()
    rk = torch.empty(int(sum(recv)), dtype=keys.dtype, device=dev)
    dist.all_to_all_single(rk, ko, output_split_sizes=recv, input_split_sizes=send, group=group)
    rv = None
    if vals is not None:
        rv = torch.empty(int(sum(recv)), dtype=vals.dtype, device=dev)
        dist.all_to_all_single(rv, vo, output_split_sizes=recv, input_split_sizes=send, group=group)
    # 5. the received range, in process order, sorted stably
    if rk.numel() > 1:
        rk, rv = ops.sort_pairs(rk, rv, key_bits, radix_bits)
    return rk, rv, counts

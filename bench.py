"""Benchmark: stable LSD radix sort of n = 2^28 uint32 keys (uniform on
[0, 2^32), seed 2) with a uint32 payload (= original index), radix 2^8
(4 count-sort rounds), on one GB300.

One step = one sort through the library's out-of-place call (all kernels of
the path: digit histogram, digit scan, one rank-and-scatter launch per round).
Inputs stay pristine, so every step does identical work; they are 2 GiB, far
larger than the 129 MB L2, so no L2 flush is needed between steps.

Prints ONE JSON line (rank 0). Besides the headline it carries, at one GPU:
  cpu_baseline  the serial C oracle on the host, on the whole workload;
  cpu_parallel  the paper's parallel radix sort on all host cores (and its
                BTN / OET block networks at small n);
  configs       every other configuration -- the small case and the block
                networks, radix 2^11, the known 20-bit key range, the batched
                segmented sort, the learned-bucket sort on three skewed key
                distributions with each model, 64-bit keys, float keys -- each
                with its time, its roofline fraction, plain LSD on the same
                data, and a full check of its output (sorted, stable with
                payload = index, a permutation of the input).
``--workload <name>`` runs one of those configurations alone.
``--impl reference`` times the serial CPU oracle instead, on a bounded sample
of the same workload, on the host cores.
Multi-GPU (torchrun): independent replicas, one per GPU (weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

E2E_SLOTS = 3  # e2e: streams (and host output buffers) in flight
MODELS = {0: "piecewise-linear CDF", 1: "1-32-1 MLP CDF", 2: "regular sampling, no trained model"}
METRIC = "Gkeys/s (u32 n=2^28) & % HBM roofline; learned/batched vs plain LSD, bit-exact"
UNIT = "Gkeys/s"
N = 1 << 28
SEED = 2
RADIX_BITS = 8
KEY_BITS = 32
ROUNDS = 4
WORKLOAD = ("stable LSD radix sort, u32 keys uniform on [0,2^32) (seed 2) + u32 payload = index, "
            "n = 2^28, radix 2^8 (4 rounds), out of place")
# Algorithmic bytes (fixed formula): one key read for the digit counts of all
# rounds, then per round one read and one write of key + payload.
BYTES_PER_KEY = 4 + ROUNDS * 2 * (4 + 4)
ROUND_BYTES_PER_KEY = 2 * (4 + 4)  # one rank-and-scatter launch


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"isort_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # start timing only once the sampler is live (its start-up takes a while)
            t0 = time.time()
            while time.time() - t0 < 3.0 and self.proc.poll() is None:
                self.f.flush()
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            for ln in open(self.path):
                p = [x.strip() for x in ln.split(",")]
                if len(p) >= 9 and p[1].replace(".", "").isdigit():
                    rows.append(p)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


def max_over_ranks(ms: float, dist, device) -> float:
    """The largest per-rank time (replicas: the job ends when the slowest rank does)."""
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, steps: int, n: int, ms_max: float) -> float:
    """Whole-job throughput in Gkeys/s: every rank sorts n keys per step."""
    return world * steps * n / (ms_max * 1e-3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_inputs():
    from gen import workloads

    return workloads.large_uniform(N, 32, SEED, payload=True)


def configure(args):
    """--log2n / --radix-bits select a smaller or differently-digited case of
    the same workload (profiling); the defaults are the benchmark."""
    global N, RADIX_BITS, ROUNDS, BYTES_PER_KEY, WORKLOAD
    N = 1 << args.log2n
    RADIX_BITS = args.radix_bits
    ROUNDS = -(-KEY_BITS // RADIX_BITS)
    BYTES_PER_KEY = 4 + ROUNDS * 2 * (4 + 4)
    WORKLOAD = (f"stable LSD radix sort, u32 keys uniform on [0,2^32) (seed 2) + u32 payload = index, "
                f"n = 2^{args.log2n}, radix 2^{RADIX_BITS} ({ROUNDS} rounds), out of place")


def cpu_baseline_oracle(keys, vals, sample_n: int, reps: int):
    """The serial C oracle (1 core) on the first sample_n keys; Gkeys/s."""
    import oracle

    k, v = keys[:sample_n].copy(), vals[:sample_n].copy()
    oracle.lsd(k[:1024], v[:1024], KEY_BITS, RADIX_BITS)  # load + warm
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.lsd(k, v, KEY_BITS, RADIX_BITS)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    return sample_n / t / 1e9, t, times


def cpu_parallel_baseline(keys, vals, reps: int = 3):
    """The paper's parallel radix sort (and its BTN / OET block networks at
    small n) on all host cores: the multicore baseline, timed on the whole
    workload (median of reps)."""
    import cpu_baseline
    from gen import workloads

    threads = cpu_baseline.hardware_threads()
    times = []
    for _ in range(reps):
        k, v = keys.copy(), vals.copy()
        t0 = time.perf_counter()
        cpu_baseline.pr_sort(k, v, KEY_BITS, RADIX_BITS, threads)
        times.append(time.perf_counter() - t0)
    if not (bool(np.all(k[1:] >= k[:-1])) and bool(np.array_equal(keys[v], k))):
        raise RuntimeError("cpu baseline output is not the stable sort")
    t = statistics.median(times)
    small = workloads.small_uniform()
    net = small[: workloads.SMALL_BTN_N]

    def us(fn, a, reps_small=200):
        best = []
        for _ in range(5):
            t0 = time.perf_counter()
            for _ in range(reps_small):
                x = a.copy()
                fn(x)
            best.append((time.perf_counter() - t0) / reps_small * 1e6)
        return min(best)

    p = 4  # the paper's small-n tables use p = 4 (Tables 3-5)
    return {
        "value": N / t / 1e9, "unit": UNIT, "cores": threads, "kind": "parallel radix sort (Section 3), std::thread",
        "cpu_model": cpu_baseline.cpu_model(), "seconds": t, "runs": times,
        "sample": f"the whole workload (2^{int(round(np.log2(N)))} pairs), median of {reps}",
        "small_us": {f"pr_{small.size}_p{p}": us(lambda x: cpu_baseline.pr_sort(x, None, 32, 8, p), small, 20),
                     f"btn_{net.size}_p{p}": us(lambda x: cpu_baseline.btn(x, None, p), net),
                     f"oet_{net.size}_p{p}": us(lambda x: cpu_baseline.oet(x, None, p), net)},
    }


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    keys, vals = make_inputs()
    sample_n = min(N, 1 << 23)
    import oracle

    k, v = keys[:sample_n].copy(), vals[:sample_n].copy()
    for _ in range(args.warmup):
        oracle.lsd(k, v, KEY_BITS, RADIX_BITS)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.lsd(k, v, KEY_BITS, RADIX_BITS)
    dt = time.perf_counter() - t0
    val = args.steps * sample_n / dt / 1e9
    sample = f"first 2^23 keys (+payload) of the workload per step, serial oracle, {args.steps} steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_n": sample_n, "radix_bits": RADIX_BITS, "key_bits": KEY_BITS},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_1708_09495_gb300 as isort

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = isort.load()
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)

    keys, vals = make_inputs()
    ki = torch.from_numpy(keys.view(np.int32)).cuda()
    vi = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo = torch.empty_like(ki), torch.empty_like(vi)
    args_c = [ctypes.c_void_p(ki.data_ptr()), ctypes.c_void_p(vi.data_ptr()), ctypes.c_void_p(ko.data_ptr()),
              ctypes.c_void_p(vo.data_ptr()), N, KEY_BITS, RADIX_BITS, sp]

    def step():
        rc = lib.isort_radix_copy(*args_c)
        if rc != 0:
            raise RuntimeError(f"isort_radix_copy failed: {isort.STATUS.get(rc, rc)}")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the bench's own output, checked in full (sorted, stable, a permutation of
    # the input pairs)
    head_check = check_pairs(keys, ko.cpu().numpy().view(np.uint32), vo.cpu().numpy().view(np.uint32))
    if not head_check["ok"]:
        raise RuntimeError(f"bench output is not the stable sort: {head_check}")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    isort.profile_read()  # clear
    launches0 = isort.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    isort.profile_enable(True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    isort.profile_enable(False)
    launches = isort.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    prof = isort.profile_read()
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = replica_value(world, args.steps, N, ms_max)

    # dominant kernel: the rank-and-scatter launch of a round (chunked rounds:
    # "downsweep"; single-pass rounds: "onesweep"). Algorithmic bytes per
    # launch: one read and one write of n keys and payloads.
    peak, peak_kind = peaks()
    round_kernel = "downsweep" if "downsweep" in prof else "onesweep"
    rl, rms = prof.get(round_kernel, (0, 0.0))
    avg_round_ms = rms / max(rl, 1)
    achieved = N * ROUND_BYTES_PER_KEY / (avg_round_ms * 1e-3) / 1e9 if rl else None
    # DRAM bytes per launch of that kernel from one ncu capture (a "key: value"
    # text summary under profiles/), when it was taken on this workload
    traffic = None
    tpath = os.path.join(ROOT, "profiles", f"{round_kernel}_traffic.txt")
    if os.path.exists(tpath):
        try:
            t = {}
            with open(tpath) as f:
                for ln in f:
                    if ":" in ln and not ln.startswith("#"):
                        k, v = ln.split(":", 1)
                        t[k.strip()] = v.strip()
            if int(t.get("log2n", -1)) == int(round(np.log2(N))) and int(t.get("radix_bits", -1)) == RADIX_BITS:
                traffic = float(t["bytes_per_launch"])
        except Exception:
            traffic = None
    kernels = {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in prof.items()}

    # end to end: host (pinned) buffers through the same C call, copies included
    e2e = None
    if not args.no_e2e:
        # Every step is one isort_radix_copy from pinned host input buffers to
        # pinned host output buffers (copy in, sort, copy out inside the call).
        # Steps go round-robin over E2E_SLOTS streams with their own output
        # buffers in the asynchronous status mode, so that one step's copy out
        # overlaps the next steps' copies in and sorts; the timed region ends
        # when every step's result is back on the host; device-detected errors
        # are collected after it.
        hk = torch.from_numpy(keys.view(np.int32)).pin_memory()
        hv = torch.from_numpy(vals.view(np.int32)).pin_memory()
        slots = max(1, args.e2e_slots)
        hko = [torch.empty_like(hk).pin_memory() for _ in range(slots)]
        hvo = [torch.empty_like(hv).pin_memory() for _ in range(slots)]
        e2e_streams = [torch.cuda.Stream() for _ in range(slots)]

        def e2e_step(i):
            j = i % slots
            rc = lib.isort_radix_copy(ctypes.c_void_p(hk.data_ptr()), ctypes.c_void_p(hv.data_ptr()),
                                      ctypes.c_void_p(hko[j].data_ptr()), ctypes.c_void_p(hvo[j].data_ptr()), N,
                                      KEY_BITS, RADIX_BITS, ctypes.c_void_p(e2e_streams[j].cuda_stream))
            if rc != 0:
                raise RuntimeError(f"e2e failed: {isort.STATUS.get(rc, rc)}")

        lib.isort_set_sync(0)
        try:
            for i in range(slots):
                e2e_step(i)
            torch.cuda.synchronize()
            e2e_steps = max(slots, min(args.steps, 3 * slots))
            barrier()
            t0 = time.perf_counter()
            for i in range(e2e_steps):
                e2e_step(i)
            torch.cuda.synchronize()
            barrier()
            dt = time.perf_counter() - t0
        finally:
            lib.isort_set_sync(1)
        rc = lib.isort_device_status(1, None)
        if rc != 0:
            raise RuntimeError(f"e2e device status: {isort.STATUS.get(rc, rc)}")
        last = (e2e_steps - 1) % slots
        e2e_check = check_pairs(keys, hko[last].numpy().view(np.uint32), hvo[last].numpy().view(np.uint32))
        if not e2e_check["ok"]:
            raise RuntimeError(f"e2e output is not the stable sort: {e2e_check}")
        del hk, hv, hko, hvo
        e2e = {"value": world * e2e_steps * N / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": N * 8,
               "d2h_bytes_per_step": N * 8, "steps": e2e_steps,
               "how": f"isort_radix_copy host->host, {slots} streams in flight (asynchronous status mode)"}

    cpu = cpu_par = configs = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample_n = min(N, args.cpu_sample)
        v, t, times = cpu_baseline_oracle(keys, vals, sample_n, 3)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {sample_n} keys (+payload) of the workload, serial C oracle, median of 3 runs",
               "seconds": t}
        cpu_par = cpu_parallel_baseline(keys, vals)
    if rank == 0 and world == 1 and not args.no_configs:
        del ki, vi, ko, vo
        torch.cuda.empty_cache()
        configs = run_configs(min(args.steps, 5), args.warmup)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "key_bits": KEY_BITS, "radix_bits": RADIX_BITS,
                       "payload": "u32 index", "l2": "inputs (2 GiB) larger than L2; no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "kernel": f"{round_kernel} (rank and scatter of one count-sort round)",
                         "peak_kind": peak_kind,
                         "whole_sort_frac": N * BYTES_PER_KEY / (ms_max / args.steps * 1e-3) / 1e9 / peak},
            "cpu_baseline": cpu,
            "cpu_parallel": cpu_par,
            "e2e": e2e,
            "output_check": head_check,
            "gpu_launches": launches,
            "kernels": kernels,
            "clocks": clk.summary(),
            "configs": configs,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _timed_inplace(call, reset, steps, warmup, stream):
    """Runs reset() then call() per step; times call() alone with CUDA events
    on the stream; returns the total milliseconds over the timed steps."""
    import torch

    for _ in range(warmup):
        if reset:
            reset()
        call()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        if reset:
            reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total


# ---------------------------------------------------------------------------
# Output checks of the configs (numpy, on the host; O(n) each)

def _mix64(x):
    """A bijective 64-bit finaliser (SplitMix64's), elementwise on uint64."""
    x = x ^ (x >> np.uint64(30))
    x = x * np.uint64(0xBF58476D1CE4E5B9)
    x = x ^ (x >> np.uint64(27))
    x = x * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def _multiset_hash(keys, chunk=1 << 24):
    """Commutative hash of a key multiset: sum of mixed keys mod 2^64."""
    h = np.uint64(0)
    with np.errstate(over="ignore"):
        for i in range(0, keys.size, chunk):
            h = h + _mix64(keys[i:i + chunk].astype(np.uint64)).sum(dtype=np.uint64)
    return int(h)


def check_keys(in_k, out_k):
    """Keys only: non-decreasing and the same multiset as the input."""
    srt = bool(np.all(out_k[1:] >= out_k[:-1]))
    same = _multiset_hash(in_k) == _multiset_hash(out_k)
    return {"ok": srt and same, "non_decreasing": srt, "multiset_hash_equal": same}


def check_pairs(in_k, out_k, out_v, seg_id=None):
    """Payload = original index: non-decreasing keys (within segments when
    seg_id is given), every key equal to the input key its payload names,
    payloads a permutation, and stable (payloads increase within equal keys)."""
    n = in_k.size
    pv = out_v.astype(np.int64)
    perm_ok = bool(pv.size == n and np.all(pv < n))
    if perm_ok:
        mark = np.zeros(n, dtype=bool)
        mark[pv] = True
        perm_ok = bool(mark.all())
        del mark
    gather = perm_ok and bool(np.array_equal(in_k[pv], out_k))
    same_seg = True
    if seg_id is not None and perm_ok:
        same_seg = bool(np.array_equal(seg_id[pv], seg_id))
    if seg_id is None:
        srt = bool(np.all(out_k[1:] >= out_k[:-1]))
        eq = out_k[1:] == out_k[:-1]
    else:
        cont = seg_id[1:] == seg_id[:-1]
        srt = bool(np.all((out_k[1:] >= out_k[:-1]) | ~cont))
        eq = (out_k[1:] == out_k[:-1]) & cont
    stable = bool(np.all(out_v[1:][eq] > out_v[:-1][eq]))
    ok = srt and gather and perm_ok and stable and same_seg
    return {"ok": ok, "non_decreasing": srt, "payload_permutation": perm_ok, "keys_match_payload": gather,
            "stable": stable, **({"within_segments": same_seg} if seg_id is not None else {})}


# ---------------------------------------------------------------------------
# The configurations besides the headline, each against plain LSD on the same
# data. Algorithmic bytes per key as the measurement plan fixes them: one key
# read for the counts + per pass one read and one write of keys (+ payloads);
# segmented 16 (one on-chip pass); learned u32 20; learned u64 + payload 56.

def _entry(ms, n, bytes_per_key, peak, **extra):
    e = {"ms_per_call": ms, "gkeys_per_s": n / (ms * 1e-3) / 1e9}
    if bytes_per_key:
        e["roofline"] = {"bytes_per_key": bytes_per_key, "achieved_gbs": n * bytes_per_key / (ms * 1e-3) / 1e9,
                         "frac": n * bytes_per_key / (ms * 1e-3) / 1e9 / peak}
    e.update(extra)
    return e


TUNE_CACHE = None  # --tune-cache: the autotuner's cache file for the segmented configuration


class _Ctx:
    def __init__(self, steps, warmup):
        import torch

        import paper_1708_09495_gb300 as isort

        self.isort = isort
        self.lib = isort.load()
        self.stream = torch.cuda.current_stream()
        self.sp = ctypes.c_void_p(self.stream.cuda_stream)
        self.peak, self.peak_kind = peaks()
        self.steps, self.warmup = steps, warmup

    def ok(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what}: {self.isort.STATUS.get(rc, rc)}")

    def time(self, call, reset=None):
        return _timed_inplace(call, reset, self.steps, self.warmup, self.stream) / self.steps


def _dev(a):
    import torch

    return torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int64)).cuda()


def _host(t, dt):
    return t.cpu().numpy().view(dt)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def cfg_small(c):
    """65,536 u32 keys (seed 1), keys only, radix 2^8; BTN and OET on the
    first 1,024 keys: microseconds per call (launch-bound)."""
    import torch
    from gen import workloads

    keys = workloads.small_uniform()
    net = keys[: workloads.SMALL_BTN_N].copy()
    kin, kout = _dev(keys), torch.empty(keys.size, dtype=torch.int32, device="cuda")
    nin, nw = _dev(net), torch.empty(net.size, dtype=torch.int32, device="cuda")
    steps = max(50, c.steps)
    lsd = lambda: c.ok(c.lib.isort_radix_copy(_vp(kin), None, _vp(kout), None, keys.size, 32, 8, c.sp), "radix")
    btn = lambda: c.ok(c.lib.isort_btn(_vp(nw), None, net.size, c.sp), "btn")
    oet = lambda: c.ok(c.lib.isort_oet(_vp(nw), None, net.size, c.sp), "oet")
    reset = lambda: nw.copy_(nin)
    us = {}
    for name, call, rs in (("lsd_65536", lsd, None), ("btn_1024", btn, reset), ("oet_1024", oet, reset)):
        us[name] = _timed_inplace(call, rs, steps, c.warmup, c.stream) / steps * 1e3
        out = _host(kout if name.startswith("lsd") else nw, np.uint32)
        ref = np.sort(keys if name.startswith("lsd") else net)
        us[name + "_ok"] = bool(np.array_equal(out, ref))
    return {"us_per_call": us, "ok": all(v for k, v in us.items() if k.endswith("_ok")),
            "workload": "65,536 u32 keys uniform (seed 1), keys only, radix 2^8; BTN and OET on the first 1,024"}


def cfg_radix(c, keys, vals, key_bits, rb, plain_bits=32, plain_rb=8, label=""):
    """Out-of-place LSD of u32 pairs at (key_bits, rb) against the full-width
    radix-2^8 sort of the same data."""
    import torch

    n = keys.size
    kin, vin = _dev(keys), _dev(vals)
    ko, vo = torch.empty_like(kin), torch.empty_like(vin)

    def run(kb, r):
        return lambda: c.ok(c.lib.isort_radix_copy(_vp(kin), _vp(vin), _vp(ko), _vp(vo), n, kb, r, c.sp), "radix")

    ms = c.time(run(key_bits, rb))
    chk = check_pairs(keys, _host(ko, np.uint32), _host(vo, np.uint32))
    ms_p = c.time(run(plain_bits, plain_rb))
    rounds = -(-key_bits // rb)
    del kin, vin, ko, vo
    return _entry(ms, n, 4 + rounds * 16, c.peak, rounds=rounds, check=chk, ok=chk["ok"], workload=label,
                  plain_lsd={"ms_per_call": ms_p, "call": f"isort_radix_copy, {plain_bits} key bits, radix 2^{plain_rb}"},
                  speedup_vs_plain=ms_p / ms)


def cfg_segmented(c):
    """The batched segmented sort of the log-uniform-length batch against one
    plain LSD of composite u64 keys (segment id << 32 | key)."""
    import torch
    from gen import workloads

    keys, vals, off = workloads.segmented()
    n, nseg = int(off[-1]), off.size - 1
    kin, vin, doff = _dev(keys), _dev(vals), _dev(off)
    kw, vw = torch.empty_like(kin), torch.empty_like(vin)
    seg_id = np.repeat(np.arange(nseg, dtype=np.uint32), np.diff(off).astype(np.int64))
    comp = (seg_id.astype(np.uint64) << np.uint64(32)) | keys.astype(np.uint64)
    cin = _dev(comp)
    cw = torch.empty_like(cin)
    cbits = 32 + int(nseg - 1).bit_length()

    def reset_s():
        kw.copy_(kin)
        vw.copy_(vin)

    def reset_c():
        cw.copy_(cin)
        vw.copy_(vin)

    seg = lambda: c.ok(c.lib.isort_segmented(_vp(kw), _vp(vw), _vp(doff), nseg, 32, c.sp), "segmented")
    cmp_ = lambda: c.ok(c.lib.isort_radix_u64(_vp(cw), _vp(vw), n, cbits, 8, c.sp), "radix_u64")
    # the router's cut-offs measured on this GPU (untimed), then the timed runs
    import tempfile

    # a given cache file keeps the cut-offs of an earlier run (e.g. a profiled
    # run takes those of the plain run before it); else a fresh one is measured
    tune_path = TUNE_CACHE or os.path.join(tempfile.mkdtemp(prefix="isort_tune_"), "cache.txt")
    c.isort.autotune(True, tune_path)
    try:
        reset_s()
        seg()
        router = [ln.split()[1:] for ln in open(tune_path) if ln.startswith("router")]
        c.isort.profile_read()
        c.isort.profile_enable(True)
        ms = c.time(seg, reset_s)
        c.isort.profile_enable(False)
        prof = c.isort.profile_read()
    finally:
        c.isort.autotune(False)
    chk = check_pairs(keys, _host(kw, np.uint32), _host(vw, np.uint32), seg_id)
    ms_p = c.time(cmp_, reset_c)
    del kin, vin, doff, kw, vw, cin, cw
    return _entry(ms, n, 16, c.peak, check=chk, ok=chk["ok"], segments=nseg,
                  workload=f"{nseg} segments of log-uniform length in [2, 65536], {n} u32 keys + u32 payload (seed 4)",
                  plain_lsd={"ms_per_call": ms_p, "call": f"isort_radix_u64 on (segment id << 32 | key), "
                                                          f"{cbits} key bits, radix 2^8"},
                  speedup_vs_plain=ms_p / ms,
                  router_cutoffs={"payload" if r[0] == "1" else "keys_only":
                                  {"oet_max": int(r[1]), "btn_warp_max": int(r[2]), "btn_cta_max": int(r[3])}
                                  for r in router},
                  kernels={k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in prof.items()})


def cfg_learned(c, dist, models=(0, 1, 2), n=1 << 28):
    """Keys-only skewed u32 keys: the learned-bucket sort with each model
    against the plain radix-2^8 rounds on the same keys."""
    import torch
    from gen import workloads

    keys = workloads.skewed(dist, n)
    kin = _dev(keys)
    kw = torch.empty_like(kin)
    reset = lambda: kw.copy_(kin)
    ms_p = c.time(lambda: c.ok(c.lib.isort_radix(_vp(kw), None, n, 32, 8, c.sp), "radix"), reset)
    out = {"workload": f"{dist} u32 keys, keys only, n = 2^{int(round(np.log2(n)))} (seed 6)",
           "plain_lsd": {"ms_per_call": ms_p, "gkeys_per_s": n / (ms_p * 1e-3) / 1e9,
                         "call": "isort_radix, radix 2^8, 4 rounds, in place"}, "models": {}}
    ok_all = True
    for m in models:
        st = c.isort.LearnedStats()
        call = lambda: c.ok(c.lib.isort_learned(_vp(kw), None, n, 32, 0, m, ctypes.byref(st), c.sp), "learned")
        ms = c.time(call, reset)
        chk = check_keys(keys, _host(kw, np.uint32))
        ok_all = ok_all and chk["ok"]
        s = st.as_dict()
        out["models"][MODELS[m]] = _entry(ms, n, 20, c.peak, speedup_vs_plain=ms_p / ms, check=chk, ok=chk["ok"],
                                          imbalance_max_over_mean=s["imbalance_max_over_mean"],
                                          overflow_fraction=s["overflow_fraction"],
                                          fell_back_to_lsd=bool(s["fell_back_to_lsd"]), nbuckets=s["nbuckets"],
                                          train_loss_initial=s["train_loss_initial"], train_loss=s["train_loss"])
    out["ok"] = ok_all
    del kin, kw
    return out


def cfg_learned64(c, bits, model=0):
    """2^27 u64 keys + u32 payload: the learned first pass with on-chip finish
    against the plain radix-2^8 rounds (8 or 6 of them)."""
    import torch
    from gen import workloads

    keys, vals = workloads.wide_u64(bits=bits)
    n = keys.size
    kin, vin = _dev(keys), _dev(vals)
    kw, vw = torch.empty_like(kin), torch.empty_like(vin)

    def reset():
        kw.copy_(kin)
        vw.copy_(vin)

    st = c.isort.LearnedStats()
    learned = lambda: c.ok(c.lib.isort_learned_u64(_vp(kw), _vp(vw), n, bits, 0, model, ctypes.byref(st), c.sp),
                           "learned_u64")
    plain = lambda: c.ok(c.lib.isort_radix_u64(_vp(kw), _vp(vw), n, bits, 8, c.sp), "radix_u64")
    ms = c.time(learned, reset)
    chk = check_pairs(keys, _host(kw, np.uint64), _host(vw, np.uint32))
    ms_p = c.time(plain, reset)
    rounds = -(-bits // 8)
    s = st.as_dict()
    del kin, vin, kw, vw
    return _entry(ms, n, 56, c.peak, check=chk, ok=chk["ok"], model=MODELS[model],
                  workload=f"u64 keys uniform on [0, 2^{bits}) + u32 payload = index, n = 2^27 (seed 5)",
                  plain_lsd={"ms_per_call": ms_p, "gkeys_per_s": n / (ms_p * 1e-3) / 1e9,
                             "call": f"isort_radix_u64, radix 2^8, {rounds} rounds, in place",
                             "roofline_frac": n * (8 + rounds * 24) / (ms_p * 1e-3) / 1e9 / c.peak},
                  speedup_vs_plain=ms_p / ms, imbalance_max_over_mean=s["imbalance_max_over_mean"],
                  overflow_fraction=s["overflow_fraction"], fell_back_to_lsd=bool(s["fell_back_to_lsd"]),
                  nbuckets=s["nbuckets"])


def cfg_typed(c, n=1 << 28):
    """float32 keys + payload in IEEE totalOrder (through the order-preserving
    bit map around the radix-2^8 rounds) against the same bits sorted as u32."""
    import torch

    r = np.random.default_rng(7)
    keys = (r.standard_normal(n, dtype=np.float32) * np.float32(1e3)).astype(np.float32)
    keys[::1021] = -0.0
    bits = keys.view(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    kin, vin = _dev(bits), _dev(vals)
    kw, vw = torch.empty_like(kin), torch.empty_like(vin)

    def reset():
        kw.copy_(kin)
        vw.copy_(vin)

    typed = lambda: c.ok(c.lib.isort_radix_typed(_vp(kw), 2, _vp(vw), n, 8, c.sp), "radix_typed")
    plain = lambda: c.ok(c.lib.isort_radix(_vp(kw), _vp(vw), n, 32, 8, c.sp), "radix")
    ms = c.time(typed, reset)
    # totalOrder on floats without NaNs: the bit map's order is the float order
    # with -0.0 before +0.0; check it on the mapped keys
    ok_bits = _host(kw, np.uint32)
    mapped_in = np.where(bits >> np.uint32(31), ~bits, bits | np.uint32(0x80000000)).astype(np.uint32)
    mapped_out = np.where(ok_bits >> np.uint32(31), ~ok_bits, ok_bits | np.uint32(0x80000000)).astype(np.uint32)
    chk = check_pairs(mapped_in, mapped_out, _host(vw, np.uint32))
    ms_p = c.time(plain, reset)
    del kin, vin, kw, vw
    return _entry(ms, n, 4 + 4 * 16 + 16, c.peak, check=chk, ok=chk["ok"],
                  workload="2^28 float32 keys normal(0, 1e3) with -0.0 (seed 7) + u32 payload, IEEE totalOrder, "
                           "radix 2^8 (bytes: the rounds plus the two bit-map passes)",
                  plain_lsd={"ms_per_call": ms_p, "call": "isort_radix on the same bits as u32 keys, radix 2^8"},
                  speedup_vs_plain=ms_p / ms)


def run_configs(steps=5, warmup=3, only=None):
    """Every configuration besides the headline, keyed by name."""
    import torch
    from gen import workloads

    c = _Ctx(steps, warmup)
    todo = {
        "1_small": lambda: cfg_small(c),
        "2b_radix11": lambda: cfg_radix(c, *workloads.large_uniform(1 << 28, 32, 2, payload=True), 32, 11,
                                        label="2^28 u32 uniform (seed 2) + payload, radix 2^11 (3 rounds)"),
        "2c_range20_radix8": lambda: cfg_radix(c, *workloads.large_range20(), 20, 8,
                                               label="2^28 u32 on [0, 2^20) (seed 3) + payload, key_bits 20, "
                                                     "radix 2^8 (3 rounds); plain: 32 key bits"),
        "2c_range20_radix11": lambda: cfg_radix(c, *workloads.large_range20(), 20, 11,
                                                label="2^28 u32 on [0, 2^20) (seed 3) + payload, key_bits 20, "
                                                      "radix 2^11 (2 rounds); plain: 32 key bits, radix 2^8"),
        "3_segmented": lambda: cfg_segmented(c),
        "4_learned_zipf": lambda: cfg_learned(c, "zipf"),
        "4_learned_lognormal": lambda: cfg_learned(c, "lognormal"),
        "4_learned_gmm": lambda: cfg_learned(c, "gmm"),
        "5_u64_range64": lambda: cfg_learned64(c, 64),
        "5_u64_range48": lambda: cfg_learned64(c, 48),
        "f2_typed_f32": lambda: cfg_typed(c),
    }
    out = {}
    for name, fn in todo.items():
        if only and name not in only:
            continue
        t0 = time.time()
        try:
            out[name] = fn()
        except Exception as e:  # reported, not hidden: the entry says what failed
            out[name] = {"ok": False, "error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = round(time.time() - t0, 1)
        torch.cuda.empty_cache()
    return out


def run_compare(args):
    """One configuration on its own (one JSON line)."""
    names = {"small": "1_small", "segmented": "3_segmented", "radix11": "2b_radix11",
             "range20": "2c_range20_radix8", "learned": f"4_learned_{args.dist}",
             "learned64": "5_u64_range48" if args.dist == "range48" else "5_u64_range64", "typed": "f2_typed_f32"}
    name = names[args.workload]
    res = run_configs(args.steps, args.warmup, only={name})[name]
    print(json.dumps({"metric": METRIC, "unit": UNIT, "n_gpus": 1, "config_name": name, **res}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-slots", type=int, default=E2E_SLOTS, help="e2e: calls (streams) in flight")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1 << 28, help="keys the serial oracle sorts per timed run")
    ap.add_argument("--no-configs", action="store_true", help="only the headline (skip the other configurations)")
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--radix-bits", type=int, default=8)
    ap.add_argument("--workload", default="uniform",
                    choices=["uniform", "learned", "learned64", "segmented", "small", "radix11", "range20", "typed"],
                    help="uniform: the benchmark (with every other configuration under 'configs'); the others: "
                         "one of those configurations alone, as its own JSON line")
    ap.add_argument("--tune-cache", default=None,
                    help="segmented: autotuner cache file (router cut-offs read from it if present, else measured "
                         "and written to it)")
    ap.add_argument("--dist", default="lognormal", choices=["zipf", "lognormal", "gmm", "range48"],
                    help="learned: key distribution; learned64: range48 for keys on [0, 2^48)")
    args = ap.parse_args()
    global TUNE_CACHE
    TUNE_CACHE = args.tune_cache
    configure(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "uniform":
        return run_compare(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

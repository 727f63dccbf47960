"""Benchmark: stable LSD radix sort of n = 2^28 uint32 keys (uniform on
[0, 2^32), seed 2) with a uint32 payload (= original index), radix 2^8
(4 count-sort rounds), on one GB300.

One step = one sort through the library's out-of-place call (all kernels of
the path: digit histogram, digit scan, one rank-and-scatter launch per round).
Inputs stay pristine, so every step does identical work; they are 2 GiB, far
larger than the 129 MB L2, so no L2 flush is needed between steps.

Prints ONE JSON line (rank 0). ``--impl reference`` times the serial CPU oracle
instead, on a bounded sample of the same workload, on the host cores.
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
    # correctness spot check of the bench's own output (sorted + stable)
    sk = ko[:: max(1, N // 4096)].cpu().numpy().view(np.uint32)
    if not np.all(sk[1:] >= sk[:-1]):
        raise RuntimeError("bench output not sorted")

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
        ko = hko[last].numpy().view(np.uint32)
        if not bool(np.all(ko[1:] >= ko[:-1])):
            raise RuntimeError("e2e output not sorted")
        e2e = {"value": world * e2e_steps * N / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": N * 8,
               "d2h_bytes_per_step": N * 8, "steps": e2e_steps,
               "how": f"isort_radix_copy host->host, {slots} streams in flight (asynchronous status mode)"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, t, times = cpu_baseline_oracle(keys, vals, min(N, 1 << 24), 3)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "first 2^24 keys (+payload) of the workload, serial C oracle, median of 3 runs"}

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
            "e2e": e2e,
            "gpu_launches": launches,
            "kernels": kernels,
            "clocks": clk.summary(),
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
        reset()
        call()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total


def run_compare(args):
    """Secondary workloads, each against plain LSD on the same data (one GPU):
    learned: keys-only skewed u32 (n = 2^log2n), learned-bucket sort vs the
             plain radix rounds;
    segmented: the log-uniform-length segment batch (2^28 keys, payload),
             batched segmented sort vs one plain LSD of composite u64 keys
             (segment id << 32 | key).
    typed: 2^log2n float32 keys + payload in IEEE totalOrder vs the same bits
             sorted as u32 keys.
    Inputs are restored from a pristine copy before every step (not timed)."""
    import numpy as np
    import torch

    import paper_1708_09495_gb300 as isort
    from gen import workloads

    lib = isort.load()
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    peak, peak_kind = peaks()
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "u32", "data": "synthetic"}
    if args.workload == "small":
        # the small case: LSD on 65,536 keys (keys only, radix 2^8), BTN and OET
        # on its first 1,024 keys; launch-bound, reported in microseconds per call
        keys = workloads.small_uniform()
        n = keys.size
        kin = torch.from_numpy(keys.view(np.int32)).cuda()
        kout = torch.empty_like(kin)
        small = torch.from_numpy(keys[: workloads.SMALL_BTN_N].copy().view(np.int32)).cuda()
        sw = torch.empty_like(small)
        iters = max(50, args.steps)

        def timed(call, reset=None):
            for _ in range(args.warmup):
                if reset:
                    reset()
                call()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tot = 0.0
            for _ in range(iters):
                if reset:
                    reset()
                e0.record(stream)
                call()
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            return tot / iters * 1e3  # microseconds per call

        def lsd():
            rc = lib.isort_radix_copy(ctypes.c_void_p(kin.data_ptr()), None, ctypes.c_void_p(kout.data_ptr()), None,
                                      n, 32, 8, sp)
            if rc != 0:
                raise RuntimeError(f"isort_radix_copy: {isort.STATUS.get(rc, rc)}")

        def net(fn):
            def call():
                rc = fn(ctypes.c_void_p(sw.data_ptr()), None, sw.numel(), sp)
                if rc != 0:
                    raise RuntimeError(f"network sort: {isort.STATUS.get(rc, rc)}")
            return call

        us_lsd = timed(lsd)
        us_btn = timed(net(lib.isort_btn), lambda: sw.copy_(small))
        us_oet = timed(net(lib.isort_oet), lambda: sw.copy_(small))
        line.update({
            "value": n / (us_lsd * 1e-6) / 1e9, "ms_per_step": us_lsd * 1e-3,
            "config": {"workload": "65,536 u32 keys uniform (seed 1), keys only, radix 2^8, out of place; "
                                   "BTN and OET on the first 1,024 keys", "iters": iters},
            "us_per_call": {"lsd_65536": us_lsd, "btn_1024": us_btn, "oet_1024": us_oet},
            "note": "launch-bound sizes: microseconds per call, not a roofline",
        })
    elif args.workload == "learned64":
        # 2^27 u64 keys uniform on [0, 2^64) (or [0, 2^48)) with payload = index:
        # the learned first pass and on-chip finish against the plain rounds
        bits = 48 if args.dist == "range48" else 64
        keys, vals = workloads.wide_u64(bits=bits)
        n = keys.size
        kin = torch.from_numpy(keys.view(np.int64)).cuda()
        vin = torch.from_numpy(vals.view(np.int32)).cuda()
        kw, vw = torch.empty_like(kin), torch.empty_like(vin)
        st = isort.LearnedStats()

        def learned():
            rc = lib.isort_learned_u64(ctypes.c_void_p(kw.data_ptr()), ctypes.c_void_p(vw.data_ptr()), n, bits,
                                       args.nbuckets, args.model, ctypes.byref(st), sp)
            if rc != 0:
                raise RuntimeError(f"isort_learned_u64: {isort.STATUS.get(rc, rc)}")

        def plain():
            rc = lib.isort_radix_u64(ctypes.c_void_p(kw.data_ptr()), ctypes.c_void_p(vw.data_ptr()), n, bits, 8, sp)
            if rc != 0:
                raise RuntimeError(f"isort_radix_u64: {isort.STATUS.get(rc, rc)}")

        def reset():
            kw.copy_(kin)
            vw.copy_(vin)

        isort.profile_read()
        isort.profile_enable(True)
        ms_l = _timed_inplace(learned, reset, args.steps, args.warmup, stream)
        isort.profile_enable(False)
        prof = isort.profile_read()
        sk = kw[:: max(1, n // 4096)].cpu().numpy().view(np.uint64)
        if not np.all(sk[1:] >= sk[:-1]):
            raise RuntimeError("learned output not sorted")
        ms_p = _timed_inplace(plain, reset, args.steps, args.warmup, stream)
        line.update({
            "value": args.steps * n / (ms_l * 1e-3) / 1e9, "ms_per_step": ms_l / args.steps, "dtype": "u64",
            "config": {"workload": f"learned-bucket sort ({MODELS[args.model]}), u64 keys uniform on [0,2^{bits}) "
                                   f"(seed 5) + u32 payload = index, n = 2^27", "l2": "inputs larger than L2; restored before each step "
                                                               "(untimed)"},
            "plain_lsd": {"value": args.steps * n / (ms_p * 1e-3) / 1e9, "ms_per_step": ms_p / args.steps,
                          "call": f"isort_radix_u64, radix 2^8, {bits // 8} rounds, in place"},
            "speedup_vs_plain": ms_p / ms_l,
            "learned_stats": st.as_dict(),
            "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in prof.items()},
        })
    elif args.workload == "typed":
        # 2^log2n float32 keys (normal, every magnitude and sign, with -0.0) + u32 payload = index, sorted in
        # IEEE totalOrder, against the same bits sorted as u32 keys by the plain rounds
        n = 1 << args.log2n
        r = np.random.default_rng(7)
        keys = (r.standard_normal(n, dtype=np.float32) * np.float32(1e3)).astype(np.float32)
        keys[::1021] = -0.0
        vals = np.arange(n, dtype=np.uint32)
        kin = torch.from_numpy(keys.view(np.int32)).cuda()
        vin = torch.from_numpy(vals.view(np.int32)).cuda()
        kw, vw = torch.empty_like(kin), torch.empty_like(vin)

        def typed():
            rc = lib.isort_radix_typed(ctypes.c_void_p(kw.data_ptr()), 2, ctypes.c_void_p(vw.data_ptr()), n,
                                       args.radix_bits, sp)
            if rc != 0:
                raise RuntimeError(f"isort_radix_typed: {isort.STATUS.get(rc, rc)}")

        def plain():
            rc = lib.isort_radix(ctypes.c_void_p(kw.data_ptr()), ctypes.c_void_p(vw.data_ptr()), n, 32,
                                 args.radix_bits, sp)
            if rc != 0:
                raise RuntimeError(f"isort_radix: {isort.STATUS.get(rc, rc)}")

        def reset():
            kw.copy_(kin)
            vw.copy_(vin)

        isort.profile_read()
        isort.profile_enable(True)
        ms_t = _timed_inplace(typed, reset, args.steps, args.warmup, stream)
        isort.profile_enable(False)
        prof = isort.profile_read()
        sk = kw.view(torch.float32)[:: max(1, n // 65536)].cpu().numpy()
        if not np.all(sk[1:] >= sk[:-1]):
            raise RuntimeError("typed output not sorted")
        ms_p = _timed_inplace(plain, reset, args.steps, args.warmup, stream)
        line.update({
            "value": args.steps * n / (ms_t * 1e-3) / 1e9, "ms_per_step": ms_t / args.steps, "dtype": "f32",
            "config": {"workload": f"typed keys: float32 normal(0, 1e3) with -0.0 (seed 7) + u32 payload = index, "
                                   f"IEEE totalOrder, n = 2^{args.log2n}, radix 2^{args.radix_bits}",
                       "l2": "inputs larger than L2; restored before each step (untimed)"},
            "plain_lsd": {"value": args.steps * n / (ms_p * 1e-3) / 1e9, "ms_per_step": ms_p / args.steps,
                          "call": f"isort_radix on the same bits as u32 keys, radix 2^{args.radix_bits}"},
            "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in prof.items()},
        })
    elif args.workload == "learned":
        n = 1 << args.log2n
        keys = workloads.skewed(args.dist, n)
        kin = torch.from_numpy(keys.view(np.int32)).cuda()
        kw = torch.empty_like(kin)
        st = isort.LearnedStats()

        def learned():
            rc = lib.isort_learned(ctypes.c_void_p(kw.data_ptr()), None, n, 32, args.nbuckets, args.model,
                                   ctypes.byref(st), sp)
            if rc != 0:
                raise RuntimeError(f"isort_learned: {isort.STATUS.get(rc, rc)}")

        def plain():
            rc = lib.isort_radix(ctypes.c_void_p(kw.data_ptr()), None, n, 32, 8, sp)
            if rc != 0:
                raise RuntimeError(f"isort_radix: {isort.STATUS.get(rc, rc)}")

        reset = lambda: kw.copy_(kin)
        isort.profile_read()
        isort.profile_enable(True)
        ms_l = _timed_inplace(learned, reset, args.steps, args.warmup, stream)
        isort.profile_enable(False)
        prof = isort.profile_read()
        sk = kw[:: max(1, n // 4096)].cpu().numpy().view(np.uint32)
        if not np.all(sk[1:] >= sk[:-1]):
            raise RuntimeError("learned output not sorted")
        ms_p = _timed_inplace(plain, reset, args.steps, args.warmup, stream)
        stats = st.as_dict()
        value = args.steps * n / (ms_l * 1e-3) / 1e9
        sw = prof.get("bucket_sweep", (0, 0.0))
        achieved = n * 8 / (sw[1] / sw[0] * 1e-3) / 1e9 if sw[0] else None
        line.update({
            "value": value, "ms_per_step": ms_l / args.steps,
            "config": {"workload": f"learned-bucket sort ({MODELS[args.model]}), u32 keys-only, {args.dist} (seed 6), "
                                   f"n = 2^{args.log2n}",
                       "l2": "inputs larger than L2; restored before each step (untimed)"},
            "plain_lsd": {"value": args.steps * n / (ms_p * 1e-3) / 1e9, "ms_per_step": ms_p / args.steps,
                          "call": "isort_radix, radix 2^8, in place"},
            "speedup_vs_plain": ms_p / ms_l,
            "learned_stats": stats,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None, "traffic": None,
                         "kernel": "bucket_sweep (one stable distribution pass, 8 B/key)", "peak_kind": peak_kind},
            "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in prof.items()},
        })
    else:
        keys, vals, off = workloads.segmented()
        n = int(off[-1])
        nseg = off.size - 1
        kin = torch.from_numpy(keys.view(np.int32)).cuda()
        vin = torch.from_numpy(vals.view(np.int32)).cuda()
        doff = torch.from_numpy(off.view(np.int64)).cuda()
        kw, vw = torch.empty_like(kin), torch.empty_like(vin)
        seg_id = np.repeat(np.arange(nseg, dtype=np.uint64), np.diff(off).astype(np.int64))
        comp = (seg_id << np.uint64(32)) | keys.astype(np.uint64)
        cin = torch.from_numpy(comp.view(np.int64)).cuda()
        cw = torch.empty_like(cin)
        cbits = 32 + int(nseg - 1).bit_length()

        def segmented():
            rc = lib.isort_segmented(ctypes.c_void_p(kw.data_ptr()), ctypes.c_void_p(vw.data_ptr()),
                                     ctypes.c_void_p(doff.data_ptr()), nseg, 32, sp)
            if rc != 0:
                raise RuntimeError(f"isort_segmented: {isort.STATUS.get(rc, rc)}")

        def composite():
            rc = lib.isort_radix_u64(ctypes.c_void_p(cw.data_ptr()), ctypes.c_void_p(vw.data_ptr()), n, cbits, 8,
                                     sp)
            if rc != 0:
                raise RuntimeError(f"isort_radix_u64: {isort.STATUS.get(rc, rc)}")

        def reset_s():
            kw.copy_(kin)
            vw.copy_(vin)

        def reset_c():
            cw.copy_(cin)
            vw.copy_(vin)

        isort.profile_read()
        isort.profile_enable(True)
        ms_s = _timed_inplace(segmented, reset_s, args.steps, args.warmup, stream)
        isort.profile_enable(False)
        prof = isort.profile_read()
        ms_c = _timed_inplace(composite, reset_c, args.steps, args.warmup, stream)
        value = args.steps * n / (ms_s * 1e-3) / 1e9
        line.update({
            "value": value, "ms_per_step": ms_s / args.steps,
            "config": {"workload": f"batched segmented sort, {nseg} segments of log-uniform length in [2, 65536], "
                                   f"n = {n} u32 keys + u32 payload (seed 4)",
                       "l2": "inputs larger than L2; restored before each step (untimed)"},
            "plain_lsd": {"value": args.steps * n / (ms_c * 1e-3) / 1e9, "ms_per_step": ms_c / args.steps,
                          "call": f"isort_radix_u64 on (segment id << 32 | key), {cbits} key bits, radix 2^8"},
            "speedup_vs_plain": ms_c / ms_s,
            "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in prof.items()},
        })
    print(json.dumps(line), flush=True)
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
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--radix-bits", type=int, default=8)
    ap.add_argument("--workload", default="uniform",
                    choices=["uniform", "learned", "learned64", "segmented", "small", "typed"],
                    help="uniform: the benchmark; learned / segmented: secondary comparisons with plain LSD; "
                         "small: the 65,536-key case and the block networks on 1,024 keys")
    ap.add_argument("--nbuckets", type=int, default=0, help="learned: bucket count (0: the library's choice)")
    ap.add_argument("--model", type=int, default=0, choices=[0, 1, 2],
                    help="learned: 0 = piecewise-linear CDF, 1 = the 1-32-1 MLP CDF, 2 = regular sampling (untrained)")
    ap.add_argument("--dist", default="lognormal", choices=["zipf", "lognormal", "gmm", "range48"],
                    help="learned: key distribution; learned64: range48 for keys on [0, 2^48)")
    args = ap.parse_args()
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

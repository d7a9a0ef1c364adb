#!/usr/bin/env python3
"""Benchmark: effective n^2 k GOPS of Low(A A^T) mod p at n = k = 16384.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: A is 16384 x 16384 over F_p, p = 2^31 - 1 (= 3 mod 4, so Y =
[[a, b], [-b, a]] (x) I), int32 residues drawn uniformly (SplitMix64, seed
0x2101010250 + 2) and stored balanced in (-p/2, p/2).  One step is one call
of aat_modp (the whole hot path: Y from Algorithm 3, the S-block kernel, the
tensor-core leaf products, the post-additions, the recursion of Algorithm 1)
with A already resident in HBM.  A (1 GiB) is larger than L2 (129 MB), so no
flush is needed between steps.

Printed: ONE JSON line (rank 0) with the metric, the device-timed value, the
end-to-end value through aat_modp_host (host buffers, copies inside the
timed region), the roofline of the dominant kernel (the tcgen05 leaf,
measured with CUDA events on its stream during the timed steps), the plain
full product and plain lower-triangle product on the same leaf, the CPU
oracle on a bounded sample of the workload, the SM clocks sampled during the
timed region and the number of kernel launches.

Under torchrun (N > 1) every rank runs its own independent product of the
same size (replicas, weak scaling): value = N n^2 k / max-over-ranks time.

--impl reference times the CPU oracle (oracle/, test infrastructure) on the
host cores: each step computes a bounded sample of Low(A A^T) entries and the
value is scaled to the full product by its multiply-add count.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "effective n²k GOPS for Low(A·Aᵀ) mod p at n=k=16384 vs plain GPU full product"
N = K = 16384
P = 2**31 - 1
SEED_OFFSET = 2
# DRAM traffic of the dominant kernel from one ncu capture of three 8192^3
# leaf products mod 2^31-1 (dram__bytes_read.sum + dram__bytes_write.sum:
# 11.63, 11.63 and 11.63 GB for 10.995 TFLOP of algorithmic work each;
# CTA-pair form, tiles in bands of 2048 rows), scaled to the average launch
# of the step by its algorithmic work.  None whenever the kernel has changed
# since the counters were taken.
LEAF_TC_BYTES_PER_FLOP = 11.63e9 / 10.995e12
# Dense BF16 rate of the tensor pipe per SM and clock (a 128 x 256 x 16
# tcgen05.mma every 128 cycles) and the SM count: the nominal rate at the
# clock the run was sampled at.
BF16_FLOP_PER_SM_CLK = 8192
SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="skip baselines, e2e and the CPU oracle (quick runs)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuning of levels / leaf form / digit form")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (512^2, 8192^2, 16384x4096, complex, batch)")
    return ap.parse_args()


def workload_config(levels=None):
    cfg = {
        "workload": "Low(A A^T) mod p, A 16384x16384 over F_p, p=2^31-1, balanced int32 "
                    "residues (SplitMix64 seed 0x2101010250+2)",
        "n": N, "k": K, "p": P,
        "input": "balanced",
        "l2": "A is 1 GiB > L2 (129 MB): no flush between steps",
    }
    if levels is not None:
        cfg["levels"] = levels
    return cfg


def make_input():
    from paper_2101_01025_gb300 import synth
    return synth.residues(synth.SEED_BASE + SEED_OFFSET, (N, K), P, balanced=True)


# ------------------------------------------------------------ CPU oracle

def oracle_sample(A, seconds, seed=0):
    """Time the oracle on a bounded sample of lower-triangle rows; returns
    (value GOPS scaled to the full product, seconds, description, threads)."""
    import numpy as np
    import oracle
    threads = oracle.num_threads()
    rng = np.random.default_rng(seed)

    def run_rows(rows):
        ij = np.concatenate([np.stack([np.full(r + 1, r), np.arange(r + 1)], 1) for r in rows])
        t0 = time.perf_counter()
        oracle.aat_modp_entries(A, P, ij, threads=threads)
        return time.perf_counter() - t0, float(len(ij)) * K

    # calibrate on a few rows, then size the sample to `seconds`
    cal_rows = [int(x) for x in rng.integers(N // 4, N, 2)]
    t, macs = run_rows(cal_rows)
    rate = macs / max(t, 1e-6)
    want = max(1.0, rate * seconds / (K * N / 2.0))
    rows = sorted(int(x) for x in rng.integers(0, N, int(want) + 1))
    t, macs = run_rows(rows)
    full = N * (N + 1) / 2.0 * K
    t_full = t * full / macs
    value = N * N * K / t_full / 1e9
    desc = ("%d rows of Low(A A^T) (%.3g multiply-adds, %.2f%% of the lower triangle); "
            "time scaled to the full product by multiply-add count" % (len(rows), macs,
                                                                      100.0 * macs / full))
    return value, t, desc, threads, t_full


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    A = make_input()
    per_step = min(10.0, max(2.0, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup):
        oracle_sample(A, per_step, seed=100 + i)
    vals, secs, tfull = [], [], []
    desc, threads = "", 0
    for i in range(args.steps):
        v, t, desc, threads, t_full = oracle_sample(A, per_step, seed=i)
        vals.append(v)
        secs.append(t)
        tfull.append(t_full)
    value = statistics.mean(vals)
    line = {
        "metric": METRIC, "value": value, "unit": "GOPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * statistics.mean(tfull),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int128 (exact, CPU)", "data": "synthetic", "config": workload_config(),
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "GOPS", "cores": threads, "kind": "oracle",
                         "sample": desc + "; one sample per step"},
        "e2e": {"value": value, "unit": "GOPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ clocks

class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return local_rank


# ------------------------------------------------------------ replicas

def max_over_ranks(x, world, device):
    """The largest x over all ranks (the slowest rank's time); the process
    group (NCCL on the GPUs, gloo in the CPU tests) must be initialised when
    world > 1."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, ms_step):
    """Whole-job throughput in effective n^2 k GOPS: every rank computes its
    own product of the workload's size (replicas, no exchange), and the job
    takes as long as its slowest rank (ms_step, already the max over ranks)."""
    return world * N * N * K / (ms_step * 1e-3) / 1e9


# ------------------------------------------------------------ GPU arm

def bf16_peaks(peaks):
    """(peak, its source, sustained peak) in TFLOP/s: the measured burst rate
    for a kernel timed over a sub-second region, the sustained one beside it."""
    if "bf16_tflops" in peaks:
        return (float(peaks["bf16_tflops"]), "of measured (bf16 burst)",
                float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])))
    return 1900.0, "of fallback (bf16 burst)", 1700.0


def run_configs(peaks):
    """The other workloads, each timed with CUDA events (one untimed run, then
    repetitions) with the library's per-kernel profile: ms, effective n^2 k
    GOPS and the leaf's achieved rate against the BF16 burst peak."""
    import torch

    import paper_2101_01025_gb300 as aat
    from paper_2101_01025_gb300 import _native, synth, testing
    peak, peak_src, _ = bf16_peaks(peaks)
    gen = torch.Generator(device="cuda")
    out = {}

    def measure(name, fn, work, reps, what, leaf_cls, plan_flops=None):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        _native.lib().aat_profile_begin()
        # one event pair per call, all calls back to back: the median call
        # (one slow call does not move it)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        prof = _native.Profile()
        _native.check(_native.lib().aat_profile_end(prof))
        calls = sorted(a.elapsed_time(b) for a, b in ev)
        ms = calls[len(calls) // 2]
        lf = prof.as_dict().get(leaf_cls, {"launches": 0, "ms": 0.0, "work": 0.0})
        if plan_flops is not None:
            # a graph launch carries no per-kernel events: the plan's
            # algorithmic tensor work over the whole plan's time (a lower
            # bound on its leaf kernel's rate)
            ach = plan_flops / (ms * 1e-3) / 1e12
            rf = {"kernel": leaf_cls + " (whole plan: one graph launch)", "bound": "tensor",
                  "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                  "peak_source": peak_src}
        else:
            ach = lf["work"] / max(lf["ms"], 1e-9) / 1e9
            rf = {"kernel": leaf_cls, "bound": "tensor", "achieved": ach, "peak": peak,
                  "unit": "TFLOP/s", "frac": ach / peak, "peak_source": peak_src,
                  "share": lf["ms"] / max(sum(calls), 1e-9)}
        out[name] = {"what": what, "ms": ms, "ms_min_median_max": [calls[0], ms, calls[-1]],
                     "calls": reps, "gops": work / (ms * 1e-3) / 1e9, "roofline": rf}

    def residues(n, k, p, seed):
        gen.manual_seed(seed)
        return torch.randint(0, p, (n, k), dtype=torch.int32, device="cuda", generator=gen)

    # 512 x 512 over F_131071, one level then the leaf
    A = torch.from_numpy(synth.residues(synth.SEED_BASE, (512, 512), 131071)).cuda()
    C = torch.empty((512, 512), dtype=torch.int32, device="cuda")
    measure("512x512_p131071_l1", lambda: aat.aat_modp(A, 131071, C=C, levels=1),
            512.0**3, 20, "Low(A A^T) mod 131071, one recursion level, tensor-core leaf",
            "leaf_tc")
    # 8192^2 and 16384 x 4096 over F_65521 and F_131071 (default depth)
    for (n, k) in ((8192, 8192), (16384, 4096)):
        for p in (65521, 131071):
            A = residues(n, k, p, synth.SEED_BASE + 1)
            C = torch.empty((n, n), dtype=torch.int32, device="cuda")
            lv = testing.plan_stats(n, k, p).levels
            measure("%dx%d_p%d" % (n, k, p), lambda: aat.aat_modp(A, p, C=C), float(n) * n * k,
                    5, "Low(A A^T) mod %d, %d recursion levels (default depth)" % (p, lv),
                    "leaf_tc")
            del A, C
    # complex 8192 x 8192: A A^H by 2M and A A^T by Algorithm 1, FP32 class
    gen.manual_seed(synth.SEED_BASE + 3)
    Z = torch.view_as_complex(torch.randn((8192, 8192, 2), device="cuda", generator=gen))
    CZ = torch.empty((8192, 8192), dtype=torch.complex64, device="cuda")
    measure("complex8192_aah_2m_fp32", lambda: aat.aah_complex(Z, C=CZ), 8192.0**3, 5,
            "Low(A A^H) by 2M, FP32-accurate (3 BF16 pieces)", "leaf_f32")
    measure("complex8192_aat_alg1_fp32", lambda: aat.aat_complex(Z, C=CZ), 8192.0**3, 5,
            "Low(A A^T) by Algorithm 1 (Y = i I, default depth), FP32-accurate", "leaf_f32")
    del Z, CZ
    # batch: 256 problems over F_65521 + 64 complex A A^H, log-uniform sizes
    ns = synth.log_uniform_ints(synth.SEED_BASE + 4, 256, 64, 2048)
    ks = synth.log_uniform_ints(synth.SEED_BASE + 5, 256, 64, 4096)
    cn = synth.log_uniform_ints(synth.SEED_BASE + 6, 64, 64, 2048)
    ck = synth.log_uniform_ints(synth.SEED_BASE + 7, 64, 64, 4096)
    gen.manual_seed(synth.SEED_BASE + 5)
    fp = [("modp", torch.randint(0, 65521, (int(n), int(k)), dtype=torch.int32, device="cuda",
                                 generator=gen),
           torch.empty((int(n), int(n)), dtype=torch.int32, device="cuda"), 65521, 0)
          for n, k in zip(ns, ks)]
    cx = [("aah", torch.view_as_complex(torch.randn((int(n), int(k), 2), device="cuda",
                                                    generator=gen)),
           torch.empty((int(n), int(n)), dtype=torch.complex64, device="cuda"), 0, 0)
          for n, k in zip(cn, ck)]
    # algorithmic tensor FLOPs: mod 65521 three plane products (two digit
    # planes, one pair sum) of the lower triangle; complex A A^H (FP32 class)
    # six piece products of H (all n^2 entries) and of G (lower triangle)
    def flops(probs):
        f = 0.0
        for kind, Ap, _, _, _ in probs:
            n, k = float(Ap.shape[0]), float(Ap.shape[1])
            low = n * (n + 1) / 2 * k
            f += 2 * 3 * low if kind == "modp" else 2 * 6 * (n * n * k + low)
        return f
    for name, probs, cls in (("batch256_p65521", fp, "leaf_tc"), ("batch64_complex_aah", cx,
                                                                   "leaf_f32"),
                             ("batch256_p65521_plus_64_complex", fp + cx, "leaf_tc+leaf_f32")):
        plan = aat.Plan(probs)
        work = sum(float(Ap.shape[0]) ** 2 * Ap.shape[1] for _, Ap, _, _, _ in probs)
        measure(name, plan.execute, work, 10,
                "one plan (one CUDA graph launch), sum of n^2 k over its problems", cls,
                plan_flops=flops(probs))
        out[name]["plan"] = plan.info()
        plan.close()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    import paper_2101_01025_gb300 as aat
    from paper_2101_01025_gb300 import _native, testing

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    A_host = make_input()
    A = torch.from_numpy(A_host).cuda()
    C = torch.empty((N, N), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    # autotuning (untimed): recursion depth, leaf kernel form and digit form
    # for this shape, kept by the library for the timed calls below
    tuned = None
    if not args.no_tune:
        tuned = aat.tune_modp(N, K, P, reps=2)
    levels = testing.plan_stats(N, K, P).levels

    def step():
        aat.aat_modp(A, P, C=C)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(gpu_index(local))
    clocks.start()
    _native.lib().aat_profile_begin()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    prof = _native.Profile()
    _native.check(_native.lib().aat_profile_end(prof))
    clk = clocks.stop()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world, "cuda")
    ms_step = ms_total / args.steps
    value = job_value(world, ms_step)
    status = aat.aat_device_status()

    profd = prof.as_dict()
    launches = sum(v["launches"] for v in profd.values())
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    leaf = profd.get("leaf_tc", {"launches": 0, "ms": 0.0, "work": 0.0})
    achieved = leaf["work"] / max(leaf["ms"], 1e-9) / 1e9  # TFLOP/s
    peak, peak_src, sust = bf16_peaks(peaks)
    sm_mhz = clk.get("sm_mhz")
    roofline = {
        "bound": "tensor",
        "kernel": "leaf_tc_kernel (tcgen05 kind::f16, CTA pairs, BF16 digits)",
        "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
        "peak_source": peak_src,
        "frac_of_sustained": achieved / sust,
        "clock_normalised": None if not sm_mhz else {
            "sm_mhz": sm_mhz,
            "nominal_tflops_at_clock": SMS * BF16_FLOP_PER_SM_CLK * sm_mhz * 1e6 / 1e12,
            "frac": achieved / (SMS * BF16_FLOP_PER_SM_CLK * sm_mhz * 1e6 / 1e12),
            "what": "achieved over the tensor pipe's dense BF16 rate (8192 FLOP per SM and "
                    "clock, 152 SMs) at the median SM clock sampled in the timed region"},
        "traffic": (None if LEAF_TC_BYTES_PER_FLOP is None else
                    LEAF_TC_BYTES_PER_FLOP * leaf["work"] / max(leaf["launches"], 1)),
        "launches": leaf["launches"],
        "avg_launch_ms": leaf["ms"] / max(leaf["launches"], 1),
        "share_of_step": leaf["ms"] / max(ms_total, 1e-9),
        "work_per_step_tflop": leaf["work"] / args.steps / 1e12,
    }
    kernels = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps}
               for k, v in profd.items()}
    for name in ("sblocks", "split", "postadd", "add_low"):
        if name in profd and profd[name]["ms"] > 0:
            kernels[name]["gbs"] = profd[name]["work"] / (profd[name]["ms"] * 1e-3) / 1e9

    extras = {}
    if not args.no_extras and rank == 0:
        # plain products on the same exact leaf
        def timed(fn, reps):
            fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps
        reps = max(2, args.steps // 3)
        ms_full = timed(lambda: aat.aat_gemm_modp(A, A, P, C=C), reps)
        ms_syrk = timed(lambda: aat.aat_modp(A, P, C=C, levels=0), reps)
        extras["baselines"] = {
            "plain_full_product": {"gops": N * N * K / (ms_full * 1e-3) / 1e9, "ms": ms_full,
                                   "what": "aat_gemm_modp(A, A): all n^2 entries, same leaf"},
            "plain_lower_product": {"gops": N * N * K / (ms_syrk * 1e-3) / 1e9, "ms": ms_syrk,
                                    "what": "aat_modp with 0 recursion levels"},
            "speedup_vs_full_product": ms_full / ms_step,
            "speedup_vs_lower_product": ms_syrk / ms_step,
        }
        del C
        torch.cuda.empty_cache()
    barrier()

    e2e = None
    if not args.no_extras:
        Ah = torch.from_numpy(A_host).pin_memory()
        Ch = torch.empty((N, N), dtype=torch.int32).pin_memory()
        del A
        torch.cuda.empty_cache()
        # the host link alone (untimed for the metric): 256 MiB of A from
        # pinned memory, median of 5 copies
        probe = torch.empty((N // 4, K), dtype=torch.int32, device="cuda")
        link = []
        for _ in range(6):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            probe.copy_(Ah[: N // 4], non_blocking=True)
            torch.cuda.synchronize()
            link.append(probe.numel() * 4 / (time.perf_counter() - t1) / 1e9)
        link_gbs = sorted(link[1:])[2]
        del probe
        for _ in range(max(1, args.warmup)):
            aat.aat_modp_host(Ah, P, C=Ch)
        barrier()
        calls = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            t1 = time.perf_counter()
            aat.aat_modp_host(Ah, P, C=Ch)
            calls.append(1e3 * (time.perf_counter() - t1))
        t_e2e = max_over_ranks(time.perf_counter() - t0, world, "cuda") / args.steps
        e2e = {"value": job_value(world, 1e3 * t_e2e), "unit": "GOPS",
               "ms_per_step": 1e3 * t_e2e,
               "ms_per_call_min_median_max": [min(calls), sorted(calls)[len(calls) // 2],
                                              max(calls)],
               "host_link_h2d_gbs": link_gbs,
               "h2d_bytes_per_step": N * K * 4,
               "d2h_bytes_per_step": aat.aat_modp_host_d2h_bytes(N),
               "api": "aat_modp_host (pinned host A and C; copies inside the call: A11 "
                      "first so that P1 runs while the rest of A arrives; the lower "
                      "triangle of C back in row bands, the rows below n/2 while the last "
                      "product runs)"}

    configs = None
    if not args.no_configs and rank == 0:
        configs = run_configs(peaks)

    cpu = None
    if not args.no_extras and rank == 0 and world == 1:
        v, t, desc, threads, _ = oracle_sample(A_host, 12.0)
        cpu = {"value": v, "unit": "GOPS", "cores": threads, "kind": "oracle", "sample": desc,
               "seconds": t}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GOPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "arith": "exact: bf16 digit products, fp32 partial sums "
                                      "< 2^24 drained to int32, int32/int64 mod p",
            "data": "synthetic", "config": dict(workload_config(levels), tuned=tuned),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "kernels": kernels,
            "device_status": status, "configs": configs,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

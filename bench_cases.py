"""Named single-GPU workloads for profiling the kernels in isolation.

    python bench_cases.py leaf 8192 [--p P] [--reps R]
    python bench_cases.py syrk 8192 [--k K] ...
    python bench_cases.py aat 16384 [--k K] [--levels L] ...
    python bench_cases.py full 16384 ...
    python bench_cases.py peaks 4 --reps 5

leaf: one leaf product X Y^T mod p of n x n x n (digit planes split first);
aah / aatc2m / aatc: complex A A^H by 2M, A A^T by 2M, A A^T by Algorithm 1
with Y = i I (--prec: BF16 pieces per FP32 value);
syrk: Low(X X^T) with 0 recursion levels; aat: Low(A A^T) by Algorithm 1;
full: the plain full product A A^T; peaks: the rates of the mma.sync
instructions of the INT8 and FP64 leaves (n blocks per SM).  Inputs are
seeded uniform residues generated on the device.  Prints the time of each
repetition.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["leaf", "syrk", "aat", "full", "aah", "aatc2m", "aatc",
                                     "batch", "peaks"])
    ap.add_argument("n", type=int)
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--p", type=int, default=2**31 - 1)
    ap.add_argument("--levels", type=int, default=None)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16x3", "bf16"],
                    help="complex cases: BF16 pieces per FP32 value (3, 2, 1)")
    ap.add_argument("--leaf", default="tc", choices=["tc", "i8", "f64", "simt"],
                    help="leaf kind of the F_p cases")
    ap.add_argument("--plain-digits", action="store_true",
                    help="one product per digit pair instead of the pair-sum form")
    ap.add_argument("--low-memory", action="store_true",
                    help="the low-memory schedule (plane passes, AAT_LOW_MEMORY)")
    ap.add_argument("--profile", action="store_true",
                    help="per kernel class: launches, ms per repetition and the rate of "
                         "its algorithmic work (bytes or FLOPs) over the timed repetitions")
    a = ap.parse_args(argv)

    import torch

    import paper_2101_01025_gb300 as aat
    from paper_2101_01025_gb300 import build, testing

    build.build()
    torch.manual_seed(0x2101)
    n, k, p = a.n, a.k or a.n, a.p
    flags = aat.AAT_DIGITS_PLAIN if a.plain_digits else 0
    if a.low_memory:
        flags |= aat.AAT_LOW_MEMORY
    flags |= {"tc": aat.AAT_LEAF_TC, "i8": aat.AAT_LEAF_I8, "f64": aat.AAT_LEAF_F64,
              "simt": aat.AAT_LEAF_SIMT}[a.leaf]
    half = (p - 1) // 2
    if a.case == "batch":
        return batch_case(a)
    if a.case == "peaks":
        return peaks_case(a)
    if a.case in ("aah", "aatc2m", "aatc"):
        cflags = {"fp32": aat.AAT_C_FP32, "bf16x3": aat.AAT_C_BF16X3, "bf16": aat.AAT_C_BF16}[a.prec]
        Z = torch.randn((n, k), dtype=torch.complex64, device="cuda")
        CZ = torch.empty((n, n), dtype=torch.complex64, device="cuda")
        if a.case == "aatc":   # Algorithm 1 with Y = i I
            fn = lambda: aat.aat_complex(Z, C=CZ, flags=cflags, levels=a.levels)  # noqa: E731
        else:
            f = aat.aah_complex if a.case == "aah" else aat.aat_complex_2m
            fn = lambda: f(Z, C=CZ, flags=cflags)  # noqa: E731
    else:
        X = torch.randint(-half, half + 1, (n, k), dtype=torch.int32, device="cuda")
        C = torch.empty((n, n), dtype=torch.int32, device="cuda")
    if a.case in ("aah", "aatc2m", "aatc"):
        pass
    elif a.case == "leaf":
        Y = torch.randint(-half, half + 1, (n, k), dtype=torch.int32, device="cuda")
        fn = lambda: testing.leaf(X, Y, p, C=C, leafkind=flags)  # noqa: E731
    elif a.case == "syrk":
        fn = lambda: aat.aat_modp(X, p, C=C, levels=0, flags=flags)  # noqa: E731
    elif a.case == "aat":
        fn = lambda: aat.aat_modp(X, p, C=C, levels=a.levels, flags=flags)  # noqa: E731
    else:
        fn = lambda: aat.aat_gemm_modp(X, X, p, C=C, flags=flags)  # noqa: E731
    times = []
    if a.profile:
        fn()
        torch.cuda.synchronize()
        from paper_2101_01025_gb300 import _native
        _native.lib().aat_profile_begin()
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    out = {"case": a.case, "n": n, "k": k, "p": p, "levels": a.levels,
           "plain_digits": a.plain_digits, "prec": a.prec, "leaf": a.leaf,
           "ms": times, "status": aat.aat_device_status()}
    if a.profile:
        out["kernels"] = profile_end(a.reps)
    print(json.dumps(out))


def profile_end(reps):
    """Per kernel class over the profiled repetitions: launches and ms per
    repetition, and GB/s (element-wise classes) or TFLOP/s (leaf classes) of
    the algorithmic work the library counts for each launch."""
    from paper_2101_01025_gb300 import _native
    prof = _native.Profile()
    _native.check(_native.lib().aat_profile_end(prof))
    out = {}
    for name, v in prof.as_dict().items():
        per_s = v["work"] / max(v["ms"] * 1e-3, 1e-12)
        leafy = name.startswith("leaf")
        out[name] = {"launches": v["launches"] / reps, "ms": v["ms"] / reps,
                     ("tflops" if leafy else "gbs"): per_s / 1e12 if leafy else per_s / 1e9}
    return out


def peaks_case(a):
    """Peak rates of the legacy tensor instructions the INT8 and FP64 leaves
    use (mma.sync m16n8k32 s8, m8n8k4 f64), from register-only loops on every
    SM (n blocks per SM), with the SM clock sampled during each run."""
    import ctypes
    import subprocess
    import statistics
    import tempfile
    import os
    import torch

    from paper_2101_01025_gb300 import _native
    L = _native.lib()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = sms * max(1, a.n)
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    out = {"case": "peaks", "sms": sms, "blocks": blocks}
    for kind, name in ((0, "int8_mma_sync_m16n8k32"), (1, "fp64_mma_sync_m8n8k4")):
        ops = ctypes.c_double()
        iters = 2000
        # calibrate to ~0.3 s per launch
        for _ in range(3):
            _native.check(L.aatx_mma_peak(kind, iters, blocks, sink.data_ptr(),
                                          ctypes.byref(ops), st))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _native.check(L.aatx_mma_peak(kind, iters, blocks, sink.data_ptr(),
                                          ctypes.byref(ops), st))
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            iters = max(1, int(iters * 300.0 / max(ms, 1e-3)))
        fd, path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        smi = subprocess.Popen(["nvidia-smi", "-i", "0", "--query-gpu=clocks.sm",
                                "--format=csv,noheader,nounits", "-lms", "100"],
                               stdout=open(path, "w"), stderr=subprocess.DEVNULL)
        rates = []
        for _ in range(a.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _native.check(L.aatx_mma_peak(kind, iters, blocks, sink.data_ptr(),
                                          ctypes.byref(ops), st))
            e1.record()
            torch.cuda.synchronize()
            rates.append(ops.value / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        smi.terminate()
        smi.wait()
        mhz = [float(x) for x in open(path).read().split() if x.strip().isdigit()]
        os.unlink(path)
        out[name] = {"tops": max(rates), "tops_runs": rates, "iters": iters,
                     "sm_mhz_median": statistics.median(mhz) if mhz else None,
                     "unit": "TOPS (int8)" if kind == 0 else "TFLOP/s (fp64)"}
    print(json.dumps(out))


def batch_case(a):
    """n problems over F_65521 (n, k log-uniform in [64, 2048] x [64, 4096])
    plus n // 4 complex A A^H problems of the same spread, one plan; prints
    sum n^2 k / time for the whole batch and for each kind alone."""
    import torch

    import paper_2101_01025_gb300 as aat
    from paper_2101_01025_gb300 import synth

    count = a.n
    p = 65521
    ns = synth.log_uniform_ints(synth.SEED_BASE + 4, count, 64, 2048)
    ks = synth.log_uniform_ints(synth.SEED_BASE + 5, count, 64, 4096)
    cn = synth.log_uniform_ints(synth.SEED_BASE + 6, count // 4, 64, 2048)
    ck = synth.log_uniform_ints(synth.SEED_BASE + 7, count // 4, 64, 4096)
    torch.manual_seed(0x2101)
    fp = [("modp", torch.randint(0, p, (int(n), int(k)), dtype=torch.int32, device="cuda"),
           torch.empty((int(n), int(n)), dtype=torch.int32, device="cuda"), p, 0)
          for n, k in zip(ns, ks)]
    cx = [("aah", torch.randn((int(n), int(k)), dtype=torch.complex64, device="cuda"),
           torch.empty((int(n), int(n)), dtype=torch.complex64, device="cuda"), 0, 0)
          for n, k in zip(cn, ck)]
    out = {"case": "batch", "problems": count, "complex": count // 4}
    for name, probs in (("modp", fp), ("aah", cx), ("all", fp + cx)):
        if a.profile:
            # the plan's first run is eager (outside the graph): its kernels
            # carry the library's per-launch events
            torch.cuda.synchronize()
            from paper_2101_01025_gb300 import _native
            _native.lib().aat_profile_begin()
        plan = aat.Plan(probs)
        if a.profile:
            out[name + "_eager_kernels"] = profile_end(1)
        work = sum(float(A.shape[0]) ** 2 * A.shape[1] for _, A, _, _, _ in probs)
        plan.execute()
        torch.cuda.synchronize()
        times = []
        for _ in range(a.reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.execute()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        out[name] = {"ms": times, "gops": work / (min(times) * 1e-3) / 1e9, "info": plan.info()}
        plan.close()
    out["status"] = aat.aat_device_status()
    print(json.dumps(out))


if __name__ == "__main__":
    main()

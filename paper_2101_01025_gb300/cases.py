"""Named single-GPU workloads for profiling the kernels in isolation.

    python -m paper_2101_01025_gb300.cases leaf 8192 [--p P] [--reps R]
    python -m paper_2101_01025_gb300.cases syrk 8192 [--k K] ...
    python -m paper_2101_01025_gb300.cases aat 16384 [--k K] [--levels L] ...
    python -m paper_2101_01025_gb300.cases full 16384 ...

leaf: one leaf product X Y^T mod p of n x n x n (digit planes split first);
syrk: Low(X X^T) with 0 recursion levels; aat: Low(A A^T) by Algorithm 1;
full: the plain full product A A^T.  Inputs are seeded uniform residues
generated on the device.  Prints the mean time per repetition.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["leaf", "syrk", "aat", "full", "aah", "aatc2m"])
    ap.add_argument("n", type=int)
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--p", type=int, default=2**31 - 1)
    ap.add_argument("--levels", type=int, default=None)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16x3", "bf16"],
                    help="complex cases: BF16 pieces per FP32 value (3, 2, 1)")
    ap.add_argument("--plain-digits", action="store_true",
                    help="one product per digit pair instead of the pair-sum form")
    a = ap.parse_args(argv)

    import torch

    import paper_2101_01025_gb300 as aat
    from paper_2101_01025_gb300 import build, testing

    build.build()
    torch.manual_seed(0x2101)
    n, k, p = a.n, a.k or a.n, a.p
    flags = aat.AAT_DIGITS_PLAIN if a.plain_digits else 0
    half = (p - 1) // 2
    if a.case in ("aah", "aatc2m"):
        cflags = {"fp32": aat.AAT_C_FP32, "bf16x3": aat.AAT_C_BF16X3, "bf16": aat.AAT_C_BF16}[a.prec]
        Z = torch.randn((n, k), dtype=torch.complex64, device="cuda")
        CZ = torch.empty((n, n), dtype=torch.complex64, device="cuda")
        f = aat.aah_complex if a.case == "aah" else aat.aat_complex_2m
        fn = lambda: f(Z, C=CZ, flags=cflags)  # noqa: E731
    else:
        X = torch.randint(-half, half + 1, (n, k), dtype=torch.int32, device="cuda")
        C = torch.empty((n, n), dtype=torch.int32, device="cuda")
    if a.case in ("aah", "aatc2m"):
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
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    print(json.dumps({"case": a.case, "n": n, "k": k, "p": p, "levels": a.levels,
                      "plain_digits": a.plain_digits, "prec": a.prec,
                      "ms": times, "status": aat.aat_device_status()}))


if __name__ == "__main__":
    main()

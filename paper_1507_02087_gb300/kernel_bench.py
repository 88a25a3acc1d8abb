"""Micro-benchmark of the tensor-core square on its own (through the C ABI).

Builds a random symmetric FP32 matrix X of size ld, stores it as three bf16 pieces
and times C = X X^T with the same tcgen05 kernel the mixed SP2 path uses (upper
tiles + mirror, FP32 output).  Used for kernel profiling on a small, self-contained
case:  python -m paper_1507_02087_gb300.kernel_bench --ld 8192 --reps 5
With --sp2 it times the SP2 forward square itself (expansion loop of a mixed handle).
"""
from __future__ import annotations

import argparse
import json

import torch

from . import sp2


def pieces(x32: torch.Tensor) -> torch.Tensor:
    p0 = x32.to(torch.bfloat16)
    r1 = x32 - p0.float()
    p1 = r1.to(torch.bfloat16)
    p2 = (r1 - p1.float()).to(torch.bfloat16)
    return torch.stack([p0, p1, p2])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ld", type=int, default=8192)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--full", action="store_true", help="all tiles (general product) instead of upper + mirror")
    ap.add_argument("--tile", default="auto", choices=["auto", "128", "pair"],
                    help="128 x 128 tiles per SM, 256 x 256 tiles per SM pair, or auto (pair if ld % 256 == 0)")
    ap.add_argument("--sp2", action="store_true",
                    help="time the SP2 forward square instead (expansion loop only, stream launches) on the "
                         "dense gapped input of size ld, nocc = ld / 2, gap 0.01")
    ap.add_argument("--bsr", default=None, metavar="LX,LY,LZ",
                    help="time the block-sparse squares instead, on the gapped tight-binding lattice of these "
                         "dimensions (LX = 32), tau 1e-4, stream launches")
    ap.add_argument("--rule", default="error", choices=["error", "block", "mixed"])
    ap.add_argument("--products", default="tensor", choices=["tensor", "cuda"],
                    help="--bsr: block products on the tensor cores (fp16x3) or FP32 CUDA cores")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "bf16x6", "bf16x3", "fp16x3", "tf32x3"],
                    help="--sp2: the tensor-core precision mode of the handle")
    a = ap.parse_args()
    if a.sp2:
        return sp2_forward(a)
    if a.bsr:
        return bsr_squares(a)
    ld = a.ld
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn(ld, ld, device="cuda", generator=g)
    X = ((X + X.T) / (2 * ld ** 0.5)).float()
    arena = pieces(X).unsqueeze(0).contiguous()
    out = torch.empty(ld, ld, device="cuda", dtype=torch.float32)
    upper = not a.full
    sp2.sp2_test_tc_gemm(arena, ld, 1, 0, 0, upper, out, tile=a.tile)    # warm-up
    times = []
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sp2.sp2_test_tc_gemm(arena, ld, 1, 0, 0, upper, out, tile=a.tile)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = min(times)
    edge = 256 if a.tile == "pair" or (a.tile == "auto" and ld % 256 == 0) else 128
    R = ld // edge
    tiles = R * (R + 1) // 2 if upper else R * R
    executed = 6 * tiles * edge * edge * ld * 2
    print(json.dumps({"ld": ld, "upper": upper, "tile_edge": edge, "ms": ms, "tiles": tiles,
                      "executed_tflops": executed / (ms * 1e-3) / 1e12,
                      "algorithmic_tflops": 6 * ld * ld * (ld + 1) / (ms * 1e-3) / 1e12 if upper else None}))


def sp2_forward(a):
    """Forward squares of the mixed expansion (MODE_SP2_STEP epilogue: X_{k-1} read, pieces
    written, Frobenius partials) on a 4-slot-ring handle, launched on the stream one by one
    so that a kernel profiler sees each square."""
    from . import inputs
    N = a.ld
    case = inputs.dense_gapped(N, N // 2, gap=0.01, seed=0, device="cuda", want_exact=False)
    F = case.F
    D = torch.empty_like(F)
    with sp2.Purifier(N, N // 2, a.precision, corrections=0, refine_steps=0, launch_mode=1, tile=a.tile) as P:
        P.run(F, D)
        per = []
        for _ in range(a.reps):
            P.run(F, D)
            fi = P.info()
            per.append(fi["loop_ms"] / fi["hist_len"])
        info = P.info()
    ms = min(per)
    products = {"mixed": 6, "bf16x6": 6, "bf16x3": 3, "fp16x3": 3, "tf32x3": 3}[a.precision]
    print(json.dumps({"ld": N, "mode": "sp2_forward", "tile": a.tile, "precision": a.precision,
                      "squares": int(info["hist_len"]), "ms_per_square_incl_stop_test": ms,
                      "executed_tflops": products * N * N * (N + 1) / (ms * 1e-3) / 1e12,
                      "useful_tflops": N * N * (N + 1) / (ms * 1e-3) / 1e12}))


def bsr_squares(a):
    """Block-sparse SP2 (launch mode 1) on a tight-binding lattice: work counters and the
    summed device time of the numeric block-square launches."""
    from . import inputs
    dims = tuple(int(x) for x in a.bsr.split(","))
    tb = inputs.tight_binding(dims=dims)
    rp, ci, vals = (torch.from_numpy(x).cuda() for x in tb.bsr(32))
    with sp2.BsrPurifier(tb.N, tb.nocc, 1e-4, rule=a.rule, launch_mode=1, products=a.products,
                         norm="mixed" if a.rule == "mixed" else "fro") as P:
        for _ in range(max(1, a.reps)):
            P.run(rp, ci, vals, dense=False)
        w = P.info()
    sec = w["numeric_ms"] * 1e-3
    print(json.dumps({"N": tb.N, "dims": dims, "rule": a.rule, "products": a.products, "n_iter": w["n_iter"],
                      "nnzb_D": w["nnzb"], "block_products": w["block_products"],
                      "needed_products": w["needed_products"], "numeric_ms": w["numeric_ms"],
                      "executed_tflops": 2 * 32 ** 3 * w["block_products"] / sec / 1e12,
                      "useful_tflops": 2 * 32 ** 3 * w["needed_products"] / sec / 1e12,
                      "loop_ms": w["loop_ms"]}))


if __name__ == "__main__":
    main()

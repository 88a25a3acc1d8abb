#!/usr/bin/env python
"""Time-to-D of SP2 density-matrix purification on one GB300.

A step is one full purification F -> D of the dense workload N=8192, nocc=4096:
spectrum uniform in [-1,-0.005] U [0.005,1] (gap 0.01) with eigenvectors from the QR
factor of a seeded Gaussian matrix.  The timed path is the tensor-core one (Gershgorin
bounds, scaling, squares on the tcgen05 tensor cores with the device-side parameterless
stop, the F-driven subspace correction and a refinement pair; by default in the fp16x3
mode: two scaled fp16 pieces per value, three piece products per square), whose result must
be within ||D - D_exact||_F / sqrt(nocc) <= 1e-6 of the exact projector; the plain FP64
path is timed beside it for the comparison.  F (512 MiB FP64) is resident in HBM before
the timed region; every buffer the loop streams is larger than the 129 MB L2, so no flush
is needed between steps.  The default line also carries secondary records of the other
workloads (N = 400 on the FP64 and tensor-core paths, a batch of 64 uneven problems, the 32^3
block-sparse lattice, SP2-ACC).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-D & TFLOP/s, mixed vs FP64 SP2 on 1 GB300 at ||D-D_ref||_F/sqrt(nocc)<=1e-6"
N_DEFAULT, GAP_DEFAULT = 8192, 0.01
TOL = 1e-6
# FP64 runs on the SMs' FP64 pipes: the nominal 1.25 TFLOP/s over 152 SMs at the
# 2070 MHz maximum clock is 4 flop per clock per SM; taken at the measured clock.
SMS, FP64_FLOP_PER_CLK_SM, SM_MAX_MHZ = 152, 4.0, 2070.0
# 16-bit piece products per square on the tensor cores, per precision mode
PRODUCTS = {"mixed": 6, "bf16x6": 6, "bf16x3": 3, "fp16x3": 3, "tf32x3": 3}
# The roofline basis of the tensor-core square: useful flops N^2 (N+1) per square (upper triangle
# with the diagonal, N multiply-adds each) times 3 split products, the budget of an FP32-grade
# square on 16-bit tensor cores; the executed fraction counts the mode's own piece products.
SPLIT_BASIS = 3
DTYPE = {"mixed": "bf16x6->f32 (three bf16 pieces, six products), f64 reductions",
         "bf16x6": "bf16x6->f32 (three bf16 pieces, six products), f64 reductions",
         "bf16x3": "bf16x3->f32 (two bf16 pieces, three products), f64 reductions",
         "fp16x3": "fp16x3->f32 (two scaled fp16 pieces, three products), f64 reductions",
         "tf32x3": "tf32x3->f32 (two tf32 pieces, three products), f64 reductions"}


def workload_name(N, nocc, gap):
    return f"dense N={N} nocc={nocc} gap={gap:g}, random-Q (QR of seeded Gaussian, seed 0)"


# DRAM bytes (read + write) of one forward-square launch from an ncu capture of the current
# kernel (profiles/tc_gemm_pair_sp2_forward_dram_ld8192.md), keyed by (N, tile kind, precision).
FWD_TRAFFIC_BYTES = {(8192, "pair", "fp16x3"): 1.510e9 + 260.6e6}
FP32_FLOP_PER_CLK_SM = 256     # 128 FP32 FMA lanes per SM


def tensor_peak(precision: str) -> tuple[float, str]:
    """Sustained tensor peak of the mode's MMA kind: the measured bf16 figure (fp16 and bf16 share
    the kind::f16 rate); kind::tf32 at the nominal ratio 1.1 / 2.25 PFLOP/s of it."""
    bf = load_peaks().get("bf16_tflops_sustained") or 1700.0
    if precision == "tf32x3":
        return bf * 1.1 / 2.25, ("MEASURED_PEAKS.json bf16_tflops_sustained x 1.1/2.25 (the nominal "
                                 "tf32 / bf16 dense ratio)")
    return bf, "MEASURED_PEAKS.json bf16_tflops_sustained (fp16 and bf16 share the kind::f16 rate)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["dense", "batch64", "bsr"], default="dense",
                    help="dense: one N x N problem (default N=8192); batch64: 64 problems, N log-uniform "
                         "in [128, 2048], seed 1; bsr: gapped tight-binding 32^3 lattice, 32 x 32 blocks, "
                         "block truncation tau in {1e-4, 1e-6}")
    ap.add_argument("--precision", choices=["fp16x3", "bf16x6", "mixed", "bf16x3", "tf32x3", "fp64"], default="fp16x3",
                    help="fp16x3 (default): two scaled fp16 pieces, three products; bf16x6 (= mixed): three bf16 "
                         "pieces, six products; bf16x3: two bf16 pieces, three products; fp64: the plain method")
    ap.add_argument("--no-secondary", action="store_true",
                    help="dense workload: skip the secondary records (N = 400, batch of 64, 32^3 block-sparse, "
                         "SP2-ACC)")
    ap.add_argument("--refine", choices=["tc", "fp64", "mcweeny"], default="tc",
                    help="mixed path: refinement pair on the tensor cores (tc) or in FP64 (fp64), or one "
                         "McWeeny step with its square in FP64 (mcweeny)")
    ap.add_argument("--fp64-sample-squares", type=int, default=0,
                    help="with --fp64-steps 0: time this many FP64 squares and estimate the FP64 time-to-D")
    ap.add_argument("--acc", type=float, default=None, metavar="SLACK",
                    help="SP2-ACC (homo/lumo-based accelerated expansion) with the construction's homo and lumo "
                         "eigenvalues as inner bounds and SLACK as the distance of the outer ones")
    ap.add_argument("--mcweeny", choices=["mcw", "mcw-acc"], default=None,
                    help="FP64 path: the McWeeny expansion (mcw) or McW-ACC with the construction's gap as the "
                         "gap estimate, mu = 0 (the construction splits the spectrum at 0)")
    ap.add_argument("--norm", choices=["fro", "mixed", "spectral"], default="fro",
                    help="error measure of the stop: Frobenius v_i, mixed norm m_i, or the spectral e_i "
                         "(Lanczos; --precision fp64 only)")
    ap.add_argument("--rule", choices=["error", "block", "mixed"], default="error",
                    help="block-sparse truncation rule of the headline line (both rules are reported)")
    ap.add_argument("--N", type=int, default=N_DEFAULT)
    ap.add_argument("--nocc", type=int, default=None)
    ap.add_argument("--gap", type=float, default=GAP_DEFAULT)
    ap.add_argument("--input", choices=["qr", "householder"], default="qr",
                    help="eigenvectors: QR of a seeded Gaussian (seed 0) or 64 seeded Householder reflectors "
                         "(seed 3, the N=32768 workload)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="0 skips the host-buffer measurement")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed runs of the FP64 path (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    return ap.parse_args()


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, power, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("SP2_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(F_np, nocc, n_squares_full, budget_s):
    """Time the CPU oracle on a bounded sample: bounds, scaling and as many iterations
    (one N^3 matrix product each) as fit in `budget_s`; the full time-to-D is
    extrapolated linearly to `n_squares_full` products."""
    import numpy as np
    from oracle import sp2_oracle as o
    t0 = time.perf_counter()
    lmin, lmax = o.gershgorin_bounds(F_np)
    X = o.initial_scaling(F_np, lmin, lmax)
    t_setup = time.perf_counter() - t0
    iters, t_it = 0, 0.0
    while True:
        t1 = time.perf_counter()
        X2 = X @ X
        o.idempotency_error_fro(X, X2)
        tr = float(np.trace(X))
        X = X2 if tr > nocc else 2.0 * X - X2
        t_it += time.perf_counter() - t1
        iters += 1
        if t_setup + t_it >= budget_s or iters >= n_squares_full:
            break
    per = t_it / iters
    est_ms = (t_setup + per * n_squares_full) * 1e3
    return est_ms, {"setup_s": t_setup, "iters_timed": iters, "s_per_iter": per}


def oracle_squares(N, nocc, gap):
    try:
        data = json.load(open(os.path.join(ROOT, "oracle", "iteration_counts.json")))
        return data[f"dense_N{N}_nocc{nocc}_gap{gap:g}_seed0"]["squares"]
    except Exception:
        return None


def run_reference(a, ws, rank):
    """The oracle arm: the CPU FP64 oracle, as it stands, timed on the host cores."""
    if rank != 0:
        return
    import torch
    from paper_1507_02087_gb300 import inputs
    nocc = a.nocc if a.nocc is not None else a.N // 2
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    case = inputs.dense_gapped(a.N, nocc, gap=a.gap, seed=0, device=dev, want_exact=False)
    F_np = case.F.cpu().numpy()
    n_sq = oracle_squares(a.N, nocc, a.gap)
    known = n_sq is not None
    n_sq = n_sq or 60
    times, info = [], None
    budget = max(2.0, a.cpu_sample_s / 3)
    for step in range(a.warmup + a.steps):
        est, info = oracle_sample(F_np, nocc, n_sq, budget)
        if step >= a.warmup:
            times.append(est)
    ms = statistics.mean(times)
    sample = (f"per step: Gershgorin bounds, scaling and the first {info['iters_timed']} of the oracle's "
              f"{n_sq} FP64 iterations (one numpy N^3 product each) at N={a.N}, extrapolated linearly; "
              f"the square count {'comes from a full oracle run (oracle/iteration_counts.json)' if known else 'is assumed'}")
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a.N, nocc, a.gap), "N": a.N, "nocc": nocc, "gap": a.gap,
                       "precision": "fp64 (CPU oracle, numpy/OpenBLAS)"},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def useful_flops(N, squares, deriv_steps, corrected, refine_steps):
    """Algorithmic flops of one mixed run, counting each symmetric square as N^2 (N+1)
    (upper triangle with the diagonal, N multiply-adds each), a general product as 2 N^3."""
    sq = N * N * (N + 1)
    f = squares * sq
    if corrected:
        f += 2 * N ** 3 + sq + deriv_steps * 2 * sq
    f += refine_steps * sq
    return f


def tc_precision(a):
    return a.precision if a.precision in PRODUCTS else "fp16x3"


def batch_record(a, local, precision, steps, warmup, compare_tiles=False, fp64_steps=0):
    """64 problems of uneven size in one batch (one launch sequence, per-problem stops): time-to-D
    from CUDA events on the launching stream, the largest error against each exact projector, and
    the tensor rate of the whole run (useful flops of every product over the time-to-D)."""
    import torch
    from paper_1507_02087_gb300 import inputs, sp2
    torch.cuda.set_device(local)
    cases = inputs.dense_batch(device=torch.device("cuda", local))
    Ns, noccs = [c.N for c in cases], [c.nocc for c in cases]
    Fs = [c.F for c in cases]
    stream = torch.cuda.current_stream()

    def timed(B, k):
        Ds = [torch.empty_like(F) for F in Fs]
        tms = []
        for _ in range(k):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.run(Fs, Ds, stream)
            e1.record(stream)
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
        errs = [float(torch.linalg.norm(D - c.D_exact)) / math.sqrt(c.nocc) for D, c in zip(Ds, cases)]
        infos = [B.info(i) for i in range(len(cases))]
        return statistics.mean(tms), max(errs), infos

    with sp2.BatchPurifier(Ns, noccs, precision) as B:
        timed(B, warmup)
        clocks = ClockSampler(local)
        clocks.start()
        ms, err, infos = timed(B, steps)
        clk = clocks.stop()
    flops = sum(useful_flops(N, i["hist_len"], i["n_iter"], True, 2) for N, i in zip(Ns, infos))
    peak, peak_src = tensor_peak(precision)
    achieved = SPLIT_BASIS * flops / (ms * 1e-3) / 1e12
    rec = {"workload": "batch of 64 dense problems, N log-uniform in [128, 2048] (seed 1), nocc = N/2, gap "
                       "uniform in [0.005, 0.1]; one launch sequence, per-problem stops",
           "precision": precision, "time_to_d_ms": ms, "steps": steps, "warmup": warmup,
           "max_err_vs_exact": err, "meets_tolerance": bool(err <= TOL),
           "tflops_useful": flops / (ms * 1e-3) / 1e12,
           "n_iter_range": [min(i["n_iter"] for i in infos), max(i["n_iter"] for i in infos)],
           "tile": infos[0]["tile"],
           "roofline": {"bound": "tensor", "kernel": "every tensor-core launch of the run, over the whole time-to-D",
                        "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "basis": "useful flops of all products x 3 split products over the time-to-D; peak: "
                                 + peak_src,
                        "traffic": None},
           "clocks": clk, "sum_N3": sum(N ** 3 for N in Ns), "count": len(cases)}
    if compare_tiles:
        tiles = {"tuned": infos[0]["tile"]}
        for t in ("128", "pair"):
            with sp2.BatchPurifier(Ns, noccs, precision, tile=t) as Bt:
                timed(Bt, 1)
                tiles[t + "_ms"] = timed(Bt, max(1, steps))[0]
        rec["tiles"] = tiles
    if fp64_steps > 0:
        with sp2.BatchPurifier(Ns, noccs, "fp64") as B64:
            ms64, err64, inf64 = timed(B64, fp64_steps)
        rec["fp64_path"] = {"time_to_d_ms": ms64, "max_err_vs_exact": err64, "speedup_vs_fp64": ms64 / ms}
    return rec


def run_batch(a, ws, rank, local):
    """The batch workload as the headline line."""
    prec = tc_precision(a)
    rec = batch_record(a, local, prec, a.steps, a.warmup, compare_tiles=True, fp64_steps=a.fp64_steps)
    barrier(ws)
    ms = max_over_ranks(rec["time_to_d_ms"], ws)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[prec], "data": "synthetic",
            "config": {"workload": rec["workload"], "count": rec["count"], "sum_N3": rec["sum_N3"],
                       "precision": prec},
            **{k: rec[k] for k in ("max_err_vs_exact", "meets_tolerance", "tflops_useful", "n_iter_range",
                                   "tiles", "roofline", "clocks")},
            "fp64_path": rec.get("fp64_path")}), flush=True)


def bsr_launches(squares, rule):
    """Kernels of one block-sparse run (dense output off): 14 set-up kernels, 12 per loop
    round (+1 each with the error-controlled rule, +3 with the mixed-norm rule, +35 Lanczos
    launches per round for the mixed-norm stop that goes with it), rounds launched in pairs."""
    extra = {"error": 1, "mixed": 3}.get(rule, 0)
    lz = 35 if rule == "mixed" else 0
    rounds = squares + (squares & 1)
    return 14 + extra + (12 + extra + lz) * rounds


def bsr_error_bound(tb, D):
    """A-posteriori bound of ||D - P||_F / sqrt(nocc) against the exact projector P of the lattice
    Hamiltonian, from what holds at any size: with P~ the projector onto the eigenvectors of D
    above 1/2, ||D - P~||_F <= ||D^2 - D||_F / (1 - 2m) (eigenvalues of D within m of {0, 1}), and
    by the sin-theta theorem with the gap delta of F, ||P~ - P||_F <= (||[F, D]||_F + 2 ||F||
    ||D - P~||_F) / delta; delta >= 2 (1 - max |disorder|) (Weyl), ||F|| from Gershgorin."""
    import numpy as np
    import torch
    r = torch.from_numpy(tb.rows).cuda()
    c = torch.from_numpy(tb.cols).cuda()
    idx = torch.cat([torch.stack([r, c]), torch.arange(tb.N, device="cuda").repeat(2, 1)], dim=1)
    val = torch.cat([torch.full((r.numel(),), -tb.hop, dtype=torch.float64, device="cuda"),
                     torch.from_numpy(tb.onsite).cuda()])
    Fs = torch.sparse_coo_tensor(idx, val, (tb.N, tb.N)).coalesce()
    FD = torch.sparse.mm(Fs, D)
    comm = float(torch.linalg.norm(FD - FD.T))
    del FD
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    D32 = D.float()
    idem = float(torch.linalg.norm((D32 @ D32).double() - D))
    torch.backends.cuda.matmul.allow_tf32 = prev
    del D32
    delta = 2.0 * (1.0 - float(np.max(np.abs(np.abs(tb.onsite) - 1.0))))
    fnorm = float(np.max(np.abs(tb.onsite))) + 6 * tb.hop
    m = 0.01
    dpt = idem / (1 - 2 * m)
    bound = dpt + (comm + 2 * fnorm * dpt) / delta
    return {"err_bound": bound / math.sqrt(tb.nocc), "idem": idem / math.sqrt(tb.nocc),
            "comm": comm / math.sqrt(tb.nocc), "trace_err": abs(float(torch.trace(D)) - tb.nocc),
            "valid": bool(idem < m / 2)}


def bsr_roofline(w, mhz, products="tensor"):
    """Roofline of the numeric block square, summed over one run's squares (CUDA events around
    each launch, launch_mode 1).  Tensor cores: the needed 32^3 block products (both factors
    stored, output block J >= I) x 2 x 32^3 flops x the 3 split products, against the bf16
    tensor peak; frac_executed also counts the zero blocks that fill the 4 x 8-block tiles.
    FP32 CUDA cores: the products formed, against the FP32 FMA peak at the measured clock."""
    kern_s = w["numeric_ms"] * 1e-3
    need = 2 * 32 ** 3 * w["needed_products"]
    execd = 2 * 32 ** 3 * w["block_products"]
    common = {"kernel_ms_per_run": w["numeric_ms"], "block_products": w["block_products"],
              "needed_products": w["needed_products"], "square_blocks": w["square_blocks"],
              "useful_tflops": need / kern_s / 1e12, "traffic": None}
    if products == "tensor":
        peak = load_peaks().get("bf16_tflops_sustained") or 1700.0
        achieved = SPLIT_BASIS * need / kern_s / 1e12
        return {"bound": "tensor",
                "kernel": "bsr_tc_kernel (4 x 8-block tiles, fp16x3 block products, all squares)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "frac_executed": SPLIT_BASIS * execd / kern_s / 1e12 / peak,
                "basis": "needed block products x 2 x 32^3 flops x 3 split products / summed CUDA-event "
                         "time of the numeric launches",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (fp16 and bf16 inputs share the "
                               "kind::f16 tensor rate)", **common}
    peak32 = SMS * FP32_FLOP_PER_CLK_SM * mhz * 1e6 / 1e12
    streamed = 2 * 32 * 32 * 4 * w["block_products"]          # two FP32 blocks per product, no reuse
    return {"bound": "alu", "kernel": "bsr_numeric_kernel (FP32 CUDA-core block products, all squares)",
            "achieved": execd / kern_s / 1e12, "peak": peak32, "unit": "TFLOP/s",
            "frac": execd / kern_s / 1e12 / peak32,
            "peak_source": f"152 SMs x 128 FP32 FMA/clk x 2 x {mhz:.0f} MHz (median SM clock)",
            "streamed_gbs": streamed / kern_s / 1e9,
            "streamed_frac_of_hbm": streamed / kern_s / 1e9 / (load_peaks().get("hbm_gbs") or 6800.0),
            **common}


def bsr_record(a, local, steps, warmup, tau=1e-4, rule="mixed"):
    """The 32^3 block-sparse lattice (N = 32768) with the mixed-norm truncation and the mixed-norm
    stop (the pairing of the paper's §6 calculations): time-to-D from CUDA events, the a-posteriori
    error bound (computed once, outside the timed region), and the roofline of the numeric block
    square from a stream-launched run (CUDA events around each of its launches)."""
    import torch
    from paper_1507_02087_gb300 import inputs, sp2
    torch.cuda.set_device(local)
    tb = inputs.tight_binding(L=32)
    rp, ci, vals = tb.bsr(32)
    rp_d, ci_d, vals_d = (torch.from_numpy(x).cuda() for x in (rp, ci, vals))
    stream = torch.cuda.current_stream()
    norm = "mixed" if rule == "mixed" else "fro"
    with sp2.BsrPurifier(tb.N, tb.nocc, tau, rule=rule, norm=norm) as P:
        for _ in range(warmup):
            P.run(rp_d, ci_d, vals_d, dense=False, stream=stream)
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        tms = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.run(rp_d, ci_d, vals_d, dense=False, stream=stream)
            e1.record(stream)
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
        clocks = clk.stop()
        info = P.info()
        D = P.run(rp_d, ci_d, vals_d, stream=stream)
        torch.cuda.synchronize()
    err = bsr_error_bound(tb, D)
    del D
    with sp2.BsrPurifier(tb.N, tb.nocc, tau, rule=rule, launch_mode=1, norm=norm) as P1:
        P1.run(rp_d, ci_d, vals_d, dense=False, stream=stream)
        w = P1.info()
    mhz = clocks.get("sm_mhz") or SM_MAX_MHZ
    nb = tb.N // 32
    return {"workload": "gapped tight-binding 32x32x32 simple cubic (N=32768), delta=1, t=0.3, sigma=0.05 (seed 2), "
                        "nocc=N/2, 32x32 FP32 blocks; mixed-norm truncation tau=%g with the mixed-norm stop" % tau,
            "time_to_d_ms": statistics.mean(tms), "steps": steps, "warmup": warmup,
            "n_iter": info["n_iter"], "squares": info["hist_len"], "kept_fraction": info["nnzb"] / nb ** 2,
            "err_bound_vs_exact": err["err_bound"], "idem": err["idem"], "comm": err["comm"],
            "trace_err": err["trace_err"], "bound_valid": err["valid"],
            "roofline": bsr_roofline(w, mhz), "clocks": clocks}


def run_bsr(a, ws, rank, local):
    """Block-sparse path on the 32^3 tight-binding Hamiltonian (N = 32768)."""
    import numpy as np
    import torch
    from paper_1507_02087_gb300 import inputs, sp2
    torch.cuda.set_device(local)
    tb = inputs.tight_binding(L=32)
    rp, ci, vals = tb.bsr(32)
    rp_d, ci_d, vals_d = (torch.from_numpy(x).cuda() for x in (rp, ci, vals))
    stream = torch.cuda.current_stream()
    out = {}
    rules = [a.rule] + [r for r in ("error", "block", "mixed") if r != a.rule]
    # SP2-ACC bounds without an eigensolver: the lattice without disorder has |lambda| >= delta = 1
    # with equality attained (eps_k = 0 at k = (pi/2, pi/2, pi/2)), and the onsite disorder moves
    # every eigenvalue by at most its largest magnitude (Weyl)
    mn = float(np.max(np.abs(np.abs(tb.onsite) - 1.0)))
    acc_bounds = (-1.0 - mn, -1.0 + mn, 1.0 - mn, 1.0 + mn)
    cases = [(r, t, None) for r in rules for t in (1e-4, 1e-6)] + [(r, 1e-4, acc_bounds) for r in ("error", "mixed")]
    for rule, tau, acc in cases:
        # the mixed-norm rule runs with the mixed-norm stop (the pairing of the paper's §6)
        with sp2.BsrPurifier(tb.N, tb.nocc, tau, rule=rule, norm="mixed" if rule == "mixed" else "fro") as P:
            if acc is not None:
                P.set_homo_lumo(acc)
            for _ in range(a.warmup):
                P.run(rp_d, ci_d, vals_d, dense=False, stream=stream)
            torch.cuda.synchronize()
            tms = []
            for _ in range(a.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                P.run(rp_d, ci_d, vals_d, dense=False, stream=stream)
                e1.record(stream)
                e1.synchronize()
                tms.append(e0.elapsed_time(e1))
            info = P.info()
        nb = tb.N // 32
        out[f"{rule}:tau={tau:g}" + (":sp2-acc" if acc is not None else "")] = {
                               "time_to_d_ms": statistics.mean(tms), "n_iter": info["n_iter"],
                               "squares": info["hist_len"], "stop_reason": info["stop_reason"],
                               "nnzb_D": info["nnzb"], "kept_fraction": info["nnzb"] / nb ** 2,
                               "v_last": float(info["v"][-1]) if len(info["v"]) else None,
                               "trace_err": abs(float(info["trace"][info["n_iter"]]) - tb.nocc),
                               "ms_per_square": info["loop_ms"] / max(1, info["hist_len"])}
    # roofline of the numeric block square (the dominant kernel): a launch-mode-1 handle
    # records CUDA events around each of its launches; work from the device's counters
    with sp2.BsrPurifier(tb.N, tb.nocc, 1e-4, rule=a.rule, launch_mode=1,
                         norm="mixed" if a.rule == "mixed" else "fro") as P1:
        P1.run(rp_d, ci_d, vals_d, dense=False, stream=stream)
        P1.run(rp_d, ci_d, vals_d, dense=False, stream=stream)
        w = P1.info()
    clk = ClockSampler(local)
    clk.start()
    with sp2.BsrPurifier(tb.N, tb.nocc, 1e-4, rule=a.rule, launch_mode=1,
                         norm="mixed" if a.rule == "mixed" else "fro") as P1:
        P1.run(rp_d, ci_d, vals_d, dense=False, stream=stream)
        w = P1.info()
    clocks = clk.stop()
    mhz = clocks.get("sm_mhz") or SM_MAX_MHZ
    roofline = bsr_roofline(w, mhz)
    if rank == 0:
        main_ms = out[f"{a.rule}:tau=0.0001"]["time_to_d_ms"]
        print(json.dumps({
            "metric": "time-to-D, block-sparse SP2 with block truncation (FP32 blocks, FP64 reductions)",
            "value": main_ms, "unit": "ms", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": main_ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp16x3->f32 block products (two scaled fp16 pieces, three products), f32 blocks, "
                     "f64 reductions", "data": "synthetic",
            "config": {"workload": "gapped tight-binding 32x32x32 simple cubic (N=32768), delta=1, t=0.3, "
                                   "sigma=0.05 (seed 2), nocc=N/2, 32x32 blocks (x-lines)",
                       "nnzb_F": int(rp[-1]), "tau": 1e-4,
                       "truncation": {"error": "error-controlled, ||E_i||_F <= tau",
                                      "block": "per block, ||X_IJ||_F < tau dropped",
                                      "mixed": "mixed norm, ||E_i||_M <= tau (block-row sums), "
                                               "with the mixed-norm stop"}[a.rule]},
            "runs": out, "roofline": roofline,
            "gpu_launches": a.steps * bsr_launches(out[f"{a.rule}:tau=0.0001"]["squares"], a.rule)}), flush=True)


def main():
    a = parse()
    ws, rank, local = dist_setup()
    if a.impl == "reference":
        run_reference(a, ws, rank)
        return
    if a.workload == "batch64":
        run_batch(a, ws, rank, local)
        return
    if a.workload == "bsr":
        run_bsr(a, ws, rank, local)
        return
    import torch
    from paper_1507_02087_gb300 import inputs, sp2

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nocc = a.nocc if a.nocc is not None else a.N // 2
    N = a.N
    if a.input == "householder":
        case = inputs.householder_gapped(N, nocc, gap=a.gap, n_reflectors=64, seed=3, device=dev)
    else:
        case = inputs.dense_gapped(N, nocc, gap=a.gap, seed=0, device=dev, want_exact=True)
    F = case.F.contiguous()
    D_exact = case.D_exact
    D = torch.empty_like(F)
    stream = torch.cuda.current_stream()
    if a.norm == "spectral" and a.precision != "fp64":
        raise SystemExit("--norm spectral needs --precision fp64")
    P = sp2.Purifier(N, nocc, a.precision, refine_fp64={"tc": 0, "fp64": 1, "mcweeny": 2}[a.refine], norm=a.norm)
    if a.mcweeny is not None:
        if a.precision != "fp64":
            raise SystemExit("--mcweeny needs --precision fp64")
        P.set_mcweeny(a.mcweeny, 0.0, a.gap)
    acc_bounds = None
    if a.acc is not None:
        import numpy as np
        lam = np.sort(np.asarray(case.lam))
        homo, lumo = float(lam[nocc - 1]), float(lam[nocc])
        acc_bounds = (homo - a.acc, homo, lumo, lumo + a.acc)
        P.set_homo_lumo(acc_bounds)

    def err_vs_exact():
        return float(torch.linalg.norm(D - D_exact)) / math.sqrt(nocc)

    for _ in range(a.warmup):
        P.run(F, D, stream)
    torch.cuda.synchronize()
    err_first = err_vs_exact()

    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    step_ms, loop_ms, infos = [], [], []
    for _ in range(a.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.run(F, D, stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        inf = P.info()
        loop_ms.append(inf["loop_ms"])
        infos.append(inf)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(step_ms), ws)
    info = infos[-1]
    err = err_vs_exact()
    status_ok = all(i["status"] == 0 for i in infos)
    mixed = a.precision in PRODUCTS
    squares = info["hist_len"]
    n_iter = info["n_iter"]
    flops = useful_flops(N, squares, n_iter, mixed, 2 if mixed else 0) if mixed else N * N * (N + 1) * squares
    tflops = flops / (ms * 1e-3) / 1e12
    # FP64 path per square: square (+ McWeeny product) + finalize (+ 35 Lanczos launches for the
    # spectral stop); bounds, init, scaling and the output copy once
    per_square = 2 + (1 if a.mcweeny else 0) + (35 if a.norm == "spectral" else 0)
    # tensor-core path: bounds, init, scaling; {square, finalize, loop check} per forward round; two
    # correction products; {derivative step, advance} per derivative round; refinement input and pair;
    # the output assembly
    launches_per_step = (3 + per_square * squares + 1) if not mixed else (3 + 3 * squares + 2 + 2 * n_iter + 3 + 1)

    # roofline of the dominant kernel, timed on its own inside the same device loop:
    # a forward-only handle runs the square + stop-test loop; loop time / squares is
    # the average duration of one square launch (plus the few-microsecond stop test).
    peaks = load_peaks()
    if mixed:
        with sp2.Purifier(N, nocc, a.precision, corrections=0, refine_steps=0) as Pf:
            if acc_bounds is not None:
                Pf.set_homo_lumo(acc_bounds)
            Pf.run(F, D, stream)
            kt = []
            for _ in range(max(1, min(3, a.steps))):
                Pf.run(F, D, stream)
                fi = Pf.info()
                kt.append(fi["loop_ms"] / fi["hist_len"])
            tile_used = fi["tile"]
        kern_ms = statistics.mean(kt)
        useful = N * N * (N + 1)                      # one upper-triangle square with the diagonal
        alg = SPLIT_BASIS * useful
        executed = PRODUCTS[a.precision] * useful
        achieved = alg / (kern_ms * 1e-3) / 1e12
        peak, peak_src = tensor_peak(a.precision)
        kname = ("tc_gemm_pair_kernel (256x256 tiles per SM pair" if tile_used == "pair"
                 else "tc_gemm_kernel (128x128 tiles per SM")
        roofline = {"bound": "tensor", "kernel": kname + ", forward square, MODE_SP2_STEP, " + a.precision + ")",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "frac_executed": executed / (kern_ms * 1e-3) / 1e12 / peak,
                    "basis": "achieved = N^2 (N+1) useful flops per square x 3 split products / CUDA-event time "
                             "per square; frac_executed counts the mode's own %d piece products" % PRODUCTS[a.precision],
                    "useful_tflops": useful / (kern_ms * 1e-3) / 1e12,
                    "ms_per_launch": kern_ms,
                    "peak_source": peak_src + "; the sustained figure, the kernel is timed inside a long step",
                    "algorithmic_flops_per_launch": alg,
                    "traffic": FWD_TRAFFIC_BYTES.get((N, tile_used, a.precision))}
    else:
        kern_ms = statistics.mean(l / s for l, s in zip(loop_ms, [i["hist_len"] for i in infos]))
        mhz = clk.get("sm_mhz") or SM_MAX_MHZ
        peak = SMS * FP64_FLOP_PER_CLK_SM * mhz * 1e6 / 1e12
        alg = N * N * (N + 1) * (2 if a.mcweeny else 1)     # McWeeny: two products per step
        achieved = alg / (kern_ms * 1e-3) / 1e12
        kname = ("mcw_square_kernel + mcw_prod_kernel (+finalize), one McWeeny step" if a.mcweeny
                 else "syrk_f64_kernel (+finalize)")
        roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "ms_per_launch": kern_ms,
                    "peak_source": f"152 SMs x 4 FP64 flop/clk x {mhz:.0f} MHz (median SM clock under load)",
                    "algorithmic_flops_per_launch": alg, "traffic": None}

    # end to end through the public API with host buffers (copies inside the timed region), right
    # after the device-timed steps and before the long FP64 comparison run
    e2e = None
    if a.e2e_steps > 0:
        F_h = torch.empty((N, N), dtype=torch.float64, pin_memory=True)
        F_h.copy_(F.cpu())
        D_h = torch.empty((N, N), dtype=torch.float64, pin_memory=True)
        F_hn, D_hn = F_h.numpy(), D_h.numpy()
        P.run_host(F_hn, D_hn, stream)          # allocates the staging buffers once
        e2e_ms, e2e_loop, e2e_dev = [], [], []
        eclk = ClockSampler(local)
        eclk.start()
        for _ in range(a.e2e_steps):
            torch.cuda.synchronize()
            d0 = torch.cuda.Event(enable_timing=True)
            d1 = torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            d0.record(stream)
            P.run_host(F_hn, D_hn, stream)
            d1.record(stream)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            d1.synchronize()
            e2e_dev.append(d0.elapsed_time(d1))      # device span of the call: copies + run
            e2e_loop.append(P.info()["loop_ms"])     # device time of the same call's loop
        ec = eclk.stop()
        # the same copies alone (torch, same pinned buffers) and a resident run right after, with
        # CUDA events: the parts of the e2e device span
        def span(fn):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)
        F_probe = torch.empty_like(F)
        parts = {"h2d_ms": span(lambda: F_probe.copy_(F_h, non_blocking=True)),
                 "d2h_ms": span(lambda: D_h.copy_(F_probe, non_blocking=True)),
                 "resident_run_ms": span(lambda: P.run(F, D, stream))}
        del F_probe
        # the clocks of these steps: a long run under the power cap can drift below the clocks of
        # the device-timed steps, which then shows up in the gap between e2e and value
        e2e = {"value": max_over_ranks(statistics.mean(e2e_ms), ws), "unit": "ms",
               "h2d_bytes_per_step": N * N * 8, "d2h_bytes_per_step": N * N * 8,
               "steps_ms": e2e_ms, "device_span_ms": e2e_dev, "loop_ms": e2e_loop, "parts": parts,
               "value_loop_ms": statistics.mean(loop_ms),
               "sm_mhz": ec.get("sm_mhz"), "reasons": ec.get("reasons")}

    # the plain FP64 path, for the comparison the metric asks for
    fp64 = None
    if mixed and a.fp64_steps > 0:
        with sp2.Purifier(N, nocc, "fp64") as P64:
            if acc_bounds is not None:
                P64.set_homo_lumo(acc_bounds)
            D64 = torch.empty_like(F)
            tms = []
            for _ in range(a.fp64_steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                P64.run(F, D64, stream)
                e1.record(stream)
                e1.synchronize()
                tms.append(e0.elapsed_time(e1))
            i64 = P64.info()
            e64 = float(torch.linalg.norm(D64 - D_exact)) / math.sqrt(nocc)
            del D64
        sq64 = i64["hist_len"]
        fp64 = {"time_to_d_ms": statistics.mean(tms), "steps": a.fp64_steps, "n_iter": i64["n_iter"],
                "squares": sq64, "err_vs_exact": e64,
                "tflops": N * N * (N + 1) * sq64 / (statistics.mean(tms) * 1e-3) / 1e12,
                "speedup_mixed_vs_fp64": statistics.mean(tms) / ms}
    elif mixed and a.fp64_sample_squares > 0:
        # too long to run whole: time K FP64 squares (a handle capped at K iterations) and
        # scale by the square count of the mixed run, which the FP64 path does not undercut
        K = a.fp64_sample_squares
        with sp2.Purifier(N, nocc, "fp64", max_iter=K) as P64:
            D64 = torch.empty_like(F)
            P64.run(F, D64, stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P64.run(F, D64, stream)
            e1.record(stream)
            e1.synchronize()
            i64 = P64.info()
            del D64
        per_sq = i64["loop_ms"] / max(1, i64["hist_len"])
        est = e0.elapsed_time(e1) - i64["loop_ms"] + per_sq * squares
        fp64 = {"time_to_d_ms": est, "estimate": True,
                "sample": f"{i64['hist_len']} FP64 squares timed ({per_sq:.1f} ms each), scaled to the "
                          f"{squares} squares of the mixed run (a lower bound: the FP64 path stops at the same "
                          f"or a later square)",
                "tflops": N * N * (N + 1) / (per_sq * 1e-3) / 1e12,
                "speedup_mixed_vs_fp64": est / ms}

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        n_or = oracle_squares(N, nocc, a.gap) or (fp64["squares"] if fp64 else squares)
        est, sinfo = oracle_sample(F.cpu().numpy(), nocc, n_or, a.cpu_sample_s)
        cpu = {"value": est, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": (f"CPU FP64 oracle (numpy/OpenBLAS): Gershgorin, scaling and {sinfo['iters_timed']} of "
                          f"its {n_or} iterations at N={N}, extrapolated linearly "
                          f"({sinfo['s_per_iter']:.2f} s per iteration)")}

    if rank == 0:
        line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None,
                "dtype": (DTYPE[a.precision] + {"tc": "", "fp64": ", f64 refinement pair",
                                                "mcweeny": ", f64-square McWeeny step"}[a.refine])
                if mixed else "f64",
                "data": "synthetic",
                "config": {"workload": workload_name(N, nocc, a.gap) if a.input == "qr" else
                           f"dense N={N} nocc={nocc} gap={a.gap:g}, Q = 64 Householder reflectors (seed 3)",
                           "N": N, "nocc": nocc, "gap": a.gap,
                           "precision": a.precision, "refine": a.refine if mixed else None, "norm": a.norm,
                           "expansion": ("SP2-ACC (homo/lumo bounds, slack %g)" % a.acc if a.acc is not None
                                         else {"mcw": "McWeeny (mu = 0)", "mcw-acc": "McW-ACC (mu = 0, xi = gap)"}
                                         [a.mcweeny] if a.mcweeny else "SP2 (trace-based)"),
                           "parallelism": "replicas" if ws > 1 else "1 GPU",
                           "l2": "no flush: F 512 MiB and the streamed iterates exceed the 129 MB L2"},
                "err_vs_exact": err, "err_first_run": err_first, "meets_tolerance": bool(err <= TOL and status_ok),
                "tolerance": TOL, "status_ok": status_ok,
                "tflops_useful": tflops, "squares": squares, "n_iter": n_iter,
                "stop_reason": info["stop_reason"], "loop_ms": statistics.mean(loop_ms),
                "fp64_path": fp64, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches_per_step * a.steps), "clocks": clk}
    P.close()
    del P
    if rank == 0 and ws == 1 and mixed and not a.no_secondary and a.acc is None and a.input == "qr":
        # the other workloads, each with its own CUDA-event time, error, roofline and clock record
        steps2, warm2 = max(1, min(a.steps, 5)), max(1, min(a.warmup, 2))
        line["secondary"] = {
            "n400": n400_record(a, local, steps2, warm2),
            "batch64": batch_record(a, local, a.precision, steps2, warm2),
            "bsr32": bsr_record(a, local, max(1, min(a.steps, 3)), 1),
            "sp2_acc": acc_record(a, local, F, D_exact, case.lam, nocc, steps2, warm2),
        }
    if rank == 0:
        print(json.dumps(line), flush=True)


def n400_record(a, local, steps, warmup):
    """The small dense case (N = 400, nocc = 200, gap 0.1, seed 0: the construction of the dense
    tests, plain Alg. 3 with the parameterless stop) on the FP64 path and on the tensor-core path
    of the headline's precision: time-to-D from CUDA events, error against the exact projector."""
    import torch
    from paper_1507_02087_gb300 import inputs, sp2
    case = inputs.dense_n400()
    F = case.F.cuda().contiguous()
    D_exact = case.D_exact.cuda()
    stream = torch.cuda.current_stream()
    out = {"workload": "dense N=400 nocc=200 gap=0.1, random-Q (QR of seeded Gaussian, seed 0)"}
    for prec in ("fp64", a.precision):
        D = torch.empty_like(F)
        with sp2.Purifier(400, 200, prec) as P:
            for _ in range(warmup):
                P.run(F, D, stream)
            tms = []
            for _ in range(steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                P.run(F, D, stream)
                e1.record(stream)
                e1.synchronize()
                tms.append(e0.elapsed_time(e1))
            info = P.info()
        out[prec] = {"time_to_d_ms": statistics.mean(tms), "n_iter": info["n_iter"],
                     "stop_reason": info["stop_reason"], "status": info["status"],
                     "err_vs_exact": float(torch.linalg.norm(D - D_exact)) / math.sqrt(200)}
    return out


def acc_record(a, local, F, D_exact, lam, nocc, steps, warmup, slack=1e-3):
    """SP2-ACC (Alg. 4 / Alg. 5) on the headline workload, with the construction's homo and lumo
    eigenvalues as inner bounds and outer bounds `slack` beyond them: time-to-D, error, and the
    forward square's roofline from a forward-only handle on the same schedule."""
    import numpy as np
    import torch
    from paper_1507_02087_gb300 import sp2
    N = F.shape[0]
    lam = np.sort(np.asarray(lam))
    homo, lumo = float(lam[nocc - 1]), float(lam[nocc])
    bounds = (homo - slack, homo, lumo, lumo + slack)
    stream = torch.cuda.current_stream()
    D = torch.empty_like(F)
    with sp2.Purifier(N, nocc, a.precision) as P:
        P.set_homo_lumo(bounds)
        for _ in range(warmup):
            P.run(F, D, stream)
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        tms = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.run(F, D, stream)
            e1.record(stream)
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
        clocks = clk.stop()
        info = P.info()
    err = float(torch.linalg.norm(D - D_exact)) / math.sqrt(nocc)
    del D
    with sp2.Purifier(N, nocc, a.precision, corrections=0, refine_steps=0) as Pf:
        Pf.set_homo_lumo(bounds)
        D2 = torch.empty_like(F)
        Pf.run(F, D2, stream)
        Pf.run(F, D2, stream)
        fi = Pf.info()
        del D2
    kern_ms = fi["loop_ms"] / fi["hist_len"]
    peak, _ = tensor_peak(a.precision)
    achieved = SPLIT_BASIS * N * N * (N + 1) / (kern_ms * 1e-3) / 1e12
    return {"workload": workload_name(N, nocc, a.gap) + ", SP2-ACC with homo/lumo bounds (slack %g)" % slack,
            "precision": a.precision, "time_to_d_ms": statistics.mean(tms), "steps": steps, "warmup": warmup,
            "err_vs_exact": err, "meets_tolerance": bool(err <= TOL and info["status"] == 0),
            "n_iter": info["n_iter"], "stop_reason": info["stop_reason"],
            "roofline": {"bound": "tensor", "kernel": "forward square of the accelerated expansion",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "ms_per_launch": kern_ms, "basis": "N^2 (N+1) x 3 split products per square",
                         "traffic": None},
            "clocks": clocks}


if __name__ == "__main__":
    main()

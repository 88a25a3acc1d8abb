"""Parity of the tensor-core path (squares, correction, refinement) with the CPU oracle,
through the C ABI, in its FP32-grade precision modes: bf16x6 (three bf16 pieces, six piece
products), fp16x3 (two scaled fp16 pieces, three piece products) and tf32x3 (two tf32 pieces,
three piece products on kind::tf32 tensor cores).

Tolerance: ||D - D_ref||_F / sqrt(nocc) <= 1e-6 against the FP64 oracle.

Stop: the low-precision expansion must detect its own rounding floor with the paper's
parameterless test.  The oracle that models it keeps every iterate as FP32 values (Alg. 1's
E_i = the storage rounding) and takes Tr[X_i] from ||X~_{i-1}||_F^2 as the tensor-core path
does; its products stay FP64.  The tensor cores' products add their own rounding (FP32
accumulation of N terms in 64-term chunks), which raises the floor of v_i above the storage
floor (measured: 1.7e-6 against 3.0e-7 at N = 300); v_i falls quadratically over each
alternating pair (v_i ~ C v_{i-2}^2), so a higher floor is met at most one pair (two squares)
earlier.  At the floor every stop condition compares rounding-level values: the trace choice
there can delay the alternation the order test needs, and the trace guard's own condition (the
order estimate over the last pair below q~) becomes certain only once v_{i-3} has reached the
floor too, up to two squares after v did, on either side.  An iterate that becomes exactly
idempotent (v = 0, as tf32x3 reaches on the 2 x 2 input) keeps its polynomial, and the stop
then waits for the guard's order condition on v_{i-3} = 0: three squares, which can be one
square after the FP64 oracle, whose iterate keeps a rounding-level v > 0 and stops by the order
test.  Window: n32 - 3 <= n <= n32 + 3; never after the FP64 oracle's stop, or one square after
it once the run's own history holds v = 0.  Measured over 21 dense inputs (N = 2 .. 3000), every
FP32-grade mode and both tile kinds: bf16x6 and fp16x3 -3 .. +2, tf32x3 -3 .. +1 and +3 on N = 2
(13 squares against the FP64 oracle's 12); every other run at or before the FP64 stop.
"""
import math

import numpy as np
import pytest
import torch

from oracle import sp2_oracle as o
from paper_1507_02087_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-6
FP32_GRADE = ["bf16x6", "fp16x3", "tf32x3"]


@pytest.fixture(scope="module")
def sp2mod():
    from paper_1507_02087_gb300 import sp2
    sp2.lib()
    return sp2


def assert_stop(n, F, nocc, bounds=None, ref=None, v=None):
    """The stopping iteration against the FP32-storage oracle (window in the module notes).

    v is the run's own history of v_i; a run whose iterate became exactly idempotent (some
    v_i = 0) may stop one square after the FP64 oracle, every other run at or before it."""
    F = F.cpu().numpy() if isinstance(F, torch.Tensor) else np.asarray(F)
    ref32 = o.sp2(F, nocc, storage="fp32", trace="fro", bounds=bounds)
    ref = ref if ref is not None else o.sp2(F, nocc, bounds=bounds)
    assert ref32.n - 3 <= n <= ref32.n + 3, (n, ref32.n)
    exact = v is not None and bool(np.any(np.asarray(v)[:n + 1] == 0.0))
    assert n <= ref.n + (1 if exact else 0), (n, ref.n, exact)


def run_gpu(sp2mod, F, nocc, prec="bf16x6", **opts):
    F = F if isinstance(F, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(F))
    F = F.to("cuda", torch.float64).contiguous()
    with sp2mod.Purifier(F.shape[0], nocc, prec, **opts) as P:
        D = P.run(F)
        info = P.info()
    return D, info


@pytest.mark.parametrize("prec", FP32_GRADE)
@pytest.mark.parametrize("N,nocc,gap", [(2, 1, 0.2), (17, 9, 0.1), (129, 64, 0.1), (300, 120, 0.05),
                                         (1500, 700, 0.02)])
def test_mixed_small_and_ragged(sp2mod, N, nocc, gap, prec):
    case = inputs.dense_gapped(N, nocc, gap=gap, seed=N)
    F = case.F.numpy()
    ref = o.sp2(F, nocc)
    D, info = run_gpu(sp2mod, F, nocc, prec)
    assert info["status"] == 0
    assert info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    assert_stop(info["n_iter"], F, nocc, ref=ref, v=info["v"])
    assert o.rel_error(D.cpu().numpy(), ref.D, nocc) <= TOL_MIXED
    assert torch.equal(D, D.T)


@pytest.mark.parametrize("prec", FP32_GRADE)
@pytest.mark.parametrize("N,nocc,gap,seed", [(600, 300, 0.05, 3), (1000, 500, 0.02, 5)])
def test_stop_window_edges(sp2mod, N, nocc, gap, seed, prec):
    # the two inputs at the edges of the measured window: N = 600 stops two squares after the
    # FP32-storage oracle, N = 1000 three before it (where the oracle stops by the trace guard)
    case = inputs.dense_gapped(N, nocc, gap=gap, seed=seed)
    F = case.F.numpy()
    ref = o.sp2(F, nocc)
    D, info = run_gpu(sp2mod, F, nocc, prec)
    assert info["status"] == 0 and info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    assert_stop(info["n_iter"], F, nocc, ref=ref, v=info["v"])
    assert o.rel_error(D.cpu().numpy(), ref.D, nocc) <= TOL_MIXED


@pytest.mark.parametrize("prec", FP32_GRADE)
def test_mixed_n400(sp2mod, prec):
    case = inputs.dense_n400()
    ref = o.sp2(case.F.numpy(), case.nocc)
    D, info = run_gpu(sp2mod, case.F, case.nocc, prec)
    assert info["status"] == 0
    assert_stop(info["n_iter"], case.F, case.nocc, ref=ref, v=info["v"])
    assert o.rel_error(D.cpu().numpy(), ref.D, case.nocc) <= TOL_MIXED
    inv = o.invariants(case.F.numpy(), D.cpu().numpy(), case.nocc)
    assert inv["trace_err"] < 1e-3 and inv["idem_err"] < 1e-4 and inv["comm_err"] < 1e-4


@pytest.mark.parametrize("prec", FP32_GRADE)
def test_mixed_n2048_small_gap(sp2mod, prec):
    case = inputs.dense_gapped(2048, 1024, gap=0.01, seed=0)
    ref = o.sp2(case.F.numpy(), 1024)
    D, info = run_gpu(sp2mod, case.F, 1024, prec)
    assert info["status"] == 0
    assert_stop(info["n_iter"], case.F, 1024, ref=ref, v=info["v"])
    assert o.rel_error(D.cpu().numpy(), ref.D, 1024) <= TOL_MIXED


@pytest.mark.parametrize("N,nocc,gap", [(129, 64, 0.1), (700, 350, 0.02), (2048, 1024, 0.01)])
def test_bf16x3_comparison_mode(sp2mod, N, nocc, gap):
    # two bf16 pieces, three products: about 16 significant bits per product.  A CPU emulation of
    # the same arithmetic (exact piece products, FP32 sums) gives ~7e-6 after the correction and
    # the refinement pair, so this mode misses 1e-6 by design; it stays within 3e-5.  Its products'
    # rounding is ~2^8 above FP32's, which moves the detected floor up to two alternating pairs
    # (four squares) before the FP32-storage floor; the rounding-decided conditions at the floor
    # (module notes) can add one square after it (measured over 21 inputs: -2 .. +1).
    case = inputs.dense_gapped(N, nocc, gap=gap, seed=N)
    F = case.F.numpy()
    ref = o.sp2(F, nocc)
    ref32 = o.sp2(F, nocc, storage="fp32", trace="fro")
    D, info = run_gpu(sp2mod, F, nocc, "bf16x3")
    assert info["status"] == 0 and info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    assert ref32.n - 4 <= info["n_iter"] <= ref32.n + 1
    err = o.rel_error(D.cpu().numpy(), ref.D, nocc)
    assert 1e-6 < err <= 3e-5


@pytest.mark.parametrize("prec", FP32_GRADE)
def test_mixed_options(sp2mod, prec):
    case = inputs.dense_gapped(600, 300, gap=0.05, seed=3)
    ref = o.sp2(case.F.numpy(), 300)
    errs = {}
    for key, opts in {"none": dict(corrections=0, refine_steps=0),
                      "tc": dict(corrections=0, refine_steps=2),
                      "corr+tc": dict(corrections=1, refine_steps=2),
                      "corr+fp64": dict(corrections=1, refine_steps=2, refine_fp64=1),
                      "corr+mcw": dict(corrections=1, refine_steps=2, refine_fp64=2)}.items():
        D, info = run_gpu(sp2mod, case.F, 300, prec, **opts)
        assert info["status"] == 0
        errs[key] = o.rel_error(D.cpu().numpy(), ref.D, 300)
    # The refinement pair removes eigenvalue error but not subspace error; with it in
    # place, the correction must remove most of the low-precision subspace error.
    assert errs["corr+tc"] < errs["tc"] / 3
    assert errs["corr+tc"] <= TOL_MIXED and errs["corr+fp64"] <= TOL_MIXED and errs["corr+mcw"] <= TOL_MIXED


@pytest.mark.parametrize("prec", FP32_GRADE)
@pytest.mark.parametrize("refine", [1, 2])
def test_fp64_refinements_with_padded_ld(sp2mod, refine, prec):
    # N = 600 on CTA-pair tiles: ld = 768, not N rounded to 64; the FP64 buffers must use it.
    # refine 1: the pair in FP64; refine 2: one McWeeny step, its square in FP64
    case = inputs.dense_gapped(600, 300, gap=0.05, seed=3)
    ref = o.sp2(case.F.numpy(), 300)
    D, info = run_gpu(sp2mod, case.F, 300, prec, tile="pair", refine_fp64=refine)
    assert info["status"] == 0 and info["tile"] == "pair"
    assert o.rel_error(D.cpu().numpy(), ref.D, 300) <= TOL_MIXED
    inv = o.invariants(case.F.numpy(), D.cpu().numpy(), 300)
    # the FP64 steps square the eigenvalue error e of the corrected D (~4e^2 for the pair,
    # ~3e^2 for McWeeny, e ~ 1e-4 here): far below the FP32 floor, not at FP64 rounding
    assert inv["idem_err"] < 1e-6 and inv["trace_err"] < 1e-6


@pytest.mark.parametrize("prec", FP32_GRADE)
@pytest.mark.parametrize("N,nocc,tile", [(1500, 700, "128"), (1500, 700, "pair"), (700, 350, "pair")])
def test_mixed_tile_kinds(sp2mod, N, nocc, tile, prec):
    # 128 x 128 tiles per SM and 256 x 256 tiles per SM pair (N = 700: ld rounded to 768)
    case = inputs.dense_gapped(N, nocc, gap=0.02, seed=21)
    ref = o.sp2(case.F.numpy(), nocc)
    D, info = run_gpu(sp2mod, case.F, nocc, prec, tile=tile)
    assert info["status"] == 0
    assert_stop(info["n_iter"], case.F, nocc, ref=ref, v=info["v"])
    assert o.rel_error(D.cpu().numpy(), ref.D, nocc) <= TOL_MIXED
    assert torch.equal(D, D.T)


@pytest.mark.parametrize("prec", FP32_GRADE)
def test_batch_with_pair_tiles(sp2mod, prec):
    # every ld a multiple of 256: the batch runs on CTA-pair tiles
    Ns, noccs = [256, 512, 1024, 768], [100, 256, 500, 300]
    cases = [inputs.dense_gapped(n, k, gap=0.05, seed=40 + n) for n, k in zip(Ns, noccs)]
    with sp2mod.BatchPurifier(Ns, noccs, prec, tile="pair") as B:
        Ds = B.run([c.F.cuda() for c in cases])
        infos = [B.info(i) for i in range(len(Ns))]
    for c, k, D, info in zip(cases, noccs, Ds, infos):
        ref = o.sp2(c.F.numpy(), k)
        assert info["status"] == 0
        assert_stop(info["n_iter"], c.F, k, ref=ref, v=info["v"])
        assert o.rel_error(D.cpu().numpy(), ref.D, k) <= TOL_MIXED


@pytest.mark.parametrize("prec", FP32_GRADE)
def test_recompute_history_is_bit_identical(sp2mod, prec):
    # low-memory layout: the derivative pass recomputes the iterates instead of reading
    # them back; the kernels are deterministic, so D must not change by a bit
    case = inputs.dense_gapped(900, 400, gap=0.02, seed=13)
    F = case.F.cuda()
    out = {}
    for hist in ("full", "recompute"):
        with sp2mod.Purifier(900, 400, prec, history=hist, tile="pair") as P:
            out[hist] = (P.run(F), P.info()["n_iter"])
    assert out["full"][1] == out["recompute"][1]
    assert torch.equal(out["full"][0], out["recompute"][0])


@pytest.mark.parametrize("prec", FP32_GRADE)
def test_mixed_deterministic_and_host_entry(sp2mod, prec):
    case = inputs.dense_gapped(700, 350, gap=0.05, seed=8)
    F = case.F.numpy()
    with sp2mod.Purifier(700, 350, prec) as P:
        D1 = P.run(torch.from_numpy(F).cuda()).cpu().numpy()
        D2 = P.run_host(F)
        D3 = P.run(torch.from_numpy(F).cuda()).cpu().numpy()
        info = P.info()
    assert info["status"] == 0
    assert np.array_equal(D1, D2) and np.array_equal(D1, D3)


@pytest.mark.parametrize("prec", FP32_GRADE)
def test_mixed_special_cases(sp2mod, prec):
    F = np.diag([0.3, -0.2, 0.1, 0.7])
    D, info = run_gpu(sp2mod, F, 0, prec)
    assert info["stop_reason"] == o.STOP_EXACT and float(D.abs().max()) == 0.0
    D, info = run_gpu(sp2mod, F, 4, prec)
    assert torch.equal(D.cpu(), torch.eye(4, dtype=torch.float64))
    D, info = run_gpu(sp2mod, np.array([[0.5]]), 1, prec)
    assert float(D[0, 0]) == 1.0
    F = inputs.dense_gapped(64, 32, gap=0.1, seed=2).F.numpy().copy()
    F[1, 2] = F[2, 1] = np.nan
    D, info = run_gpu(sp2mod, F, 32, prec)
    assert info["status"] == 3 and bool(torch.isnan(D).all())
    D, info = run_gpu(sp2mod, 3.0 * np.eye(16), 8, prec)
    assert info["status"] == 6


@pytest.mark.parametrize("prec", FP32_GRADE)
def test_mixed_diagonal_f(sp2mod, prec):
    g = np.random.Generator(np.random.PCG64(4))
    N, nocc = 200, 77
    lam = np.concatenate([g.uniform(-1, -0.05, nocc), g.uniform(0.05, 1.0, N - nocc)])
    g.shuffle(lam)
    D, info = run_gpu(sp2mod, np.diag(lam), nocc, prec)
    exact = np.diag((lam < 0).astype(float))
    assert o.rel_error(D.cpu().numpy(), exact, nocc) <= TOL_MIXED


@pytest.mark.parametrize("prec", FP32_GRADE)
def test_mixed_full_size_n8192(sp2mod, prec):
    # the benchmark workload, in the launch configuration the benchmark times
    case = inputs.dense_n8192(device="cuda")
    D, info = run_gpu(sp2mod, case.F, case.nocc, prec)
    assert info["status"] == 0
    err = float(torch.linalg.norm(D - case.D_exact)) / math.sqrt(case.nocc)
    assert err <= TOL_MIXED
    # invariants at full size: trace, idempotency, commutation with F
    assert abs(float(torch.trace(D)) - case.nocc) < 1e-2
    DD = D @ D
    assert float(torch.linalg.norm(DD - D)) / math.sqrt(case.nocc) < 1e-5
    FD = case.F @ D
    assert float(torch.linalg.norm(FD - FD.T)) / math.sqrt(case.nocc) < 1e-5


@pytest.mark.parametrize("prec", FP32_GRADE)
def test_mixed_full_size_n32768_householder(sp2mod, prec):
    # the dense N = 32768 workload (Q from 64 Householder reflectors, gap 1e-3, kappa ~ 2e3) with
    # the FP64-square McWeeny refinement, against the exact projector the construction fixes
    case = inputs.householder_n32768(device="cuda")
    with sp2mod.Purifier(32768, 16384, prec, refine_fp64=2) as P:
        D = P.run(case.F)
        info = P.info()
    assert info["status"] == 0
    assert info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    err = float(torch.linalg.norm(D - case.D_exact)) / math.sqrt(case.nocc)
    assert err <= TOL_MIXED
    assert torch.equal(D, D.T)


def test_mixed_caller_bounds_save_squares(sp2mod):
    # tight outer bounds (the construction's extreme eigenvalues, widened a little) in place of
    # the Gershgorin bounds, which are about sqrt(N) too loose here: fewer squares, same accuracy
    case = inputs.dense_gapped(1024, 500, gap=0.02, seed=31)
    lam = np.sort(case.lam)
    tight = (float(lam[0]) - 1e-3, float(lam[-1]) + 1e-3)
    ref = o.sp2(case.F.numpy(), 500, bounds=tight)
    F = case.F.cuda()
    with sp2mod.Purifier(1024, 500, "fp16x3") as P:
        P.run(F)
        n_gersh = P.info()["n_iter"]
        P.set_bounds(tight)
        D = P.run(F).cpu().numpy()
        info = P.info()
        P.set_bounds(None)
        P.run(F)
        assert P.info()["n_iter"] == n_gersh
    assert (info["lambda_min"], info["lambda_max"]) == tight
    assert info["status"] == 0 and info["n_iter"] < n_gersh
    assert_stop(info["n_iter"], case.F, 500, bounds=tight, ref=ref, v=info["v"])
    assert o.rel_error(D, ref.D, 500) <= TOL_MIXED
    # batches: per problem, the others keep their Gershgorin bounds
    cases = [inputs.dense_gapped(N, k, gap=0.05, seed=s) for N, k, s in [(256, 100, 1), (512, 250, 2)]]
    with sp2mod.BatchPurifier([c.N for c in cases], [c.nocc for c in cases], "mixed") as B:
        lam1 = np.sort(cases[1].lam)
        B.set_bounds(1, (float(lam1[0]) - 1e-3, float(lam1[-1]) + 1e-3))
        Ds = B.run([c.F.cuda() for c in cases])
        infos = [B.info(i) for i in range(2)]
    assert infos[1]["lambda_max"] == float(lam1[-1]) + 1e-3
    assert infos[0]["lambda_max"] == pytest.approx(o.gershgorin_bounds(cases[0].F.numpy())[1], rel=1e-12)
    for c, D, inf in zip(cases, Ds, infos):
        assert inf["status"] == 0
        assert o.rel_error(D.cpu().numpy(), o.sp2(c.F.numpy(), c.nocc).D, c.nocc) <= TOL_MIXED


def test_no_gap_at_the_fermi_level_ends_without_hanging(sp2mod):
    # Fermi-level-degenerate F (eigenvalues nocc - 1 and nocc both 0): the tensor-core path ends
    # by a stop rule within the cap, status ok; the other 62 eigenvalues converge
    g = inputs.rng(5)
    lam = np.concatenate([g.uniform(-1, -0.05, 31), [0.0, 0.0], g.uniform(0.05, 1, 31)])
    case = inputs.dense_from_spectrum(lam, 32, seed=5)
    for prec in FP32_GRADE:
        D, info = run_gpu(sp2mod, case.F, 32, prec, max_iter=60)
        assert info["status"] == 0 and info["n_iter"] <= 60
        assert info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD, o.STOP_CAP)
        w = np.linalg.eigvalsh(D.cpu().numpy())
        assert np.count_nonzero((w > 1e-3) & (w < 1 - 1e-3)) <= 2

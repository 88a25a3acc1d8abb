"""SP2-ACC (homo/lumo-based accelerated expansion, Alg. 4 and Alg. 5) on the GPU through
the C ABI, against the CPU oracle of the same algorithm.

The oracle is given the GPU's Gershgorin bounds, so both sides compute the Alg. 4 schedule
from identical inputs with the same correctly rounded operations: the polynomial sequence
must agree exactly.  Tolerances are those of the plain path: 1e-10 (FP64), 1e-6 (mixed).
"""
import numpy as np
import pytest
import torch

from oracle import sp2_oracle as o
from oracle import sp2acc_oracle as oa
from paper_1507_02087_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_FP64, TOL_MIXED = 1e-10, 1e-6


@pytest.fixture(scope="module")
def sp2mod():
    from paper_1507_02087_gb300 import sp2
    sp2.lib()
    return sp2


def homo_lumo(case, slack):
    lam = np.sort(case.lam)
    homo, lumo = float(lam[case.nocc - 1]), float(lam[case.nocc])
    return (homo - slack, homo, lumo, lumo + slack)


def run(sp2mod, case, precision, bounds, **opts):
    with sp2mod.Purifier(case.N, case.nocc, precision, **opts) as P:
        P.set_homo_lumo(bounds)
        D = P.run(case.F.cuda())
        info = P.info()
    return D.cpu().numpy(), info


@pytest.mark.parametrize("N,nocc,gap,seed", [(17, 9, 0.1, 1), (129, 64, 0.05, 2), (400, 200, 0.1, 0),
                                             (700, 300, 0.01, 3)])
def test_fp64_acc_matches_oracle(sp2mod, N, nocc, gap, seed):
    case = inputs.dense_gapped(N, nocc, gap=gap, seed=seed)
    bounds = homo_lumo(case, 1e-3)
    D, info = run(sp2mod, case, "fp64", bounds)
    assert info["status"] == 0
    ref = oa.sp2_acc(case.F.numpy(), nocc, *bounds, bounds=(info["lambda_min"], info["lambda_max"]))
    # the stop compares v_i at the rounding floor: the iteration may differ by one
    assert abs(info["n_iter"] - ref.n) <= 1
    m = min(info["n_iter"], ref.n)
    assert list(info["p"][1:m + 1]) == ref.p[1:m + 1]          # the schedule, step by step
    assert o.rel_error(D, ref.D, nocc) <= TOL_FP64
    # fewer squares than the trace-based expansion on the same input
    plain = o.sp2(case.F.numpy(), nocc, bounds=(info["lambda_min"], info["lambda_max"]))
    assert info["n_iter"] < plain.n


@pytest.mark.parametrize("prec", ["bf16x6", "fp16x3", "tf32x3"])
@pytest.mark.parametrize("N,nocc,gap,seed,slack", [(1500, 700, 0.02, 5, 1e-3), (700, 300, 0.01, 3, 1e-3),
                                                   (129, 64, 0.05, 2, 1e-3)])
def test_mixed_acc_matches_oracle(sp2mod, N, nocc, gap, seed, slack, prec):
    # the stop against the SP2-ACC oracle that keeps its iterates as FP32 values, with the window
    # of the plain mixed path (tests/test_gpu_mixed.py: the tensor-core products raise the floor of
    # v_i above the storage floor, met at most one alternating pair earlier): n32 - 2 <= n <= n32 + 1
    case = inputs.dense_gapped(N, nocc, gap=gap, seed=seed)
    bounds = homo_lumo(case, slack)
    D, info = run(sp2mod, case, prec, bounds)
    assert info["status"] == 0
    lb = (info["lambda_min"], info["lambda_max"])
    ref = oa.sp2_acc(case.F.numpy(), nocc, *bounds, bounds=lb)
    ref32 = oa.sp2_acc(case.F.numpy(), nocc, *bounds, bounds=lb, storage="fp32")
    assert ref32.n - 2 <= info["n_iter"] <= ref32.n + 1 and info["n_iter"] <= ref.n
    m = min(info["n_iter"], ref.n)
    assert list(info["p"][1:m + 1]) == ref.p[1:m + 1]
    assert o.rel_error(D, ref.D, nocc) <= TOL_MIXED


def test_mixed_acc_full_size_subset(sp2mod):
    # the bench's construction at N = 4096: accelerated and plain mixed runs both meet the bound
    case = inputs.dense_gapped(4096, 2048, gap=0.01, seed=0, device="cuda")
    bounds = homo_lumo(case, 1e-4)
    with sp2mod.Purifier(4096, 2048, "mixed") as P:
        Dp = P.run(case.F)
        n_plain = P.info()["n_iter"]
        P.set_homo_lumo(bounds)
        Da = P.run(case.F)
        ia = P.info()
    for D in (Dp, Da):
        err = float(torch.linalg.norm(D - case.D_exact)) / np.sqrt(2048)
        assert err <= TOL_MIXED
    assert ia["status"] == 0 and ia["n_iter"] < n_plain


def test_acc_on_diagonal_f_matches_scalar_map(sp2mod):
    g = np.random.Generator(np.random.PCG64(7))
    N, nocc = 200, 80
    lam = np.concatenate([g.uniform(-1, -0.03, nocc), g.uniform(0.03, 1.0, N - nocc)])
    g.shuffle(lam)
    homo, lumo = float(np.max(lam[lam < 0])), float(np.min(lam[lam > 0]))
    bounds = (homo - 1e-3, homo, lumo, lumo + 1e-3)
    with sp2mod.Purifier(N, nocc, "fp64") as P:
        P.set_homo_lumo(bounds)
        D = P.run(torch.from_numpy(np.diag(lam)).cuda()).cpu().numpy()
        info = P.info()
    sched = oa.acc_schedule(info["lambda_min"], info["lambda_max"], *bounds)
    xs, n, reason, p = oa.sp2_acc_scalar(lam, nocc, info["lambda_min"], info["lambda_max"], sched)
    # the GPU forms a x^2 + b x + c, the scalar map ((1 - a) + a x)^2: equal up to rounding,
    # so the floor-level stop may move by one step
    assert abs(info["n_iter"] - n) <= 1
    assert float(np.max(np.abs(np.diag(D) - np.array(xs)))) < 1e-12
    assert np.array_equal(np.diag(D) > 0.5, lam < 0)


def test_set_homo_lumo_arguments_and_reset(sp2mod):
    case = inputs.dense_gapped(300, 150, gap=0.05, seed=11)
    F = case.F.cuda()
    with sp2mod.Purifier(300, 150, "fp64") as P:
        D0 = P.run(F)
        n0 = P.info()["n_iter"]
        for bad in [(0.1, 0.0, 0.2, 0.3), (-0.1, 0.0, 0.0, 0.3), (float("nan"), 0.0, 0.1, 0.2)]:
            with pytest.raises(sp2mod.SP2Error):
                P.set_homo_lumo(bad)
        P.set_homo_lumo(homo_lumo(case, 1e-3))
        P.run(F)
        assert P.info()["n_iter"] < n0
        P.set_homo_lumo(None)                     # back to the trace-based expansion
        D1 = P.run(F)
        assert P.info()["n_iter"] == n0 and torch.equal(D0, D1)


def test_batch_acc_per_problem(sp2mod):
    cases = [inputs.dense_gapped(N, k, gap=g, seed=s) for N, k, g, s in
             [(256, 100, 0.05, 1), (300, 150, 0.02, 2), (520, 260, 0.03, 3)]]
    with sp2mod.BatchPurifier([c.N for c in cases], [c.nocc for c in cases], "mixed") as B:
        B.set_homo_lumo(1, homo_lumo(cases[1], 1e-3))     # only the middle problem accelerated
        Ds = B.run([c.F.cuda() for c in cases])
        infos = [B.info(i) for i in range(3)]
    for c, D, info in zip(cases, Ds, infos):
        assert info["status"] == 0
        assert o.rel_error(D.cpu().numpy(), o.sp2(c.F.numpy(), c.nocc).D, c.nocc) <= TOL_MIXED
    plain1 = o.sp2(cases[1].F.numpy(), cases[1].nocc)
    assert infos[1]["n_iter"] < plain1.n

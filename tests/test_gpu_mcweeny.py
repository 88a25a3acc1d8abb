"""The McWeeny expansion and McW-ACC (§3) on the FP64 path, through the C ABI, against the
CPU oracle of the same algorithms (tolerance of the FP64 path: 1e-10)."""
import numpy as np
import pytest
import torch

from oracle import mcweeny_oracle as om
from oracle import sp2_oracle as o
from paper_1507_02087_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp2mod():
    from paper_1507_02087_gb300 import sp2
    sp2.lib()
    return sp2


def run(sp2mod, case, mode, xi=0.0, **opts):
    with sp2mod.Purifier(case.N, case.nocc, "fp64", **opts) as P:
        P.set_mcweeny(mode, 0.0, xi)
        D = P.run(case.F.cuda())
        info = P.info()
    return D.cpu().numpy(), info


@pytest.mark.parametrize("mode,xi", [("mcw", 0.0), ("mcw-acc", 0.02)])
@pytest.mark.parametrize("N,nocc,seed", [(33, 15, 1), (300, 150, 2)])
def test_mcweeny_matches_oracle(sp2mod, mode, xi, N, nocc, seed):
    # the spectrum of dense_gapped is split at 0, so mu = 0 is in the gap
    case = inputs.dense_gapped(N, nocc, gap=0.05, seed=seed)
    D, info = run(sp2mod, case, mode, xi)
    assert info["status"] == 0 and info["stop_reason"] == o.STOP_ORDER
    ref = om.mcweeny(case.F.numpy(), 0.0, xi=xi, accelerate=(mode == "mcw-acc"),
                     bounds=(info["lambda_min"], info["lambda_max"]))
    assert abs(info["n_iter"] - ref.n) <= 1
    assert o.rel_error(D, ref.D, nocc) <= 1e-10
    assert o.rel_error(D, o.sp2(case.F.numpy(), nocc).D, nocc) <= 1e-10
    for i in range(min(info["hist_len"], len(ref.v))):
        if ref.v[i] > 1e-8:
            assert info["v"][i] == pytest.approx(ref.v[i], rel=1e-8)


def test_mcw_acc_saves_steps_and_modes_agree(sp2mod):
    case = inputs.dense_gapped(400, 200, gap=0.01, seed=4)
    _, i_plain = run(sp2mod, case, "mcw")
    Dg, i_acc = run(sp2mod, case, "mcw-acc", 0.01)
    Dp, i_acc1 = run(sp2mod, case, "mcw-acc", 0.01, launch_mode=1)
    assert i_acc["n_iter"] < i_plain["n_iter"]
    assert i_acc1["n_iter"] == i_acc["n_iter"] and np.array_equal(Dg, Dp)


def test_mcweeny_switch_and_errors(sp2mod):
    case = inputs.dense_gapped(200, 100, gap=0.05, seed=5)
    F = case.F.cuda()
    with sp2mod.Purifier(200, 100, "fp64") as P:
        D0 = P.run(F)
        n0 = P.info()["n_iter"]
        with pytest.raises(sp2mod.SP2Error):
            P.set_mcweeny("mcw-acc", 0.0, 0.0)          # McW-ACC needs a gap estimate
        P.set_mcweeny("mcw", 0.0)
        P.run(F)
        P.set_mcweeny(None)                            # back to SP2: the same result
        D1 = P.run(F)
        assert P.info()["n_iter"] == n0 and torch.equal(D0, D1)
    with sp2mod.Purifier(200, 100, "mixed") as P:
        with pytest.raises(sp2mod.SP2Error):
            P.set_mcweeny("mcw", 0.0)

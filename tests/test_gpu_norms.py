"""The mixed-norm stop (§2: spectral norm of the matrix of block Frobenius norms of X - X^2)
on the GPU through the C ABI, against the oracle's mixed norm with the same block size
(64 on the FP64 path, the 128 x 128 tiles on the mixed path)."""
import math

import numpy as np
import pytest

from oracle import sp2_oracle as o
from paper_1507_02087_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp2mod():
    from paper_1507_02087_gb300 import sp2
    sp2.lib()
    return sp2


def run(sp2mod, case, precision, **opts):
    with sp2mod.Purifier(case.N, case.nocc, precision, **opts) as P:
        D = P.run(case.F.cuda())
        info = P.info()
    return D.cpu().numpy(), info


@pytest.mark.parametrize("N,nocc,seed", [(200, 90, 1), (640, 320, 2)])
def test_fp64_mixed_norm_stop(sp2mod, N, nocc, seed):
    case = inputs.dense_gapped(N, nocc, gap=0.05, seed=seed)
    D, info = run(sp2mod, case, "fp64", norm="mixed")
    assert info["status"] == 0
    ref = o.sp2(case.F.numpy(), nocc, norm="mixed", block=64, bounds=(info["lambda_min"], info["lambda_max"]))
    assert abs(info["n_iter"] - ref.n) <= 1
    assert o.rel_error(D, ref.D, nocc) <= 1e-10
    # the recorded measure is m_i: equal to the oracle's before the rounding floor
    for i in range(min(len(ref.v), info["hist_len"])):
        if ref.v[i] > 1e-8:
            assert info["v"][i] == pytest.approx(ref.v[i], rel=1e-7)


@pytest.mark.parametrize("tile", ["128", "pair"])
def test_tc_mixed_norm_stop(sp2mod, tile):
    case = inputs.dense_gapped(1024, 500, gap=0.02, seed=6)
    Dm, im = run(sp2mod, case, "mixed", norm="mixed", tile=tile)
    Df, iff = run(sp2mod, case, "mixed", tile=tile)
    assert im["status"] == 0 and iff["status"] == 0
    ref = o.sp2(case.F.numpy(), 500)
    assert o.rel_error(Dm, ref.D, 500) <= 1e-6
    # same iterates, different measure: v / sqrt(nb) <= m <= v at every recorded step
    nb = 1024 // 128
    k = min(im["hist_len"], iff["hist_len"])
    for i in range(k):
        m, v = im["v"][i], iff["v"][i]
        assert m <= v * (1 + 1e-9) and m >= v / math.sqrt(nb) * (1 - 1e-9)
    # and the block bookkeeping gives the oracle's mixed norm: compared on the first iterates,
    # before the FP32 iterates drift from the FP64 ones (rounding amplified up to 2x per step:
    # 1e-4 relative by the tenth step, 1e-3 by the twentieth)
    refm = o.sp2(case.F.numpy(), 500, norm="mixed", block=128, bounds=(im["lambda_min"], im["lambda_max"]))
    for i in range(3):
        assert im["v"][i] == pytest.approx(refm.v[i], rel=1e-5)


def test_batch_mixed_norm(sp2mod):
    cases = [inputs.dense_gapped(N, k, gap=0.05, seed=s) for N, k, s in [(300, 140, 1), (520, 260, 2)]]
    with sp2mod.BatchPurifier([c.N for c in cases], [c.nocc for c in cases], "mixed", norm="mixed") as B:
        Ds = B.run([c.F.cuda() for c in cases])
        infos = [B.info(i) for i in range(2)]
    for c, D, info in zip(cases, Ds, infos):
        assert info["status"] == 0
        assert o.rel_error(D.cpu().numpy(), o.sp2(c.F.numpy(), c.nocc).D, c.nocc) <= 1e-6

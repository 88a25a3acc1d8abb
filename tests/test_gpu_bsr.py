"""Block-sparse path (32 x 32 FP32 blocks, Frobenius block truncation) through the C ABI.

Index work (the truncation decision and the symbolic square) must equal the host's bit
for bit given the same stored blocks.  The purification itself is compared with the
FP64 oracle that applies the same truncation after every step: the GPU keeps FP32
blocks, so its result agrees to FP32 accuracy plus the effect of the few blocks whose
truncation decision flips between the FP32 and FP64 iterates (each of norm ~tau).
"""
import math

import numpy as np
import pytest
import torch

from oracle import bsr_oracle as bo
from oracle import sp2_oracle as o
from paper_1507_02087_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp2mod():
    from paper_1507_02087_gb300 import sp2
    sp2.lib()
    return sp2


def test_truncation_decision_bit_exact(sp2mod):
    g = np.random.Generator(np.random.PCG64(5))
    nb, b = 24, 32
    N = nb * b
    tau = 1e-4
    X = g.standard_normal((N, N)) * 1e-3
    # blocks spread around the threshold: scale each block so its norm is tau * f
    for I in range(nb):
        for J in range(nb):
            f = g.choice([0.5, 0.999999, 1.0, 1.000001, 2.0, 30.0])
            blk = X[I * b:(I + 1) * b, J * b:(J + 1) * b]
            blk *= tau * f / np.linalg.norm(blk)
    X32 = X.astype(np.float32)
    keep_gpu = torch.zeros(nb * nb, dtype=torch.uint8, device="cuda")
    rc = sp2mod.lib().sp2_test_bsr_keep(torch.from_numpy(X32).cuda().data_ptr(), N, tau, 0, keep_gpu.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    keep_ref = bo.keep_mask(X32.astype(np.float64), b, tau)
    assert np.array_equal(keep_gpu.cpu().numpy().reshape(nb, nb).astype(bool), keep_ref)
    assert 0 < keep_ref.sum() < nb * nb


def _keep_gpu(sp2mod, X32, tau, rule):
    N = X32.shape[0]
    nb = N // 32
    keep = torch.zeros(nb * nb, dtype=torch.uint8, device="cuda")
    rc = sp2mod.lib().sp2_test_bsr_keep(torch.from_numpy(np.ascontiguousarray(X32)).cuda().data_ptr(), N, tau,
                                        rule, keep.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    return keep.cpu().numpy().reshape(nb, nb).astype(bool)


@pytest.mark.parametrize("nb,seed", [(3, 1), (24, 2), (90, 3)])
def test_error_truncation_decision_bit_exact(sp2mod, nb, seed):
    # symmetric block matrix with block norms spread over many decades, exact ties
    # (repeated blocks), zero blocks, and budgets that cut inside a tie group
    g = np.random.Generator(np.random.PCG64(seed))
    b = 32
    X = np.zeros((nb * b, nb * b))
    proto = g.standard_normal((b, b))
    for I in range(nb):
        for J in range(I, nb):
            kind = g.integers(0, 4)
            if kind == 0:
                blk = g.standard_normal((b, b)) * 10.0 ** g.uniform(-9, 0)
            elif kind == 1:
                blk = proto * 1e-5                       # the same block many times: exact ties
            elif kind == 2:
                blk = np.zeros((b, b))
            else:
                blk = g.standard_normal((b, b)) * 1e-4
            if I == J:
                blk = 0.5 * (blk + blk.T) + np.eye(b)
            X[I * b:(I + 1) * b, J * b:(J + 1) * b] = blk
            X[J * b:(J + 1) * b, I * b:(I + 1) * b] = blk.T
    X32 = X.astype(np.float32)
    n2 = bo.block_norms2(X32.astype(np.float64), b)
    tie = float(np.float64(np.linalg.norm((proto * 1e-5).astype(np.float32).astype(np.float64)) ** 2))
    for tau in (0.0, 1e-7, 1e-4, 3e-3, np.sqrt(7.5 * tie), 1e3):
        keep_gpu = _keep_gpu(sp2mod, X32, tau, 1)
        keep_ref = bo.keep_mask_error(X32.astype(np.float64), b, tau)
        assert np.array_equal(keep_gpu, keep_ref), tau
        E = X32.astype(np.float64) * np.kron(~keep_ref, np.ones((b, b)))
        assert np.linalg.norm(E) <= tau * (1 + 1e-9) + 1e-300
    assert n2.size == nb * nb


@pytest.mark.parametrize("dims,tau,tol", [((32, 8, 4), 1e-6, 4e-6), ((32, 8, 8), 1e-4, 4e-6)])
def test_bsr_error_rule_against_oracle(sp2mod, dims, tau, tol):
    tb, (rp, ci, vals) = tb_case(dims)
    F = tb.dense().numpy()
    ref = bo.sp2_bsr(F, tb.nocc, 32, tau, rule="error")
    with sp2mod.BsrPurifier(tb.N, tb.nocc, tau, rule="error") as P:
        D = P.run(rp, ci, vals)
        info = P.info()
    assert info["status"] == 0
    assert info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    assert ref.n - 3 <= info["n_iter"] <= ref.n + 3
    err = o.rel_error(D.cpu().numpy(), ref.D, tb.nocc)
    assert err <= tol, err
    Dn = D.cpu().numpy()
    assert np.array_equal(Dn, Dn.T)


@pytest.mark.parametrize("nb,density", [(1, 1.0), (5, 0.4), (70, 0.08), (130, 0.03)])
def test_symbolic_square_bit_exact(sp2mod, nb, density):
    g = np.random.Generator(np.random.PCG64(nb))
    m = g.random((nb, nb)) < density
    m = m | m.T
    np.fill_diagonal(m, True)
    out = np.zeros((nb, nb), dtype=np.uint8)
    mask = np.ascontiguousarray(m.astype(np.uint8))
    rc = sp2mod.lib().sp2_test_bsr_square_pattern(mask.ctypes.data, nb, out.ctypes.data)
    assert rc == 0
    ref = np.triu(bo.square_pattern(m))
    assert np.array_equal(out.astype(bool), ref)


def tb_case(dims):
    tb = inputs.tight_binding(dims=dims)
    rp, ci, vals = tb.bsr(32)
    return tb, (torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(vals).cuda())


@pytest.mark.parametrize("dims,tau,tol", [((32, 8, 4), 0.0, 3e-6), ((32, 8, 8), 1e-6, 4e-6),
                                          ((32, 16, 8), 1e-4, 4e-6)])
def test_bsr_sp2_against_oracle(sp2mod, dims, tau, tol):
    tb, (rp, ci, vals) = tb_case(dims)
    F = tb.dense().numpy()
    ref = bo.sp2_bsr(F, tb.nocc, 32, tau)
    with sp2mod.BsrPurifier(tb.N, tb.nocc, tau) as P:
        D = P.run(rp, ci, vals)
        info = P.info()
    assert info["status"] == 0
    assert info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    # FP32 blocks reach their rounding floor at a different square than FP64: earlier,
    # or a few squares later when the trace-chosen polynomial repeats at the floor before
    # the (alternation-requiring) order test can fire
    assert ref.n - 3 <= info["n_iter"] <= ref.n + 3
    assert info["lambda_min"] == pytest.approx(ref.lmin, rel=1e-12)
    assert info["lambda_max"] == pytest.approx(ref.lmax, rel=1e-12)
    err = o.rel_error(D.cpu().numpy(), ref.D, tb.nocc)
    assert err <= tol, err
    Dn = D.cpu().numpy()
    assert np.array_equal(Dn, Dn.T)
    # the stored pattern of D is what the truncation keeps
    assert info["nnzb"] == int(np.count_nonzero(np.abs(Dn).reshape(tb.N // 32, 32, tb.N // 32, 32).sum(axis=(1, 3))))


def test_bsr_launch_modes_agree_and_errors(sp2mod):
    tb, (rp, ci, vals) = tb_case((32, 8, 4))
    out = []
    for mode in (0, 1):
        with sp2mod.BsrPurifier(tb.N, tb.nocc, 1e-5, launch_mode=mode) as P:
            out.append((P.run(rp, ci, vals), P.info()["n_iter"]))
    assert out[0][1] == out[1][1] and torch.equal(out[0][0], out[1][0])
    bad = vals.clone()
    bad[0, 1, 2] = float("nan")
    with sp2mod.BsrPurifier(tb.N, tb.nocc, 1e-5) as P:
        D = P.run(rp, ci, bad)
        assert P.info()["status"] == 3 and bool(torch.isnan(D).all())

"""Pins of the block-truncation oracle (Alg. 1 with E_i = block truncation)."""
import numpy as np
import pytest

from oracle import bsr_oracle as bo
from oracle import sp2_oracle as o
from paper_1507_02087_gb300 import inputs


def test_block_norms_against_library_norm():
    g = np.random.Generator(np.random.PCG64(1))
    X = g.standard_normal((96, 96))
    n2 = bo.block_norms2(X, 32)
    for I in range(3):
        for J in range(3):
            ref = np.linalg.norm(X[32 * I:32 * I + 32, 32 * J:32 * J + 32]) ** 2
            assert n2[I, J] == pytest.approx(ref, rel=1e-13)


def test_block_norm_order_is_rows_then_columns():
    # one block whose sum depends on the order: the documented order gives this value
    blk = np.zeros((32, 32))
    blk[0, 0], blk[0, 1], blk[1, 0] = 1.0, 2.0 ** -27, 2.0 ** -27
    rows = [0.0] * 32
    for r in range(32):
        s = 0.0
        for c in range(32):
            s += blk[r, c] * blk[r, c]
        rows[r] = s
    tot = 0.0
    for r in range(32):
        tot += rows[r]
    assert bo.block_norms2(blk, 32)[0, 0] == tot


def test_keep_mask_rules():
    g = np.random.Generator(np.random.PCG64(2))
    X = g.standard_normal((128, 128)) * 1e-6
    X = 0.5 * (X + X.T)
    X[:32, 96:] *= 1e6
    X[96:, :32] *= 1e6
    keep = bo.keep_mask(X, 32, 1e-3)
    assert np.array_equal(keep, keep.T)
    assert keep.diagonal().all()
    assert keep[0, 3] and keep[3, 0] and not keep[1, 2]
    assert bo.keep_mask(X, 32, 0.0).all()


def test_square_pattern_brute_force():
    g = np.random.Generator(np.random.PCG64(3))
    m = g.random((20, 20)) < 0.15
    m = m | m.T
    np.fill_diagonal(m, True)
    sp = bo.square_pattern(m)
    for I in range(20):
        for J in range(20):
            assert sp[I, J] == any(m[I, K] and m[K, J] for K in range(20))


def test_zero_tau_is_the_plain_expansion():
    tb = inputs.tight_binding(dims=(32, 4, 4))
    F = tb.dense().numpy()
    a = bo.sp2_bsr(F, tb.nocc, 32, 0.0)
    b = o.sp2(F, tb.nocc)
    assert a.n == b.n and np.array_equal(a.D, b.D)


def test_truncation_error_grows_with_tau():
    tb = inputs.tight_binding(dims=(32, 8, 8))
    F = tb.dense().numpy()
    w, V = np.linalg.eigh(F)
    De = V[:, :tb.nocc] @ V[:, :tb.nocc].T
    errs = [o.rel_error(bo.sp2_bsr(F, tb.nocc, 32, tau).D, De, tb.nocc) for tau in (0.0, 1e-6, 1e-4)]
    assert errs[0] < 1e-13 and errs[0] <= errs[1] < errs[2] < 1e-3

"""Pins of the block-truncation oracle (Alg. 1 with E_i = block truncation)."""
import math

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


# ---- error-controlled truncation ----------------------------------------------------------

def _blocks_with_norms(nb, b, norms2):
    """Symmetric matrix whose off-diagonal upper block (I, J) has ||X_IJ||_F^2 = norms2[(I, J)]
    exactly (one nonzero element per block, a power-of-two multiple), diagonal blocks = I."""
    X = np.zeros((nb * b, nb * b))
    for I in range(nb):
        X[I * b:(I + 1) * b, I * b:(I + 1) * b] = np.eye(b)
    for (I, J), v in norms2.items():
        x = np.sqrt(v)
        X[I * b, J * b] = X[J * b, I * b] = x
    return X


def test_error_truncation_worked_example():
    # pairs with ||X_IJ||^2 = 1, 2, 3, 4 (x 2^-30); counted twice they weigh 2, 4, 6, 8.
    # tau^2 = 6.5 x 2^-30 admits the first two (2 + 4 = 6) and not the third (12).
    c = 2.0 ** -30
    norms2 = {(0, 1): 1 * c, (0, 2): 2 * c, (1, 2): 3 * c, (2, 3): 4 * c}
    X = _blocks_with_norms(4, 32, norms2)
    keep = bo.keep_mask_error(X, 32, np.sqrt(6.5 * c))
    dropped = {(I, J) for I in range(4) for J in range(I + 1, 4) if not keep[I, J]}
    assert dropped == {(0, 1), (0, 2), (0, 3), (1, 3)}       # zero blocks weigh nothing and go first
    assert np.array_equal(keep, keep.T) and keep.diagonal().all()
    # the per-block rule at the same tau drops every pair with ||X_IJ|| < tau: all six off-diagonal
    # pairs (1, 2, 3, 4 x c and the two zero blocks), so ||E||_F^2 = 20 c > tau^2
    kb = bo.keep_mask(X, 32, np.sqrt(6.5 * c))
    assert int((~kb).sum()) // 2 == 6


def test_error_truncation_ties_broken_by_index():
    c = 2.0 ** -20
    norms2 = {(0, 3): c, (1, 2): c, (0, 1): c, (2, 3): 5 * c}
    X = _blocks_with_norms(4, 32, norms2)
    keep = bo.keep_mask_error(X, 32, np.sqrt(4 * c))        # room for two of the three equal pairs
    dropped = {(I, J) for I in range(4) for J in range(I + 1, 4) if not keep[I, J]}
    assert dropped - {(0, 2), (1, 3)} == {(0, 1), (0, 3)}    # (I, J) order among equal norms
    assert not keep[0, 2] and not keep[1, 3]                 # the zero blocks


def test_error_truncation_bound_and_maximality():
    g = np.random.Generator(np.random.PCG64(11))
    nb, b = 10, 32
    X = g.standard_normal((nb * b, nb * b))
    X = 0.5 * (X + X.T)
    scale = np.exp(g.uniform(-12, 0, (nb, nb)))
    scale = np.minimum(scale, scale.T)
    X = X * np.kron(scale, np.ones((b, b)))
    for tau in (1e-3, 1e-1, 3.0):
        keep = bo.keep_mask_error(X, b, tau)
        E = X - bo.apply_mask(X, keep, b)
        e2 = np.linalg.norm(E) ** 2                          # library norm, independent of the rule's sums
        assert e2 <= tau * tau * (1 + 1e-9)
        # maximal: the smallest kept off-diagonal block would overflow the budget
        n2 = np.array([[np.linalg.norm(X[I*b:(I+1)*b, J*b:(J+1)*b]) ** 2 for J in range(nb)] for I in range(nb)])
        kept_off = [n2[I, J] for I in range(nb) for J in range(I + 1, nb) if keep[I, J]]
        if kept_off:
            assert e2 + 2 * min(kept_off) > tau * tau * (1 - 1e-9)


def test_error_truncation_edge_cases():
    g = np.random.Generator(np.random.PCG64(12))
    X = g.standard_normal((128, 128))
    X = 0.5 * (X + X.T)
    assert bo.keep_mask_error(X, 32, 0.0).all()               # tau = 0: nothing dropped
    keep = bo.keep_mask_error(X, 32, 1e6)                     # everything fits the budget
    assert keep.diagonal().all() and int(keep.sum()) == 4
    e, budget = bo.error_units(0.75)
    assert 2.0 ** e <= 0.75 ** 2 < 2.0 ** (e + 1) and budget == int(np.floor(0.5625 * 2.0 ** (40 - e)))


def test_bsr_oracle_error_rule_runs_and_bounds_each_step():
    tb = inputs.tight_binding(L=4, delta=1.0, t=0.3, sigma=0.05, seed=2, dims=(32, 2, 2))
    F = tb.dense()
    res = bo.sp2_bsr(F, tb.nocc, 32, 1e-4, rule="error")
    assert res.stop_reason in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    ref = o.sp2(F, tb.nocc)
    assert o.rel_error(res.D, ref.D, tb.nocc) < 1e-3


# ---- mixed-norm truncation (||E||_M <= tau through the block-row sums) ----------------------

def _mixed_norm_of_removed(X, keep, b):
    # library block norms and library spectral norm, independent of the rule's unit sums
    nb = X.shape[0] // b
    E = X - bo.apply_mask(X, keep, b)
    M = np.array([[np.linalg.norm(E[I*b:(I+1)*b, J*b:(J+1)*b]) for J in range(nb)] for I in range(nb)])
    return E, M


def test_mixed_truncation_worked_example():
    # pairs with ||X_IJ|| = 1, 2, 3, 4 (x 2^-20) on (0,1), (0,2), (1,2), (2,3); tau = 4.5 x 2^-20.
    # In order: the zero blocks (0,3), (1,3); then (0,1) (rows 0, 1: 1, 1), (0,2) (rows 0, 2: 3, 2);
    # (1,2) would bring row 2 to 5 > 4.5 and ends the prefix, so (2,3) stays although row 3 is empty.
    c = 2.0 ** -20
    norms2 = {(0, 1): (1 * c) ** 2, (0, 2): (2 * c) ** 2, (1, 2): (3 * c) ** 2, (2, 3): (4 * c) ** 2}
    X = _blocks_with_norms(4, 32, norms2)
    keep = bo.keep_mask_mixed(X, 32, 4.5 * c)
    dropped = {(I, J) for I in range(4) for J in range(I + 1, 4) if not keep[I, J]}
    assert dropped == {(0, 1), (0, 2), (0, 3), (1, 3)}
    assert np.array_equal(keep, keep.T) and keep.diagonal().all()
    E, M = _mixed_norm_of_removed(X, keep, 32)
    assert np.linalg.norm(M, 2) == pytest.approx(np.sqrt(5.0) * c, rel=1e-12)   # [[0,1,2],[1,0,0],[2,0,0]] c
    # the error rule with this selection's ||E||_F^2 = 2 (1 + 4) c^2 as its budget drops the same
    # blocks: both walk the same order, here only the budgets differ
    ke = bo.keep_mask_error(X, 32, np.sqrt(2 * (1 + 4) * c * c))
    assert np.array_equal(ke, keep)


def test_mixed_truncation_bound_and_maximality():
    g = np.random.Generator(np.random.PCG64(21))
    nb, b = 10, 32
    X = g.standard_normal((nb * b, nb * b))
    X = 0.5 * (X + X.T)
    scale = np.exp(g.uniform(-12, 0, (nb, nb)))
    scale = np.minimum(scale, scale.T)
    X = X * np.kron(scale, np.ones((b, b)))
    for tau in (1e-3, 1e-1, 3.0, 30.0):
        keep = bo.keep_mask_mixed(X, b, tau)
        E, M = _mixed_norm_of_removed(X, keep, b)
        mn = np.linalg.norm(M, 2)
        assert mn <= tau * (1 + 1e-9)                                  # ||E||_M <= tau
        assert np.max(np.abs(np.linalg.eigvalsh(E))) <= mn * (1 + 1e-9)  # ||E||_2 <= ||E||_M
        assert M.sum(axis=1).max() <= tau * (1 + 1e-9)                 # the row sums the rule bounds
        # maximal: the first kept candidate in (norm^2, I, J) order overflows one of its rows
        n2 = np.array([[np.linalg.norm(X[I*b:(I+1)*b, J*b:(J+1)*b]) ** 2 for J in range(nb)] for I in range(nb)])
        kept = sorted((n2[I, J], I, J) for I in range(nb) for J in range(I + 1, nb)
                      if keep[I, J] and np.sqrt(n2[I, J]) <= tau)
        if kept:
            v, I, J = kept[0]
            rs = M.sum(axis=1)
            assert max(rs[I], rs[J]) + np.sqrt(v) > tau * (1 - 1e-9)


def test_mixed_truncation_edge_cases():
    g = np.random.Generator(np.random.PCG64(22))
    X = g.standard_normal((128, 128))
    X = 0.5 * (X + X.T)
    assert bo.keep_mask_mixed(X, 32, 0.0).all()                    # tau = 0: nothing dropped
    keep = bo.keep_mask_mixed(X, 32, 1e6)                          # every row sum fits
    assert keep.diagonal().all() and int(keep.sum()) == 4
    e, budget = bo.mixed_units(0.75)
    assert 2.0 ** e <= 0.75 < 2.0 ** (e + 1) and budget == int(np.floor(0.75 * 2.0 ** (40 - e)))


def test_bsr_oracle_mixed_rule_and_mixed_norm_stop():
    # the pairing of the §6 calculations: mixed-norm truncation and the mixed-norm stop with the
    # truncation's blocks
    tb = inputs.tight_binding(L=4, delta=1.0, t=0.3, sigma=0.05, seed=2, dims=(32, 2, 2))
    F = tb.dense()
    res = bo.sp2_bsr(F, tb.nocc, 32, 1e-4, rule="mixed", norm="mixed")
    assert res.stop_reason in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    ref = o.sp2(F, tb.nocc)
    assert o.rel_error(res.D, ref.D, tb.nocc) < 1e-3
    fro = bo.sp2_bsr(F, tb.nocc, 32, 1e-4, rule="mixed")
    for i in range(min(len(res.v), len(fro.v))):                    # m_i <= v_i on the same iterates
        assert res.v[i] <= fro.v[i] * (1 + 1e-12)


def test_bsr_oracle_acc_with_truncation():
    # SP2-ACC with the block truncation (the accelerated expansion of the §6 calculations):
    # tau = 0 reproduces the untruncated SP2-ACC oracle exactly; with tau = 1e-4 the result stays
    # near the projector and takes fewer squares than the trace-based expansion
    from oracle import sp2acc_oracle as oa
    tb = inputs.tight_binding(L=4, delta=1.0, t=0.3, sigma=0.05, seed=2, dims=(32, 2, 2))
    F = tb.dense().numpy()
    lam = np.linalg.eigvalsh(F)
    homo, lumo = float(lam[tb.nocc - 1]), float(lam[tb.nocc])
    acc = (homo - 1e-2, homo, lumo, lumo + 1e-2)
    plain = oa.sp2_acc(F, tb.nocc, *acc)
    zero = bo.sp2_bsr(F, tb.nocc, 32, 0.0, rule="error", acc=acc)
    assert zero.n == plain.n and zero.p == plain.p and np.array_equal(zero.D, plain.D)
    res = bo.sp2_bsr(F, tb.nocc, 32, 1e-4, rule="error", acc=acc)
    assert res.stop_reason in (o.STOP_ORDER, o.STOP_TRACE_GUARD, oa.STOP_SCHEDULE)
    V = np.linalg.eigh(F)[1]
    exact = V[:, :tb.nocc] @ V[:, :tb.nocc].T
    assert o.rel_error(res.D, exact, tb.nocc) < 1e-3
    assert res.n < bo.sp2_bsr(F, tb.nocc, 32, 1e-4, rule="error").n


def _per_row_cut(n2, tau):
    """The per-row formulation of the mixed-norm cut, restated here from its argument (each
    row's own first overflow in key order; the cut is the earliest over the rows): returns the
    keep mask it implies, for comparison with the oracle's sequential walk."""
    nb = n2.shape[0]
    e, budget = bo.mixed_units(tau)
    cand = {}
    for I in range(nb):
        for J in range(I + 1, nb):
            w = math.sqrt(float(n2[I, J]))
            if w <= tau:
                cand[(I, J)] = ((float(n2[I, J]), I, J), int(math.floor(math.ldexp(w, 40 - e))))
    first = None
    for r in range(nb):
        mine = sorted((key, u) for (I, J), (key, u) in cand.items() if r in (I, J))
        run = 0
        for key, u in mine:
            run += u
            if run > budget:
                first = key if first is None or key < first else first
                break
    keep = np.ones((nb, nb), dtype=bool)
    for (I, J), (key, _) in cand.items():
        if first is None or key < first:
            keep[I, J] = keep[J, I] = False
    return keep


@pytest.mark.parametrize("seed", range(12))
def test_mixed_cut_per_row_equals_sequential_walk(seed):
    # random symmetric block-norm patterns with many exact ties and zero blocks
    g = np.random.Generator(np.random.PCG64(100 + seed))
    nb, b = int(g.integers(3, 14)), 32
    levels = 2.0 ** -np.arange(18, 26)
    norms2 = {}
    for I in range(nb):
        for J in range(I + 1, nb):
            kind = g.integers(0, 3)
            norms2[(I, J)] = 0.0 if kind == 0 else float(g.choice(levels)) ** 2
    X = _blocks_with_norms(nb, b, norms2)
    n2 = bo.block_norms2(X, b)
    for tau in (2.0 ** -20, 3 * 2.0 ** -21, 2.0 ** -18, 1.0):
        assert np.array_equal(bo.keep_mask_mixed(X, b, tau), _per_row_cut(n2, tau)), (seed, tau)

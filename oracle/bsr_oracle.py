"""CPU oracle for SP2 with block truncation (the E_i of Alg. 1) -- TEST INFRASTRUCTURE ONLY.

Only the tests and the benchmark's CPU-baseline leg import this module.

The recursive expansion of Alg. 1 adds a perturbation E_i to every iterate; in a
sparse setting E_i removes small parts of X_i (§1; §5 and §6 use element-magnitude
and error-controlled removal).  Here the matrix is split into b x b blocks and E_i
drops every off-diagonal block whose Frobenius norm is below tau (diagonal blocks
are always kept), applied to X_0 and after every step, on a symmetric pattern.

Reading (the paper fixes no block rule): a block is dropped iff ||X_IJ||_F^2 < tau^2,
with ||X_IJ||_F^2 evaluated in FP64 from the stored values in a fixed order: each
row's squares summed left to right, then the row sums top to bottom (each square of
an FP32 value is exact in FP64).  The GPU path evaluates the same sums in the same
order, so given the same stored block both sides take the same decision bit for bit.

Second rule, error-controlled truncation (`keep_mask_error`): the removed part E is
bounded directly, ||E||_F <= tau.  The off-diagonal blocks are ordered by
(||X_IJ||_F^2, I, J), and the longest prefix of that order whose norms, counted twice
(a symmetric pair (I, J), (J, I) is removed together), sum to at most tau^2 is dropped;
blocks with 2 ||X_IJ||_F^2 > tau^2 are never dropped.  Reading: the sum is taken in
exact integer units of 2^(e - 40), where 2^e <= tau^2 < 2^(e+1) (each 2 ||X_IJ||_F^2
rounded down to a unit, the budget tau^2 rounded down as well), so it does not depend
on the summation order and host and device take the same decision bit for bit; the
quantisation moves the budget by at most 2^-40 of tau^2 per dropped block.  tau = 0
drops nothing.

Third rule, mixed-norm truncation (`keep_mask_mixed`; §6 removes small elements with
the mixed norm of the removed part bounded, citing its selection algorithm): the
off-diagonal blocks are ordered by (||X_IJ||_F^2, I, J) as above, and the longest prefix
is dropped in which every block row of the removed part's matrix of block norms,
M_E[I, J] = ||E_IJ||_F (both triangles), sums to at most tau.  The spectral norm of a
nonnegative symmetric matrix is at most its largest row sum, so ||E||_2 <= ||E||_M =
||M_E||_2 <= tau.  Reading: the row sums are taken in exact integer units of 2^(e - 40),
2^e <= tau < 2^(e+1), each ||X_IJ||_F (the correctly rounded square root of the FP64
||X_IJ||_F^2) rounded down to a unit and the budget tau rounded down, so host and device
take the same decision bit for bit; blocks with ||X_IJ||_F > tau are never dropped.

`sp2_bsr` runs Alg. 3 on dense FP64 matrices with the blocks masked after every
step; `keep_mask`, `keep_mask_error`, `keep_mask_mixed` and `square_pattern` are the
index work on their own.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import sp2_oracle as o


def block_norms2(X: np.ndarray, b: int) -> np.ndarray:
    """||X_IJ||_F^2 for every b x b block, rows of squares summed left to right, then
    the row sums top to bottom (sequential FP64 sums via cumsum)."""
    N = X.shape[0]
    nb = N // b
    Y = np.asarray(X, dtype=np.float64).reshape(nb, b, nb, b).transpose(0, 2, 1, 3)  # [I, J, r, c]
    sq = Y * Y
    rows = np.cumsum(sq, axis=3)[..., -1]          # [I, J, r]
    return np.cumsum(rows, axis=2)[..., -1]         # [I, J]


def keep_mask(X: np.ndarray, b: int, tau: float) -> np.ndarray:
    """Blocks kept by the truncation: diagonal blocks, and off-diagonal blocks with
    ||X_IJ||_F^2 >= tau^2.  For symmetric X the mask is symmetric."""
    n2 = block_norms2(X, b)
    keep = n2 >= tau * tau
    np.fill_diagonal(keep, True)
    return keep


def error_units(tau: float) -> tuple[int, int]:
    """(e, budget): 2^e <= tau^2 < 2^(e+1) and the budget floor(tau^2 / 2^(e-40))."""
    tau2 = tau * tau
    _, ex = math.frexp(tau2)          # tau2 = m 2^ex, m in [1/2, 1)
    e = ex - 1
    return e, int(math.floor(math.ldexp(tau2, 40 - e)))


def keep_mask_error(X: np.ndarray, b: int, tau: float) -> np.ndarray:
    """Blocks kept by the error-controlled truncation (module docstring): drop the longest
    prefix, in (||X_IJ||^2, I, J) order over the off-diagonal upper blocks with
    2 ||X_IJ||^2 <= tau^2, whose units 2 ||X_IJ||^2 / 2^(e-40) (rounded down) add up to
    at most the budget."""
    n2 = block_norms2(X, b)
    nb = n2.shape[0]
    keep = np.ones((nb, nb), dtype=bool)
    tau2 = tau * tau
    if tau2 == 0.0:
        return keep
    e, budget = error_units(tau)
    cands = [(float(n2[I, J]), I, J) for I in range(nb) for J in range(I + 1, nb) if 2.0 * n2[I, J] <= tau2]
    cands.sort()
    total = 0
    for v, I, J in cands:
        u = int(math.floor(math.ldexp(v, 41 - e)))      # floor(2 v / 2^(e-40))
        if total + u > budget:
            break
        total += u
        keep[I, J] = keep[J, I] = False
    return keep


def mixed_units(tau: float) -> tuple[int, int]:
    """(e, budget): 2^e <= tau < 2^(e+1) and the budget floor(tau / 2^(e-40))."""
    _, ex = math.frexp(tau)
    e = ex - 1
    return e, int(math.floor(math.ldexp(tau, 40 - e)))


def keep_mask_mixed(X: np.ndarray, b: int, tau: float) -> np.ndarray:
    """Blocks kept by the mixed-norm truncation (module docstring): in (||X_IJ||^2, I, J) order
    over the off-diagonal upper blocks with ||X_IJ|| <= tau, drop blocks while both block rows
    they touch stay within the budget of units; the first block that does not fit ends the
    prefix."""
    n2 = block_norms2(X, b)
    nb = n2.shape[0]
    keep = np.ones((nb, nb), dtype=bool)
    if tau == 0.0:
        return keep
    e, budget = mixed_units(tau)
    cands = [(float(n2[I, J]), I, J) for I in range(nb) for J in range(I + 1, nb)
             if math.sqrt(float(n2[I, J])) <= tau]
    cands.sort()
    rows = [0] * nb
    for v, I, J in cands:
        u = int(math.floor(math.ldexp(math.sqrt(v), 40 - e)))
        if rows[I] + u > budget or rows[J] + u > budget:
            break
        rows[I] += u
        rows[J] += u
        keep[I, J] = keep[J, I] = False
    return keep


def apply_mask(X: np.ndarray, keep: np.ndarray, b: int) -> np.ndarray:
    return X * np.kron(keep, np.ones((b, b)))


def square_pattern(keep: np.ndarray) -> np.ndarray:
    """Block pattern of X^2 for X with block pattern `keep`: (I, J) is structurally
    nonzero iff some K has keep[I, K] and keep[K, J]."""
    k = keep.astype(np.int64)
    return (k @ k) > 0


def sp2_bsr(F: np.ndarray, nocc: int, b: int, tau: float, *, bounds=None, max_iter: int = 200,
            guard: bool = True, rule: str = "block", norm: str = "fro", acc=None, storage: str = "fp64"):
    """Alg. 3 with X~_i = X_i + E_i, E_i the block truncation above (FP64 values);
    rule "block" (drop blocks with norm below tau), "error" (||E_i||_F <= tau) or "mixed"
    (||E_i||_M <= tau through the row sums); norm "fro" (v_i) or "mixed" (m_i with the
    b x b blocks, the pairing of the §6 calculations).  acc = (homo_out, homo_in, lumo_in,
    lumo_out) runs SP2-ACC (Alg. 4 / Alg. 5) with the same truncation instead of Alg. 3.
    storage "fp32": every iterate is rounded to FP32 values as soon as it is formed and the
    truncation is decided on the rounded values (E_i = storage rounding + truncation)."""
    mask = {"block": keep_mask, "error": keep_mask_error, "mixed": keep_mask_mixed}[rule]

    def perturb(i, X):
        return apply_mask(X, mask(X, b, tau), b) - X
    if acc is not None:
        from oracle import sp2acc_oracle as oa
        return oa.sp2_acc(F, nocc, *acc, bounds=bounds, guard=guard, norm=norm, block=b, perturb=perturb,
                          storage=storage)
    return o.sp2(F, nocc, bounds=bounds, max_iter=max_iter, guard=guard, perturb=perturb, norm=norm, block=b,
                 storage=storage)


def gershgorin_bounds_blocks(F: np.ndarray) -> tuple[float, float]:
    """Gershgorin discs of F (the same bounds as the dense oracle)."""
    return o.gershgorin_bounds(F)

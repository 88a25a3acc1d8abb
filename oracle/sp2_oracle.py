"""CPU FP64 oracle for SP2 density-matrix purification -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this module.  The library's product path never calls it: it is the plain, slow,
readable statement of what the GPU path must compute, written from the paper
(Kruchinina, Rudberg, Rubensson, "Parameterless stopping criteria for recursive
density matrix expansions", arXiv:1507.02087) and sharing no code with it.

Every step is FP64 numpy; a matrix product is the only library primitive used.

What it computes (Alg. 3, the original SP2 algorithm with the new stop):
  X_0 = (lmax I - F) / (lmax - lmin)                       (Alg. 3, initial scaling)
  for i = 1, 2, ...:
     p_i = 1, X_i = X_{i-1}^2          if Tr[X_{i-1}] > nocc  (Alg. 3, trace test)
     p_i = 0, X_i = 2 X_{i-1} - X_{i-1}^2   otherwise
     v_i = ||X_i - X_i^2||_F                              (§2, Frobenius estimate of e_i)
     stop at the first i >= 2 with p_i != p_{i-1}, v_{i-2} < 1 and
        log(v_i / C) / log(v_{i-2}) < qtilde,   C = (71 + 17 sqrt 17) / 32, qtilde = 1.8
                                                          (Alg. 3 stop; §2 relaxed order)
  output n = i and X_n.

Readings where the paper is silent (each also listed in the design notes):
  * bounds: Gershgorin discs give lmin/lmax (the paper allows any outer bounds, §3).
  * the order test is only evaluated when v_{i-2} < 1: the Frobenius argument of §2
    assumes it, and §2 notes the test is not checked otherwise.  For
    0 < v_{i-2} < 1 it is equivalent to v_i > C v_{i-2}^qtilde; v_{i-2} == 0 stops.
  * a trace tie Tr[X_{i-1}] == nocc takes the `else` branch (2X - X^2), as written.
  * guard G (not in the paper): with eigenvalues in [0,1], x^2 <= x and 2x - x^2 >= x,
    so in exact arithmetic the trace moves strictly down after X^2 and strictly up
    after 2X - X^2 unless X is already idempotent.  If after forming X_i the trace did not
    move that way, and the observed convergence order over the last pair has fallen below
    qtilde (the order test on v_{i-1}, v_{i-3} without the alternation it needs), rounding
    or truncation dominates and the expansion stops with n = i (reason TRACE_GUARD).  This
    catches the repeated-polynomial runs that §4.2 (Thm 2) says trace-based selection
    cannot bound (their error grows, order ~1), and it does not fire while the error still
    converges, when a systematic rounding bias summed over many converged eigenvalues can
    outweigh the trace change of the last unconverged ones.
  * a hard iteration cap (reason CAP) is a safety net only.
  * nocc == 0 gives D = 0 and nocc == N gives D = I directly (the definition of D in
    §1); lmax == lmin (F a multiple of I) with 0 < nocc < N has no gap and is an error.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Alg. 3 and §4: smallest constant with log(e_i/C)/log(e_{i-2}) >= 2 in exact
# arithmetic for alternating SP2 polynomials (Theorem 1 applied to p^(12), p^(21)).
C2_SP = (71.0 + 17.0 * math.sqrt(17.0)) / 32.0
QTILDE = 1.8  # §2: relaxed order used in place of q = 2

STOP_ORDER = 0        # the paper's convergence-order test fired
STOP_TRACE_GUARD = 1  # guard G fired
STOP_EXACT = 2        # trivial or exactly idempotent case
STOP_CAP = 3          # iteration cap reached


@dataclasses.dataclass
class SP2Result:
    D: np.ndarray
    n: int                 # output iteration index: D = X_n
    stop_reason: int
    lmin: float
    lmax: float
    v: list                # v[i] = ||X_i - X_i^2||_F for i = 0..len-1
    trace: list            # trace[i] = Tr[X_i]
    p: list                # p[i] for i >= 1 (p[0] is None)


def gershgorin_bounds(F: np.ndarray) -> tuple[float, float]:
    """Outer spectral bounds from Gershgorin discs: every eigenvalue lies in some
    [F_ii - R_i, F_ii + R_i] with R_i = sum_{j != i} |F_ij|."""
    F = np.asarray(F, dtype=np.float64)
    d = np.diag(F)
    R = np.abs(F).sum(axis=1) - np.abs(d)
    return float(np.min(d - R)), float(np.max(d + R))


def initial_scaling(F: np.ndarray, lmin: float, lmax: float) -> np.ndarray:
    """X_0 = (lmax I - F) / (lmax - lmin): maps the spectrum into [0, 1] in reverse
    order, occupied eigenvalues towards 1 (Alg. 3)."""
    N = F.shape[0]
    return (lmax * np.eye(N) - F) / (lmax - lmin)


def idempotency_error_fro(X: np.ndarray, X2: np.ndarray) -> float:
    """v = ||X - X^2||_F (§2, Frobenius-norm estimate of e = ||X - X^2||_2)."""
    return float(np.linalg.norm(X - X2, "fro"))


def idempotency_error_spectral(X: np.ndarray, X2: np.ndarray) -> float:
    """e = ||X - X^2||_2 for symmetric X (§2, the error the stop is defined on)."""
    w = np.linalg.eigvalsh(X - X2)
    return float(np.max(np.abs(w)))


def mixed_norm(A: np.ndarray, b: int) -> float:
    """||A||_M (§2): the spectral norm of the matrix of Frobenius norms of the b x b blocks of
    A (zero-padded to a multiple of b).  e <= m <= v for e = ||A||_2, v = ||A||_F."""
    A = np.asarray(A, dtype=np.float64)
    N = A.shape[0]
    nb = -(-N // b)
    P = np.zeros((nb * b, nb * b))
    P[:N, :N] = A
    M = np.sqrt((P.reshape(nb, b, nb, b) ** 2).sum(axis=(1, 3)))
    return float(np.linalg.norm(M, 2))


def order_stagnates(v: list, i: int, qtilde: float = QTILDE) -> bool:
    """The error condition of the trace guard at X_i: the order test on the last pair,
    log(v_{i-1} / C) / log(v_{i-3}) < qtilde (with its v_{i-3} < 1 and v = 0 rules), i >= 3."""
    return i >= 3 and order_test_stops(v[i - 1], v[i - 3], qtilde)


def order_test_stops(v_i: float, v_im2: float, qtilde: float = QTILDE, C: float = C2_SP) -> bool:
    """Alg. 3 stop condition log(v_i/C)/log(v_{i-2}) < qtilde, evaluated only when
    v_{i-2} < 1 (see the module notes)."""
    if v_im2 == 0.0:
        return True
    if not (v_im2 < 1.0):
        return False
    if v_i == 0.0:
        return False  # log(0) = -inf: observed order +inf, no stop
    return math.log(v_i / C) / math.log(v_im2) < qtilde


def store_fp32(X: np.ndarray) -> np.ndarray:
    """The nearest FP32 value of every entry (round to nearest even), held in FP64: the
    storage part of Alg. 1's perturbation, X~ = X + E with E = fl32(X) - X."""
    return np.asarray(X, dtype=np.float64).astype(np.float32).astype(np.float64)


def sp2(F: np.ndarray, nocc: int, *, bounds: tuple[float, float] | None = None,
        max_iter: int = 200, qtilde: float = QTILDE, norm: str = "fro", guard: bool = True,
        perturb=None, block: int = 128, storage: str = "fp64", trace: str = "diag") -> SP2Result:
    """Alg. 3 step by step in FP64.

    `perturb(i, X)` (optional) returns the truncation/noise matrix E_i added to X_i
    (Alg. 1, X~_i = X_i + E_i); by default E_i = 0 (dense, no truncation).
    `norm` is "fro" (v_i, what the GPU path uses by default), "spectral" (e_i, the paper's
    definition; eigvalsh, small N only) or "mixed" (m_i, the mixed norm of §2 with blocks of
    `block` x `block`).
    `storage` "fp32" keeps every iterate as FP32 values: X_0 and each X_i are rounded to the
    nearest FP32 value as soon as they are formed, before `perturb` (Alg. 1: E_i holds that
    rounding, plus the truncation if any).  Products, traces, norms and the stop test stay
    FP64; this is the expansion the low-precision paths carry out in exact arithmetic on
    their stored iterates, so its stop is where their rounding floor is detected.
    `trace` "diag" (Alg. 3) takes Tr[X~_{i-1}] from the diagonal of the stored iterate;
    "fro" takes it from the identity Tr[Y^2] = ||Y||_F^2 for symmetric Y: Tr[X_i] =
    ||X~_{i-1}||_F^2 after X^2 and 2 Tr[X~_{i-1}] - ||X~_{i-1}||_F^2 after 2X - X^2 (the
    trace of X_i before its perturbation), and the trace guard compares it with the diagonal
    sum Tr[X~_{i-1}]."""
    F = np.asarray(F, dtype=np.float64)
    N = F.shape[0]
    if F.shape != (N, N):
        raise ValueError("F must be square")
    if not (0 <= nocc <= N):
        raise ValueError("nocc must lie in [0, N]")
    if bounds is None:
        lmin, lmax = gershgorin_bounds(F) if N > 0 else (0.0, 0.0)
    else:
        lmin, lmax = bounds
    if nocc == 0 or nocc == N:
        D = np.zeros((N, N)) if nocc == 0 else np.eye(N)
        return SP2Result(D, 0, STOP_EXACT, lmin, lmax, [], [], [None])
    if not (lmax > lmin):
        raise ValueError("F has no spectral width: there is no homo-lumo gap")
    if norm == "mixed":
        def err(X, X2):
            return mixed_norm(X - X2, block)
    else:
        err = idempotency_error_fro if norm == "fro" else idempotency_error_spectral

    if storage not in ("fp64", "fp32") or trace not in ("diag", "fro"):
        raise ValueError("storage is 'fp64' or 'fp32', trace is 'diag' or 'fro'")

    def stored(i, Y):
        # X~_i = X_i + E_i: FP32 storage rounding first, then the prescribed perturbation
        if storage == "fp32":
            Y = store_fp32(Y)
        if perturb is not None:
            Y = Y + perturb(i, Y)
        return Y

    X = stored(0, initial_scaling(F, lmin, lmax))
    X2 = X @ X
    v = [err(X, X2)]
    tr = [float(np.trace(X))]
    p = [None]
    if v[0] == 0.0:
        return SP2Result(X, 0, STOP_EXACT, lmin, lmax, v, tr, p)

    for i in range(1, max_iter + 1):
        if tr[i - 1] > nocc:
            Xi, pi = X2, 1                 # X_i = X~_{i-1}^2
        else:
            Xi, pi = 2.0 * X - X2, 0       # X_i = 2 X~_{i-1} - X~_{i-1}^2
        if trace == "fro":
            fro2 = float(np.sum(X * X))
            tr_prev = float(np.trace(X))
            tr_i = fro2 if pi == 1 else 2.0 * tr_prev - fro2
        Xi = stored(i, Xi)
        if trace == "diag":
            tr_prev = tr[i - 1]
            tr_i = float(np.trace(Xi))
        tr.append(tr_i)
        p.append(pi)
        if guard and ((pi == 1 and tr[i] >= tr_prev) or (pi == 0 and tr[i] <= tr_prev)) and \
                order_stagnates(v, i, qtilde):
            return SP2Result(Xi, i, STOP_TRACE_GUARD, lmin, lmax, v, tr, p)
        X2i = Xi @ Xi
        v.append(err(Xi, X2i))
        if i >= 2 and p[i] != p[i - 1] and order_test_stops(v[i], v[i - 2], qtilde):
            return SP2Result(Xi, i, STOP_ORDER, lmin, lmax, v, tr, p)
        X, X2 = Xi, X2i
    return SP2Result(X, max_iter, STOP_CAP, lmin, lmax, v, tr, p)


# ---- scalar form: the same recursion on each eigenvalue ------------------------------

def sp2_scalar(lams, nocc: int, lmin: float, lmax: float, *, max_iter: int = 200,
               qtilde: float = QTILDE, guard: bool = True):
    """The SP2 recursion applied to a list of eigenvalues with plain Python floats.

    For a diagonal F the matrix iteration acts on each diagonal entry separately, so
    this must reproduce the matrix oracle: same polynomial sequence, same stop, and
    v_i = sqrt(sum_j (x_j - x_j^2)^2).  Returns (x_final, n, reason, v, tr, p)."""
    xs = [(lmax - lam) / (lmax - lmin) for lam in lams]

    def vnorm(vals):
        return math.sqrt(math.fsum((x - x * x) ** 2 for x in vals))

    v = [vnorm(xs)]
    tr = [math.fsum(xs)]
    p = [None]
    for i in range(1, max_iter + 1):
        if tr[i - 1] > nocc:
            xs_new, pi = [x * x for x in xs], 1
        else:
            xs_new, pi = [2.0 * x - x * x for x in xs], 0
        tr.append(math.fsum(xs_new))
        p.append(pi)
        if guard and ((pi == 1 and tr[i] >= tr[i - 1]) or (pi == 0 and tr[i] <= tr[i - 1])) and \
                order_stagnates(v, i, qtilde):
            return xs_new, i, STOP_TRACE_GUARD, v, tr, p
        v.append(vnorm(xs_new))
        if i >= 2 and p[i] != p[i - 1] and order_test_stops(v[i], v[i - 2], qtilde):
            return xs_new, i, STOP_ORDER, v, tr, p
        xs = xs_new
    return xs, max_iter, STOP_CAP, v, tr, p


# ---- the constant C_2^sp from Theorem 1 ----------------------------------------------

def p_sp1(x):
    return x * x


def p_sp2(x):
    return 2.0 * x - x * x


def ratio_g(f, x):
    """(f(x) - f(x)^2) / (x - x^2)^2: the quantity maximised in Theorem 1 with a = 0, q = 2."""
    fx = f(x)
    return (fx - fx * fx) / (x - x * x) ** 2


def c2sp_numeric(samples: int = 200_001) -> tuple[float, float]:
    """max over x in (0,1) of ratio_g for the compositions p^(12) = p1(p2(x)) and
    p^(21) = p2(p1(x)) (§4), by dense sampling then golden-section refinement.
    Returns (max for p^(12), max for p^(21))."""
    f12 = lambda x: p_sp1(p_sp2(x))
    f21 = lambda x: p_sp2(p_sp1(x))
    out = []
    for f in (f12, f21):
        xs = np.linspace(0.0, 1.0, samples)[1:-1]
        vals = ratio_g(f, xs)
        k = int(np.argmax(vals))
        a, b = xs[max(k - 1, 0)], xs[min(k + 1, len(xs) - 1)]
        phi = (math.sqrt(5.0) - 1.0) / 2.0
        for _ in range(200):
            c = b - phi * (b - a)
            d = a + phi * (b - a)
            if ratio_g(f, c) > ratio_g(f, d):
                b = d
            else:
                a = c
        out.append(float(ratio_g(f, 0.5 * (a + b))))
    return out[0], out[1]


# ---- invariants of a density matrix (§1) ---------------------------------------------

def invariants(F: np.ndarray, D: np.ndarray, nocc: int) -> dict:
    """|Tr D - nocc|, ||D^2 - D||_F and ||F D - D F||_F: zero for the exact projector."""
    D2 = D @ D
    FD = F @ D
    return {
        "trace_err": abs(float(np.trace(D)) - nocc),
        "idem_err": float(np.linalg.norm(D2 - D, "fro")),
        "comm_err": float(np.linalg.norm(FD - FD.T, "fro")),
    }


def rel_error(D: np.ndarray, D_ref: np.ndarray, nocc: int) -> float:
    """||D - D_ref||_F / sqrt(nocc), the accuracy measure the results are stated in."""
    return float(np.linalg.norm(np.asarray(D) - np.asarray(D_ref), "fro")) / math.sqrt(max(nocc, 1))

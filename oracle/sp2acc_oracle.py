"""CPU FP64 oracle for SP2-ACC, the homo/lumo-based accelerated SP2 -- TEST
INFRASTRUCTURE ONLY.

Only the tests and the benchmark's CPU-baseline leg may import this module.  It
states, plainly and slowly, what the GPU path computes for the accelerated expansion
(Alg. 4 and Alg. 5 of the paper) and shares no code with it.

Alg. 4 (polynomial schedule).  From outer spectral bounds lmin, lmax and bounds of the
homo and lumo eigenvalues, homo_out <= homo <= homo_in and lumo_in <= lumo <= lumo_out,
the images of homo and lumo under the initial scaling are bracketed by distances to
their targets: beta (homo, distance to 1) in [beta_lo, beta_up] and gamma (lumo,
distance to 0) in [gamma_lo, gamma_up].  Each step chooses the polynomial that moves
the farther one: p_i = 1 (the lumo side, X <- ((1 - a) I + a X)^2) if gamma_up >= beta_up,
else p_i = 0 (X <- 2 a X - (a X)^2), with the scale-and-fold factor
a_i = 2 / (2 - gamma_lo) or 2 / (2 - beta_lo), and maps all four bounds through the same
polynomial.  Once beta_lo and gamma_lo are both below delta = 0.01 the acceleration is
turned off for good (beta_lo = gamma_lo = 0, so a = 1 from then on) and n_min is the next
step.  The schedule ends (n_max) when beta_up - beta_up^2 and gamma_up - gamma_up^2 are
both at most machine epsilon and the last two polynomials differ.

Alg. 5 (expansion).  X_0 = (lmax I - F)/(lmax - lmin); X_i from X_{i-1} with p_i, a_i;
v_i = ||X_i - X_i^2||_F; stop at the first i >= n_min with p_i != p_{i-1} and the order
test of Alg. 3 (log(v_i / C) / log(v_{i-2}) < 1.8, evaluated only when v_{i-2} < 1, as in
the plain oracle); otherwise D = X_{n_max}.

Readings (also listed in the design notes):
  * the loop condition of Alg. 4 prints "(not converged) and p_i = p_{i-1}"; read as "or":
    with "and" the schedule would end at its first alternation, long before the bounds
    converge.  The first step has no predecessor and never ends the loop.
  * the trace guard of the plain oracle (x^2 <= x, 2x - x^2 >= x on [0, 1], with the order over
    the last pair below qtilde) holds only for the unscaled polynomials, so it is checked only
    from n_min on, where a = 1.
  * reaching n_max without the order test firing ends the run with D = X_{n_max}
    (reason STOP_SCHEDULE).
  * outer bounds beyond the spectral bounds (homo_out < lmin, lumo_out > lmax) are clamped
    to them: beta_lo and gamma_lo are distances inside [0, 1] and may not be negative.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from oracle import sp2_oracle as o

STOP_SCHEDULE = 4       # the precomputed schedule ran out (n_max reached)
DELTA = 0.01            # Alg. 4: acceleration off once both lower bounds are below it
EPS_M = float(np.finfo(np.float64).eps)


@dataclasses.dataclass
class Schedule:
    n_min: int
    n_max: int
    p: list          # p[i], i = 1..n_max (p[0] is None)
    alpha: list      # alpha[i], i = 1..n_max (alpha[0] is None)
    beta_up: list    # beta_up after step i (index 0: initial value)
    gamma_up: list


def acc_schedule(lmin: float, lmax: float, homo_out: float, homo_in: float, lumo_in: float, lumo_out: float,
                 *, delta: float = DELTA, eps: float = EPS_M, max_steps: int = 500) -> Schedule:
    """Alg. 4: the polynomial choices p_i, scale factors alpha_i, n_min and n_max."""
    homo_out, lumo_out = max(homo_out, lmin), min(lumo_out, lmax)
    W = lmax - lmin
    b_up = 1.0 - (lmax - homo_in) / W
    b_lo = 1.0 - (lmax - homo_out) / W
    g_up = (lmax - lumo_in) / W
    g_lo = (lmax - lumo_out) / W
    p, alpha = [None], [None]
    bu, gu = [b_up], [g_up]
    n_min = None
    i = 0
    while (b_up - b_up * b_up > eps or g_up - g_up * g_up > eps) or i < 2 or p[i] == p[i - 1]:
        # (the printed condition joins the two parts with "and"; see the readings above)
        if i >= max_steps:
            raise RuntimeError("the schedule did not converge")
        i += 1
        if delta > 0.0 and b_lo < delta and g_lo < delta:
            b_lo, g_lo = 0.0, 0.0
            n_min = i + 1
            delta = 0.0
        # each value is formed with one rounding per operation, in the order written
        def fold(a, x):      # ((1 - a) + a x)^2
            y = (1.0 - a) + a * x
            return y * y

        def lift(a, x):      # 2 a x - (a x)^2
            y = a * x
            return 2.0 * a * x - y * y

        if g_up >= b_up:
            a = 2.0 / (2.0 - g_lo)
            g_lo, g_up = fold(a, g_lo), fold(a, g_up)
            b_lo, b_up = lift(a, b_lo), lift(a, b_up)
            p.append(1)
        else:
            a = 2.0 / (2.0 - b_lo)
            g_lo, g_up = lift(a, g_lo), lift(a, g_up)
            b_lo, b_up = fold(a, b_lo), fold(a, b_up)
            p.append(0)
        alpha.append(a)
        bu.append(b_up)
        gu.append(g_up)
    if n_min is None:
        n_min = i + 1
    return Schedule(n_min, i, p, alpha, bu, gu)


def apply_step(X: np.ndarray, p: int, a: float) -> np.ndarray:
    """One step of Alg. 5: ((1 - a) I + a X)^2 for p = 1, 2 a X - (a X)^2 for p = 0."""
    N = X.shape[0]
    if p == 1:
        Y = (1.0 - a) * np.eye(N) + a * X
        return Y @ Y
    Y = a * X
    return 2.0 * Y - Y @ Y


def sp2_acc(F: np.ndarray, nocc: int, homo_out: float, homo_in: float, lumo_in: float, lumo_out: float, *,
            bounds: tuple[float, float] | None = None, qtilde: float = o.QTILDE, guard: bool = True,
            delta: float = DELTA, sched: Schedule | None = None, norm: str = "fro", block: int = 128,
            perturb=None, storage: str = "fp64") -> o.SP2Result:
    """Alg. 5 step by step in FP64 (Alg. 4 supplies the schedule).  `norm`: "fro" (v_i),
    "spectral" (e_i = ||X_i - X_i^2||_2, the error of §2; eigvalsh, small N only) or "mixed" (m_i
    with `block` x `block` blocks).  `perturb(i, X)` (optional) returns Alg. 1's E_i, added to X_0
    and to every X_i as soon as it is formed, as in the plain oracle; `storage` "fp32" rounds
    X_0 and every X_i to FP32 values first, as in the plain oracle."""
    if storage not in ("fp64", "fp32"):
        raise ValueError("storage is 'fp64' or 'fp32'")

    def stored(i, Y):
        if storage == "fp32":
            Y = o.store_fp32(Y)
        return Y + perturb(i, Y) if perturb is not None else Y
    if norm == "mixed":
        def err(X, X2):
            return o.mixed_norm(X - X2, block)
    else:
        err = o.idempotency_error_fro if norm == "fro" else o.idempotency_error_spectral
    F = np.asarray(F, dtype=np.float64)
    N = F.shape[0]
    lmin, lmax = o.gershgorin_bounds(F) if bounds is None else bounds
    if nocc == 0 or nocc == N:
        D = np.zeros((N, N)) if nocc == 0 else np.eye(N)
        return o.SP2Result(D, 0, o.STOP_EXACT, lmin, lmax, [], [], [None])
    if not (lmax > lmin):
        raise ValueError("F has no spectral width: there is no homo-lumo gap")
    if sched is None:
        sched = acc_schedule(lmin, lmax, homo_out, homo_in, lumo_in, lumo_out, delta=delta)
    X = stored(0, o.initial_scaling(F, lmin, lmax))
    X2 = X @ X
    v = [err(X, X2)]
    tr = [float(np.trace(X))]
    p = [None]
    if v[0] == 0.0:
        return o.SP2Result(X, 0, o.STOP_EXACT, lmin, lmax, v, tr, p)
    for i in range(1, sched.n_max + 1):
        pi = sched.p[i]
        Xi = stored(i, apply_step(X, pi, sched.alpha[i]))
        tr.append(float(np.trace(Xi)))
        p.append(pi)
        if guard and i >= sched.n_min and ((pi == 1 and tr[i] >= tr[i - 1]) or (pi == 0 and tr[i] <= tr[i - 1])) \
                and o.order_stagnates(v, i, qtilde):
            return o.SP2Result(Xi, i, o.STOP_TRACE_GUARD, lmin, lmax, v, tr, p)
        X2i = Xi @ Xi
        v.append(err(Xi, X2i))
        if i >= max(2, sched.n_min) and p[i] != p[i - 1] and o.order_test_stops(v[i], v[i - 2], qtilde):
            return o.SP2Result(Xi, i, o.STOP_ORDER, lmin, lmax, v, tr, p)
        X = Xi
    return o.SP2Result(X, sched.n_max, STOP_SCHEDULE, lmin, lmax, v, tr, p)


def sp2_acc_scalar(lams, nocc: int, lmin: float, lmax: float, sched: Schedule, *, qtilde: float = o.QTILDE,
                   guard: bool = True):
    """The same expansion on a list of eigenvalues (plain floats): for a diagonal F the
    matrix iteration acts on each diagonal entry separately.  Returns (xs, n, reason, p)."""
    xs = [(lmax - lam) / (lmax - lmin) for lam in lams]

    def vnorm(vals):
        return math.sqrt(math.fsum((x - x * x) ** 2 for x in vals))

    v = [vnorm(xs)]
    tr = [math.fsum(xs)]
    p = [None]
    for i in range(1, sched.n_max + 1):
        pi, a = sched.p[i], sched.alpha[i]
        ys = [((1.0 - a) + a * x) if pi == 1 else a * x for x in xs]
        xs_new = [y * y for y in ys] if pi == 1 else [2.0 * y - y * y for y in ys]
        tr.append(math.fsum(xs_new))
        p.append(pi)
        if guard and i >= sched.n_min and ((pi == 1 and tr[i] >= tr[i - 1]) or (pi == 0 and tr[i] <= tr[i - 1])) \
                and o.order_stagnates(v, i, qtilde):
            return xs_new, i, o.STOP_TRACE_GUARD, p
        v.append(vnorm(xs_new))
        if i >= max(2, sched.n_min) and p[i] != p[i - 1] and o.order_test_stops(v[i], v[i - 2], qtilde):
            return xs_new, i, o.STOP_ORDER, p
        xs = xs_new
    return xs, sched.n_max, STOP_SCHEDULE, p

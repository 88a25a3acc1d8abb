"""CPU FP64 oracle for the McWeeny expansion and McW-ACC (§3) -- TEST INFRASTRUCTURE ONLY.

Only the tests may import this module.  It states, plainly, what the GPU path computes for
the McWeeny purification and shares no code with it.

McWeeny (§3): with a chemical potential mu between the homo and lumo eigenvalues and outer
spectral bounds lmin, lmax,
    gamma = 2 max(lmax - mu, mu - lmin),   X_0 = (mu I - F) / gamma + I / 2,
    X_i = 3 X_{i-1}^2 - 2 X_{i-1}^3,
and the parameterless stop with C_2^mw = 4 (the maximum of (p(x) - p(x)^2) / (x - x^2)^2 =
3 + 4x - 4x^2 on [0, 1]) on consecutive errors: stop at the first i with
log(e_i / 4) / log(e_{i-1}) < 1.8.

McW-ACC (§3.1): with a gap estimate xi such that some eigenvalue of F lies in
[mu - xi/2, mu + xi/2], beta_0 = (1 - xi / gamma) / 2 and, every step,
    alpha = 3 / sqrt(12 beta^2 - 18 beta + 9),   X_s = alpha (X - I/2) + I/2,
    X_i = 3 X_s^2 - 2 X_s^3,   beta_s = alpha (beta - 1/2) + 1/2,   beta <- 3 beta_s^2 - 2 beta_s^3.

Readings (also listed in the design notes):
  * the error is v_i = ||X_i - X_i^2||_F in place of the spectral e_i by default (§3.2 shows the
    regular scheme then never stops early); norm="spectral" takes e_i itself;
  * as for SP2 the order test is evaluated only when v_{i-1} < 1 (v_{i-1} = 0 stops, v_i = 0
    does not);
  * acceleration: §3.2 shows the Frobenius estimate can stop the accelerated scheme early and
    advises switching the acceleration off when the purification phase starts; it is switched
    off for good once beta < delta = 0.01 (the threshold Alg. 4 uses for SP2-ACC), and the stop
    test runs from the step after (n_min); without acceleration n_min = 1;
  * an iteration cap (reason CAP) is a safety net.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import sp2_oracle as o

C2_MW = 4.0
DELTA = 0.01


def p_mw(x):
    return 3.0 * x * x - 2.0 * x * x * x


def mcw_schedule(gamma: float, xi: float, accelerate: bool, steps: int, delta: float = DELTA):
    """alpha_i for i = 1..steps and n_min (the first step where the stop test runs)."""
    beta = 0.5 * (1.0 - xi / gamma)
    alpha = [None]
    n_min = 1 if not accelerate else None
    on = accelerate
    for i in range(1, steps + 1):
        if on and beta < delta:
            on = False
            n_min = i + 1
        a = 3.0 / math.sqrt(12.0 * beta * beta - 18.0 * beta + 9.0) if on else 1.0
        bs = a * (beta - 0.5) + 0.5
        beta = 3.0 * bs * bs - 2.0 * bs * bs * bs
        alpha.append(a)
    if n_min is None:
        n_min = steps + 1
    return alpha, n_min


def initial_mcw(F: np.ndarray, mu: float, lmin: float, lmax: float) -> tuple[np.ndarray, float]:
    N = F.shape[0]
    gamma = 2.0 * max(lmax - mu, mu - lmin)
    return (mu * np.eye(N) - F) / gamma + 0.5 * np.eye(N), gamma


def mcweeny(F: np.ndarray, mu: float, *, xi: float = 0.0, accelerate: bool = False,
            bounds: tuple[float, float] | None = None, max_iter: int = 200, qtilde: float = o.QTILDE,
            delta: float = DELTA, norm: str = "fro") -> o.SP2Result:
    """McWeeny (accelerate False) or McW-ACC (True) step by step in FP64.  `norm`: "fro" (v_i)
    or "spectral" (e_i = ||X_i - X_i^2||_2, §2; eigvalsh, small N only)."""
    err = o.idempotency_error_fro if norm == "fro" else o.idempotency_error_spectral
    F = np.asarray(F, dtype=np.float64)
    N = F.shape[0]
    lmin, lmax = o.gershgorin_bounds(F) if bounds is None else bounds
    if not (lmax > lmin):
        raise ValueError("F has no spectral width")
    X, gamma = initial_mcw(F, mu, lmin, lmax)
    alpha, n_min = mcw_schedule(gamma, xi, accelerate, max_iter, delta)
    X2 = X @ X
    v = [err(X, X2)]
    tr = [float(np.trace(X))]
    p = [None]
    for i in range(1, max_iter + 1):
        a = alpha[i]
        Xs = a * (X - 0.5 * np.eye(N)) + 0.5 * np.eye(N)
        S = Xs @ Xs
        Xi = 3.0 * S - 2.0 * (S @ Xs)
        X2i = Xi @ Xi
        v.append(err(Xi, X2i))
        tr.append(float(np.trace(Xi)))
        p.append(1)
        if i >= n_min and o.order_test_stops(v[i], v[i - 1], qtilde, C2_MW):
            return o.SP2Result(Xi, i, o.STOP_ORDER, lmin, lmax, v, tr, p)
        X = Xi
    return o.SP2Result(X, max_iter, o.STOP_CAP, lmin, lmax, v, tr, p)


def mcweeny_scalar(lams, mu: float, lmin: float, lmax: float, alpha, n_min: int, *, max_iter: int = 200,
                   qtilde: float = o.QTILDE):
    """The same iteration on a list of eigenvalues (a diagonal F): (xs, n, reason)."""
    gamma = 2.0 * max(lmax - mu, mu - lmin)
    xs = [(mu - lam) / gamma + 0.5 for lam in lams]

    def vnorm(vals):
        return math.sqrt(math.fsum((x - x * x) ** 2 for x in vals))

    v = [vnorm(xs)]
    for i in range(1, max_iter + 1):
        a = alpha[i]
        ys = [a * (x - 0.5) + 0.5 for x in xs]
        xs_new = [3.0 * (y * y) - 2.0 * ((y * y) * y) for y in ys]
        v.append(vnorm(xs_new))
        if i >= n_min and o.order_test_stops(v[i], v[i - 1], qtilde, C2_MW):
            return xs_new, i, o.STOP_ORDER
        xs = xs_new
    return xs, max_iter, o.STOP_CAP

"""More pins of the CPU oracle: a hand-computed Gershgorin case, the closed form of the
SP2-ACC acceleration efficiency (§4, the delta discussion), and the FP32-storage
expansion (Alg. 1 with E_i = storage rounding) against an exactly rounded scalar map.
Each pin has a planted mistake it must catch."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import sp2_oracle as o
from oracle import sp2acc_oracle as oa


# ---- Gershgorin discs, by hand ------------------------------------------------------------
# F = [[2, -1, 1/2], [-1, 3, 0], [1/2, 0, -1]]: discs [2 - 3/2, 2 + 3/2] = [1/2, 7/2],
# [3 - 1, 3 + 1] = [2, 4], [-1 - 1/2, -1 + 1/2] = [-3/2, -1/2]; lmin = -3/2, lmax = 4.
F3 = np.array([[2.0, -1.0, 0.5], [-1.0, 3.0, 0.0], [0.5, 0.0, -1.0]])


def gershgorin_pin_holds(bounds_fn) -> bool:
    return bounds_fn(F3) == (-1.5, 4.0)


def test_gershgorin_hand_case():
    assert gershgorin_pin_holds(o.gershgorin_bounds)


def test_planted_gershgorin_radius_is_caught():
    # a radius that keeps |F_ii| (R_i = sum_j |F_ij|) gives (-5/2, 7): the pin fails
    def wrong(F):
        d = np.diag(F)
        R = np.abs(F).sum(axis=1)
        return float(np.min(d - R)), float(np.max(d + R))
    assert not gershgorin_pin_holds(wrong)


# ---- SP2-ACC: alpha_i against the acceleration efficiency (§4) -----------------------------
# With alpha = 2 / (2 - lam), 1 - alpha + alpha lam = lam / (2 - lam), so the efficiency the
# paper plots, |lam^2 - (1 - alpha + alpha lam)^2| / |lam - lam^2|, is lam (3 - lam) / (2 - lam)^2:
# 14/81 at lam = 1/5 and 0.0299 / 3.9601 < 1 % at lam = delta = 0.01, the paper's reason for delta.
# Spectrum [-1, 1] with homo in [-0.7, -0.5] and lumo in [0.4, 0.6]: beta_up = 1/4, beta_lo = 3/20,
# gamma_up = 3/10, gamma_lo = 1/5, so step 1 is p = 1 with alpha_1 = 2 / (2 - 1/5) = 10/9, and the
# bounds map to gamma_up = ((1 - 10/9) + (10/9)(3/10))^2 = 4/81 and
# beta_up = 2 (10/9)(1/4) - ((10/9)(1/4))^2 = 155/324 (Alg. 4).
def efficiency(alpha, lam):
    return abs(lam ** 2 - (1.0 - alpha + alpha * lam) ** 2) / abs(lam - lam ** 2)


def acc_pin_holds(s) -> bool:
    ok = s.p[1] == 1
    ok &= efficiency(s.alpha[1], 0.2) == pytest.approx(14.0 / 81.0, rel=1e-13)
    ok &= s.gamma_up[1] == pytest.approx(4.0 / 81.0, rel=1e-13)
    ok &= s.beta_up[1] == pytest.approx(155.0 / 324.0, rel=1e-13)
    return bool(ok)


def test_acc_alpha_matches_efficiency_closed_form():
    s = oa.acc_schedule(-1.0, 1.0, -0.7, -0.5, 0.4, 0.6)
    assert acc_pin_holds(s)
    assert efficiency(2.0 / (2.0 - 0.01), 0.01) == pytest.approx(0.0299 / 3.9601, rel=1e-12)
    assert efficiency(2.0 / (2.0 - 0.01), 0.01) < 0.01


def test_planted_wrong_alpha_is_caught():
    # alpha from the inner bound (2 / (2 - gamma_up)) instead of the outer one
    s = oa.acc_schedule(-1.0, 1.0, -0.7, -0.5, 0.4, 0.6)
    a = 2.0 / (2.0 - 0.3)
    wrong = oa.Schedule(s.n_min, s.n_max, s.p, [None, a] + s.alpha[2:],
                        s.beta_up[:1] + [2 * a * 0.25 - (a * 0.25) ** 2] + s.beta_up[2:],
                        s.gamma_up[:1] + [((1 - a) + a * 0.3) ** 2] + s.gamma_up[2:])
    assert not acc_pin_holds(wrong)


# ---- FP32 storage: a diagonal F against the exactly rounded scalar map --------------------

def round_fp32(r: Fraction) -> Fraction:
    """The FP32 value nearest the rational r (ties to even), from the format's definition:
    24 significant bits for normal numbers, a fixed step of 2^-149 below 2^-126."""
    if r == 0:
        return Fraction(0)
    sign = -1 if r < 0 else 1
    a = abs(r)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1                                     # 2^e <= a < 2^(e+1)
    step = Fraction(2) ** max(e - 23, -149)
    q, rem = divmod(a / step, 1)
    q = int(q)
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and q % 2 == 1):
        q += 1
    return sign * q * step


def scalar_fp32(x0s, nocc, trace_rule, max_iter=200):
    """SP2 on the eigenvalues with each new value rounded once to FP32 (exact rational
    arithmetic otherwise): p from the trace, the trace guard (trace moved the wrong way and the
    order test holds on v_{i-1}, v_{i-3}), and the order test on v_i = sqrt(sum (x - x^2)^2)."""
    xs = [Fraction(x) for x in x0s]
    v = [math.sqrt(float(sum((x - x * x) ** 2 for x in xs)))]
    tr = [float(sum(xs))]
    p = [None]
    for i in range(1, max_iter + 1):
        pi = 1 if tr[i - 1] > nocc else 0
        new = [round_fp32(x * x if pi else 2 * x - x * x) for x in xs]
        if trace_rule == "diag":
            t_prev, t_i = tr[i - 1], float(sum(new))
        else:
            s2 = sum(x * x for x in xs)
            t_prev, t_i = float(sum(xs)), float(s2 if pi else 2 * sum(xs) - s2)
        tr.append(t_i)
        p.append(pi)
        if ((pi == 1 and t_i >= t_prev) or (pi == 0 and t_i <= t_prev)) and i >= 3 and \
                o.order_test_stops(v[i - 1], v[i - 3]):
            return new, i, o.STOP_TRACE_GUARD, p
        v.append(math.sqrt(float(sum((x - x * x) ** 2 for x in new))))
        if i >= 2 and p[i] != p[i - 1] and o.order_test_stops(v[i], v[i - 2]):
            return new, i, o.STOP_ORDER, p
        xs = new
    return xs, max_iter, o.STOP_CAP, p


def fp32_diag_case(seed):
    # X_0 = (1 I - F) / 2 exactly (bounds (-1, 1)) for x_0 = k / 4096: F = 1 - 2 x_0
    g = np.random.Generator(np.random.PCG64(seed))
    N, nocc = 41, 17
    k = np.concatenate([g.integers(2100, 4000, nocc), g.integers(50, 1990, N - nocc)])
    g.shuffle(k)
    x0 = k / 4096.0
    return np.diag(1.0 - 2.0 * x0), x0, nocc


def fp32_pin_holds(res, x0, nocc, trace_rule) -> bool:
    xs, n, reason, p = scalar_fp32(x0, nocc, trace_rule)
    return (res.n, res.stop_reason) == (n, reason) and res.p == p and \
        np.array_equal(np.diag(res.D), np.array([float(x) for x in xs]))


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("trace_rule", ["diag", "fro"])
def test_fp32_storage_diagonal_matches_rounded_scalar_map(seed, trace_rule):
    F, x0, nocc = fp32_diag_case(seed)
    res = o.sp2(F, nocc, bounds=(-1.0, 1.0), storage="fp32", trace=trace_rule)
    assert res.stop_reason in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    assert fp32_pin_holds(res, x0, nocc, trace_rule)
    D = np.diag(res.D)
    assert np.array_equal(D.astype(np.float32).astype(np.float64), D)   # every entry an FP32 value
    # the FP64 expansion of the same F is a different computation: the pin separates the two
    r64 = o.sp2(F, nocc, bounds=(-1.0, 1.0))
    assert not fp32_pin_holds(r64, x0, nocc, trace_rule)


def test_fp32_storage_stops_no_later_than_fp64_and_agrees_in_exact_cases():
    # the floor of FP32 storage comes earlier than FP64's; with the trace taken from the
    # Frobenius identity the p sequence equals the diagonal rule's until the floor
    from paper_1507_02087_gb300 import inputs
    case = inputs.dense_gapped(160, 70, gap=0.05, seed=4)
    F = case.F.numpy()
    r64 = o.sp2(F, 70)
    r32 = o.sp2(F, 70, storage="fp32")
    r32f = o.sp2(F, 70, storage="fp32", trace="fro")
    assert r32.n <= r64.n and r32f.n <= r64.n
    m = min(r32.n, r32f.n) - 4
    assert r32.p[1:m] == r32f.p[1:m] == r64.p[1:m]
    assert o.rel_error(r32.D, case.D_exact, 70) < 1e-5


def test_planted_missing_iterate_rounding_is_caught(monkeypatch):
    # rounding only X_0 (the iterates kept in FP64) leaves non-FP32 entries: the pin fails
    F, x0, nocc = fp32_diag_case(0)
    calls = {"n": 0}
    real = o.store_fp32

    def first_only(X):
        calls["n"] += 1
        return real(X) if calls["n"] == 1 else np.asarray(X, dtype=np.float64)
    monkeypatch.setattr(o, "store_fp32", first_only)
    res = o.sp2(F, nocc, bounds=(-1.0, 1.0), storage="fp32")
    assert not fp32_pin_holds(res, x0, nocc, "diag")

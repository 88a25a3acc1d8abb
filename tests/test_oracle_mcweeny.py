"""Pins of the McWeeny / McW-ACC oracle (§3): the constant C_2^mw = 4 and the limits 3, the
closed form of the ratio, the accelerated counterexample ratio 2/sqrt(5) of §3.2, the
non-premature Frobenius stop of the regular scheme, the scalar map, the exact projector,
and the gain of the acceleration."""
import math

import numpy as np
import pytest

from oracle import jacobi
from oracle import mcweeny_oracle as om
from oracle import sp2_oracle as o
from paper_1507_02087_gb300 import inputs


def g(x):
    p = om.p_mw(x)
    return (p - p * p) / (x - x * x) ** 2


def test_c2mw_is_four_and_limits_three():
    xs = np.linspace(1e-6, 1 - 1e-6, 200_001)
    vals = g(xs)
    assert float(vals.max()) == pytest.approx(4.0, abs=1e-9)
    assert float(xs[np.argmax(vals)]) == pytest.approx(0.5, abs=1e-5)
    assert g(1e-7) == pytest.approx(3.0, abs=1e-5)
    x = np.array([0.1, 0.3, 0.77, 1 - 1e-3])
    assert np.allclose(g(x), 3 + 4 * x - 4 * x * x, rtol=1e-9)      # the closed form of §3
    # p(1 - x) = 1 - p(x), so g is symmetric about 1/2 and the limit at 1 is the limit at 0
    assert np.allclose(om.p_mw(1 - x) + om.p_mw(x), 1.0, rtol=0, atol=1e-15)


def test_accelerated_frobenius_counterexample():
    # X = diag(0, 0, 0, b, 1 - b): the K-ratio of the accelerated step is 2/sqrt(5)
    b = 0.3
    a = 3.0 / math.sqrt(12 * b * b - 18 * b + 9)

    def pmwa(x):
        return om.p_mw(a * (x - 0.5) + 0.5)

    lam = np.array([0, 0, 0, b, 1 - b])
    e0 = lam - lam ** 2
    pl = pmwa(lam)
    e1 = pl - pl ** 2
    ratio = (np.sum(e0 ** 2) * np.max(np.abs(e1))) / (np.max(np.abs(e0)) ** 2 * np.sqrt(np.sum(e1 ** 2)))
    assert ratio == pytest.approx(2 / math.sqrt(5), rel=1e-12)


def test_regular_scheme_frobenius_ratio_does_not_grow():
    # §3.2: K_i = v_i / e_i satisfies K_i <= K_{i-1}^2 for the regular McWeeny polynomial
    gen = np.random.Generator(np.random.PCG64(5))
    for _ in range(20):
        lam = gen.uniform(0.0, 1.0, 60)
        for _ in range(6):
            e = lam - lam ** 2
            K0 = np.sqrt(np.sum(e ** 2)) / np.max(np.abs(e))
            lam = om.p_mw(lam)
            e1 = lam - lam ** 2
            if np.max(np.abs(e1)) == 0:
                break
            K1 = np.sqrt(np.sum(e1 ** 2)) / np.max(np.abs(e1))
            assert K1 <= K0 ** 2 * (1 + 1e-12)


def test_diagonal_matches_scalar_map():
    gen = np.random.Generator(np.random.PCG64(6))
    N = 120
    lam = np.concatenate([gen.uniform(-1, -0.05, 50), gen.uniform(0.05, 1, N - 50)])
    gen.shuffle(lam)
    F = np.diag(lam)
    for acc in (False, True):
        res = om.mcweeny(F, 0.0, xi=0.1, accelerate=acc)
        gamma = 2 * max(res.lmax, -res.lmin)
        alpha, n_min = om.mcw_schedule(gamma, 0.1, acc, 200)
        xs, n, reason = om.mcweeny_scalar(lam, 0.0, res.lmin, res.lmax, alpha, n_min)
        assert res.n == n and res.stop_reason == reason
        assert np.allclose(np.diag(res.D), xs, rtol=0, atol=1e-14)
        assert np.array_equal(np.diag(res.D) > 0.5, lam < 0)


@pytest.mark.parametrize("N,nocc,seed", [(10, 4, 1), (32, 16, 2)])
def test_tiny_against_jacobi(N, nocc, seed):
    case = inputs.dense_gapped(N, nocc, gap=0.1, seed=seed)
    F = case.F.numpy()
    for acc in (False, True):
        res = om.mcweeny(F, 0.0, xi=0.1, accelerate=acc)
        assert res.stop_reason == o.STOP_ORDER
        assert o.rel_error(res.D, jacobi.density_by_definition(F, nocc), nocc) < 1e-12


def test_acceleration_saves_iterations():
    case = inputs.dense_gapped(200, 100, gap=0.01, seed=3)
    F = case.F.numpy()
    plain = om.mcweeny(F, 0.0)
    acc = om.mcweeny(F, 0.0, xi=0.01, accelerate=True)
    assert acc.stop_reason == o.STOP_ORDER and plain.stop_reason == o.STOP_ORDER
    assert acc.n < plain.n
    assert o.rel_error(acc.D, plain.D, 100) < 1e-12


def test_spectral_error_on_diagonal_is_largest_scalar_error():
    # a diagonal F keeps every X_i diagonal, so e_i = max_j |x_j - x_j^2| (no eigensolver);
    # the error measure changes only where the run stops, never the iterates
    gen = np.random.Generator(np.random.PCG64(9))
    N = 90
    lam = np.concatenate([gen.uniform(-1, -0.05, 40), gen.uniform(0.05, 1, N - 40)])
    gen.shuffle(lam)
    F = np.diag(lam)
    for acc in (False, True):
        rs = om.mcweeny(F, 0.0, xi=0.1, accelerate=acc, norm="spectral")
        rf = om.mcweeny(F, 0.0, xi=0.1, accelerate=acc)
        gamma = 2 * max(rs.lmax, -rs.lmin)
        alpha, _ = om.mcw_schedule(gamma, 0.1, acc, 200)
        xs = (0.0 - lam) / gamma + 0.5
        for i in range(len(rs.v)):
            if rs.v[i] > 1e-12:                      # above the rounding floor
                assert rs.v[i] == pytest.approx(float(np.max(np.abs(xs - xs * xs))), rel=1e-9)
            assert rs.v[i] <= rf.v[i] * (1 + 1e-12) if i < len(rf.v) else True
            ys = alpha[i + 1] * (xs - 0.5) + 0.5 if i + 1 < len(alpha) else xs
            xs = 3 * ys * ys - 2 * ys * ys * ys
        assert abs(rs.n - rf.n) <= 1 and rs.stop_reason == o.STOP_ORDER


def test_spectral_stop_dense_between_bounds():
    # e_i <= v_i <= sqrt(N) e_i on the same iterates, and the spectral stop reaches the projector
    case = inputs.dense_gapped(120, 60, gap=0.05, seed=4)
    F = case.F.numpy()
    rs = om.mcweeny(F, 0.0, xi=0.05, accelerate=True, norm="spectral")
    rf = om.mcweeny(F, 0.0, xi=0.05, accelerate=True)
    for i in range(min(len(rs.v), len(rf.v))):
        assert rs.v[i] <= rf.v[i] * (1 + 1e-12) and rf.v[i] <= math.sqrt(120) * rs.v[i] * (1 + 1e-12)
    assert o.rel_error(rs.D, jacobi.density_by_definition(F, 60), 60) < 1e-12


@pytest.mark.parametrize("beta", [0.05, 0.2, 0.3, 0.45])
def test_accelerated_ratio_limit_closed_form(beta):
    # §3.1: with alpha(beta) of McW-ACC, g1(x, beta) = (p - p^2) / (x - x^2)^2 for
    # p = p_mw(alpha (x - 1/2) + 1/2) tends, as x -> beta from above, to
    # 16 (beta - 1.5)^2 (beta - 0.75)^2 / ((beta - 1)^2 (4 beta^2 - 6 beta + 3)^3)
    alpha, _ = om.mcw_schedule(1.0, 1.0 - 2.0 * beta, True, 1)    # beta_0 = (1 - xi / gamma) / 2
    a = alpha[1]
    x = beta + 1e-9
    p = om.p_mw(a * (x - 0.5) + 0.5)
    g1 = (p - p * p) / (x - x * x) ** 2
    closed = 16 * (beta - 1.5) ** 2 * (beta - 0.75) ** 2 / ((beta - 1) ** 2 * (4 * beta ** 2 - 6 * beta + 3) ** 3)
    assert g1 == pytest.approx(closed, rel=1e-6)

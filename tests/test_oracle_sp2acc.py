"""Pins of the SP2-ACC oracle (Alg. 4 schedule, Alg. 5 expansion) against what the paper
and the mathematics fix: the worked case of Theorem 2's proof, the run-length bounds of
§4.2, the scalar map on a diagonal F, the exact projector for tiny N, and the gain of the
acceleration."""
import math

import numpy as np
import pytest

from oracle import jacobi
from oracle import sp2_oracle as o
from oracle import sp2acc_oracle as oa
from paper_1507_02087_gb300 import inputs


def runs_after_startup(p):
    """Longest run of equal polynomials after both have appeared once."""
    seq = p[1:]
    start = next((k for k in range(1, len(seq)) if seq[k] != seq[0]), len(seq))
    best, cur = 0, 0
    for k in range(start, len(seq)):
        cur = cur + 1 if k > start and seq[k] == seq[k - 1] else 1
        best = max(best, cur)
    return best


def test_theorem2_worked_case():
    # beta_0 = gamma_0 with no acceleration (outer bounds at the spectrum's ends):
    # p_1 = 1, p_2 = p_3 = 0, p_4 = 1, and gamma_1 = gamma_0^2, beta_1 = 2 gamma_0 - gamma_0^2
    g0 = 0.25                                    # exact in binary, so beta_0 == gamma_0 exactly
    lmin, lmax = -1.0, 1.0
    homo = lmax - (1.0 - g0) * (lmax - lmin)     # beta_up = g0
    lumo = lmax - g0 * (lmax - lmin)             # gamma_up = g0
    s = oa.acc_schedule(lmin, lmax, lmin, homo, lumo, lmax, delta=0.0)
    assert s.p[1:5] == [1, 0, 0, 1]
    assert all(a == 1.0 for a in s.alpha[1:])
    assert s.gamma_up[1] == pytest.approx(g0 ** 2, rel=1e-14)
    assert s.beta_up[1] == pytest.approx(2 * g0 - g0 ** 2, rel=1e-14)
    # the mirrored case (p_1 = 0 when beta_0 is the larger by a rounding step): 0, 1, 1, 0
    s2 = oa.acc_schedule(lmin, lmax, lmin, -0.4, 0.4 + 2e-16, lmax, delta=0.0)
    assert s2.p[1:5] == [0, 1, 1, 0]


@pytest.mark.parametrize("seed", range(6))
def test_run_lengths_bounded(seed):
    g = np.random.Generator(np.random.PCG64(seed))
    for _ in range(50):
        lmin, lmax = -1.0 - g.random(), 1.0 + g.random()
        homo_in = g.uniform(-0.9, -0.001)
        lumo_in = g.uniform(0.001, 0.9)
        # no acceleration: at most two equal polynomials in a row after the start-up (Theorem 2)
        s0 = oa.acc_schedule(lmin, lmax, lmin, homo_in, lumo_in, lmax)
        assert runs_after_startup(s0.p) <= 2
        # with acceleration (outer bounds close to the inner ones): at most three (§4.2)
        s1 = oa.acc_schedule(lmin, lmax, homo_in - 1e-3, homo_in, lumo_in, lumo_in + 1e-3)
        assert runs_after_startup(s1.p) <= 3
        assert s1.n_min <= s1.n_max and s1.p[s1.n_max] != s1.p[s1.n_max - 1]
        assert s1.beta_up[-1] - s1.beta_up[-1] ** 2 <= oa.EPS_M
        assert s1.gamma_up[-1] - s1.gamma_up[-1] ** 2 <= oa.EPS_M


def test_acceleration_saves_iterations():
    # small gap: the scale-and-fold schedule needs fewer steps than the unaccelerated one
    lmin, lmax = -1.0, 1.0
    homo, lumo = -0.0025, 0.0025
    plain = oa.acc_schedule(lmin, lmax, lmin, homo, lumo, lmax)
    acc = oa.acc_schedule(lmin, lmax, homo, homo, lumo, lumo)
    assert acc.n_max < plain.n_max
    assert acc.n_max <= plain.n_max - 5


def test_diagonal_f_matches_scalar_map():
    g = np.random.Generator(np.random.PCG64(3))
    N, nocc = 150, 61
    lam = np.concatenate([g.uniform(-1, -0.02, nocc), g.uniform(0.02, 1.0, N - nocc)])
    g.shuffle(lam)
    F = np.diag(lam)
    lmin, lmax = o.gershgorin_bounds(F)
    homo, lumo = float(np.max(lam[lam < 0])), float(np.min(lam[lam > 0]))
    sched = oa.acc_schedule(lmin, lmax, homo, homo, lumo, lumo)
    res = oa.sp2_acc(F, nocc, homo, homo, lumo, lumo, sched=sched)
    xs, n, reason, p = oa.sp2_acc_scalar(lam, nocc, lmin, lmax, sched)
    assert res.n == n and res.stop_reason == reason and res.p == p
    assert np.array_equal(np.diag(res.D), np.array(xs))
    assert np.array_equal(np.diag(res.D) > 0.5, lam < 0)


@pytest.mark.parametrize("N,nocc,seed", [(8, 3, 1), (24, 12, 2), (40, 7, 3)])
def test_tiny_against_jacobi_projector(N, nocc, seed):
    case = inputs.dense_gapped(N, nocc, gap=0.1, seed=seed)
    F = case.F.numpy()
    w = np.linalg.eigvalsh(F)
    homo, lumo = float(w[nocc - 1]), float(w[nocc])
    res = oa.sp2_acc(F, nocc, homo - 1e-3, homo, lumo, lumo + 1e-3)
    assert res.stop_reason in (o.STOP_ORDER, o.STOP_TRACE_GUARD, oa.STOP_SCHEDULE)
    D_def = jacobi.density_by_definition(F, nocc)
    assert o.rel_error(res.D, D_def, nocc) < 1e-12


def test_matches_plain_oracle_on_n400():
    # a different polynomial sequence reaching the same projector, in fewer iterations
    case = inputs.dense_n400()
    F = case.F.numpy()
    lam = np.linalg.eigvalsh(F)
    homo, lumo = float(lam[case.nocc - 1]), float(lam[case.nocc])
    res = oa.sp2_acc(F, case.nocc, homo - 1e-4, homo, lumo, lumo + 1e-4)
    ref = o.sp2(F, case.nocc)
    assert o.rel_error(res.D, ref.D, case.nocc) < 1e-12
    assert res.n < ref.n
    inv = o.invariants(F, res.D, case.nocc)
    assert inv["trace_err"] < 1e-9 and inv["idem_err"] < 1e-10 and inv["comm_err"] < 1e-10


def test_schedule_keeps_true_homo_lumo_in_unit_interval():
    # the fold factors use the lower bounds, so the true homo and lumo images (anywhere
    # inside their brackets) are never stretched outside [0, 1] and end at 1 and 0
    lmin, lmax = -1.0, 1.0
    homo, lumo = -0.01, 0.01
    s = oa.acc_schedule(lmin, lmax, homo - 0.004, homo, lumo, lumo + 0.004)
    W = lmax - lmin
    x_homo, x_lumo = (lmax - homo) / W, (lmax - lumo) / W
    xh, xl = x_homo, x_lumo
    for i in range(1, s.n_max + 1):
        a = s.alpha[i]
        f = (lambda x: ((1 - a) + a * x) ** 2) if s.p[i] == 1 else (lambda x: 2 * a * x - (a * x) ** 2)
        xh, xl = f(xh), f(xl)
        assert 0.0 <= xl <= 1.0 and 0.0 <= xh <= 1.0      # eigenvalues stay in [0, 1]
    assert xh > 1 - 1e-8 and xl < 1e-8


def test_spectral_error_on_diagonal_is_largest_scalar_error():
    # diagonal F: e_i = max_j |x_j - x_j^2| of the scalar map (no eigensolver involved)
    g = np.random.Generator(np.random.PCG64(12))
    N, nocc = 80, 30
    lam = np.concatenate([g.uniform(-1, -0.03, nocc), g.uniform(0.03, 1.0, N - nocc)])
    g.shuffle(lam)
    F = np.diag(lam)
    lmin, lmax = o.gershgorin_bounds(F)
    homo, lumo = float(np.max(lam[lam < 0])), float(np.min(lam[lam > 0]))
    sched = oa.acc_schedule(lmin, lmax, homo, homo, lumo, lumo)
    rs = oa.sp2_acc(F, nocc, homo, homo, lumo, lumo, sched=sched, norm="spectral")
    rf = oa.sp2_acc(F, nocc, homo, homo, lumo, lumo, sched=sched)
    d = np.diag(rs.D)
    xs, n, reason, p = oa.sp2_acc_scalar(lam, nocc, lmin, lmax, sched)
    assert np.array_equal(d, np.array(xs)) and rs.p == p[:len(rs.p)]
    # the last record is e_n of D = X_n itself: max_j |d_j - d_j^2|
    assert len(rs.v) == rs.n + 1
    assert rs.v[-1] == pytest.approx(float(np.max(np.abs(d - d * d))), rel=1e-9, abs=1e-300)
    for i in range(min(len(rs.v), len(rf.v))):
        assert rs.v[i] <= rf.v[i] * (1 + 1e-12) and rf.v[i] <= np.sqrt(N) * rs.v[i] * (1 + 1e-12)
    assert abs(rs.n - rf.n) <= 1

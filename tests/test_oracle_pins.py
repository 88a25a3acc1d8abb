"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks it against a closed
form printed in the paper, an independent computation (the Jacobi
eigendecomposition, the per-eigenvalue scalar recursion, numpy's eigh), an
invariant of the exact density matrix, or an outcome the paper prints.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import sp2_oracle as o
from oracle.jacobi import density_by_definition, jacobi_eigh
from paper_1507_02087_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- constants (§4) ------------------------------------------------------------------

def test_c2sp_closed_form_is_the_maximum_of_theorem1():
    # §4: max over [0,1] of (f - f^2)/(x - x^2)^2 for f = p^(12) and f = p^(21)
    # equals (71 + 17 sqrt(17)) / 32 ~ 4.40915.
    m12, m21 = o.c2sp_numeric()
    assert m12 == pytest.approx(o.C2_SP, rel=1e-12)
    assert m21 == pytest.approx(o.C2_SP, rel=1e-12)
    assert o.C2_SP == pytest.approx(4.40915, abs=5e-6)


def test_alternating_composition_limits():
    # §4: limits 2 and 4 of the ratio at the ends of [0,1] for p^(12), p^(21).
    f12 = lambda x: o.p_sp1(o.p_sp2(x))
    f21 = lambda x: o.p_sp2(o.p_sp1(x))
    e = 1e-6
    assert o.ratio_g(f21, e) == pytest.approx(2.0, rel=1e-4)
    assert o.ratio_g(f12, 1 - e) == pytest.approx(2.0, rel=1e-4)
    assert o.ratio_g(f21, 1 - e) == pytest.approx(4.0, rel=1e-4)
    assert o.ratio_g(f12, e) == pytest.approx(4.0, rel=1e-4)


def test_repeated_polynomial_ratio_is_unbounded():
    # §4: the limits for p^(11) at 1 and p^(22) at 0 do not exist (grow without bound),
    # which is why the stop needs p_i != p_{i-1}.
    f11 = lambda x: o.p_sp1(o.p_sp1(x))
    f22 = lambda x: o.p_sp2(o.p_sp2(x))
    assert o.ratio_g(f11, 1 - 1e-4) > 1e3 and o.ratio_g(f11, 1 - 1e-6) > 1e5
    assert o.ratio_g(f22, 1e-4) > 1e3 and o.ratio_g(f22, 1e-6) > 1e5


def test_order_test_log_form():
    # log(v_i/C)/log(v_{i-2}) < 1.8 with v_{i-2} < 1; the boundary v_i = C v_{i-2}^1.8.
    vm2 = 1e-3
    edge = o.C2_SP * vm2 ** 1.8
    assert not o.order_test_stops(edge * 0.99, vm2)
    assert o.order_test_stops(edge * 1.01, vm2)
    assert not o.order_test_stops(0.5, 1.0)       # v_{i-2} >= 1: not checked
    assert not o.order_test_stops(1e-30, 2.0)
    assert o.order_test_stops(0.3, 0.0)           # exactly idempotent two steps back
    assert not o.order_test_stops(0.0, 0.5)       # v_i = 0: observed order infinite


# ---- bounds ----------------------------------------------------------------------------

def test_gershgorin_bounds_contain_spectrum():
    g = np.random.Generator(np.random.PCG64(11))
    for N in (1, 2, 5, 40):
        A = g.standard_normal((N, N)); A = 0.5 * (A + A.T)
        lo, hi = o.gershgorin_bounds(A)
        w = np.linalg.eigvalsh(A)
        assert lo <= w[0] + 1e-12 and hi >= w[-1] - 1e-12
    d = np.array([3.0, -1.5, 0.25])
    assert o.gershgorin_bounds(np.diag(d)) == (-1.5, 3.0)
    # one off-diagonal pair: discs [a-|b|, a+|b|]
    A = np.array([[1.0, -2.0], [-2.0, 0.0]])
    assert o.gershgorin_bounds(A) == (-2.0, 3.0)


# ---- the eigensolver used as the definition of D --------------------------------------

@pytest.mark.parametrize("N", [1, 2, 3, 7, 16, 33])
def test_jacobi_against_library_eigh(N):
    g = np.random.Generator(np.random.PCG64(100 + N))
    A = g.standard_normal((N, N)); A = 0.5 * (A + A.T)
    w, V = jacobi_eigh(A)
    assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-13, rtol=0)
    assert np.allclose(V.T @ V, np.eye(N), atol=1e-13)
    assert np.allclose((V * w) @ V.T, A, atol=1e-13)


# ---- scalar recursion: diagonal F -----------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_diagonal_matrix_matches_scalar_recursion(seed):
    # For diagonal F the matrix recursion acts on each eigenvalue separately.
    g = np.random.Generator(np.random.PCG64(seed))
    N, nocc = 57, 23
    lam = np.concatenate([g.uniform(-1, -0.02, nocc), g.uniform(0.03, 1.0, N - nocc)])
    g.shuffle(lam)
    F = np.diag(lam)
    res = o.sp2(F, nocc)
    xs, n, reason, v, tr, p = o.sp2_scalar(lam, nocc, res.lmin, res.lmax)
    assert (res.n, res.stop_reason) == (n, reason)
    assert res.p == p
    np.testing.assert_allclose(res.v, v, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(res.trace, tr, rtol=1e-13)
    assert np.array_equal(np.diag(res.D), np.array(xs))   # x^2 and 2x - x^2 are exact per entry
    assert np.count_nonzero(res.D - np.diag(np.diag(res.D))) == 0


def test_scalar_recursion_separates_occupied_from_virtual():
    # The fixed points: occupied eigenvalues (below the gap) go to 1, virtual to 0.
    lam = [-0.9, -0.4, -0.06, 0.05, 0.5, 0.8]
    xs, n, reason, v, tr, p = o.sp2_scalar(lam, 3, -1.0, 1.0)
    assert reason in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    assert all(abs(x - 1.0) < 1e-10 for x in xs[:3])
    assert all(abs(x) < 1e-10 for x in xs[3:])


def test_exact_trace_tie_is_stopped_by_the_guard():
    # Exactly representable spectrum whose trace hits nocc exactly each step:
    # without the guard the expansion may cycle; with it the run ends.
    lam = np.array([-0.5, -0.25, 0.25, 0.5])
    res = o.sp2(np.diag(lam), 2, bounds=(-1.0, 1.0))
    assert res.stop_reason in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    assert np.allclose(np.diag(res.D), [1, 1, 0, 0], atol=1e-12)


# ---- dense: against the definition of D ------------------------------------------------

@pytest.mark.parametrize("N,nocc", [(2, 1), (3, 1), (8, 3), (17, 9), (33, 16), (64, 32)])
def test_small_dense_against_jacobi_definition(N, nocc):
    case = inputs.dense_gapped(N, nocc, gap=0.2, seed=N)
    F = case.F.numpy()
    res = o.sp2(F, nocc)
    D_def = density_by_definition(F, nocc)
    assert o.rel_error(res.D, D_def, nocc) < 1e-12
    assert res.stop_reason in (o.STOP_ORDER, o.STOP_TRACE_GUARD)


def test_dense_n400_against_construction_and_invariants():
    case = inputs.dense_n400()
    F = case.F.numpy()
    res = o.sp2(F, case.nocc)
    assert res.stop_reason == o.STOP_ORDER
    assert o.rel_error(res.D, case.D_exact.numpy(), case.nocc) < 1e-12
    inv = o.invariants(F, res.D, case.nocc)
    assert inv["trace_err"] < 1e-10 and inv["idem_err"] < 1e-11 and inv["comm_err"] < 1e-11
    # Gershgorin bounds are outer bounds of the true spectrum [-1, 1].
    assert res.lmin <= case.lam.min() and res.lmax >= case.lam.max()
    # the history: trace decreases after X^2 and increases after 2X - X^2
    for i in range(1, res.n + 1):
        assert (res.trace[i] < res.trace[i - 1]) == (res.p[i] == 1)


def test_trivial_occupations():
    F = np.diag([0.3, -0.2, 0.1])
    assert np.array_equal(o.sp2(F, 0).D, np.zeros((3, 3)))
    assert np.array_equal(o.sp2(F, 3).D, np.eye(3))
    with pytest.raises(ValueError):
        o.sp2(np.eye(4) * 2.0, 2)


# ---- the paper's printed outcome (§4.1) -------------------------------------------------

_DENSE1000 = {}


def _dense1000_run(norm, spec):
    N, nocc = spec["N"], spec["nocc"]
    if not _DENSE1000:
        _DENSE1000["FE"] = inputs.dense_equidistant_noisy(N, nocc, spec["occupied"], spec["unoccupied"],
                                                          spec["noise_spectral_norm"], count=40)
    F, E = _DENSE1000["FE"]

    def noise(i, X):
        return E[i]

    # The eigenvalues already lie in [0, 1], so the bounds are 0 and 1 (X_0 = I - F).
    return o.sp2(F, nocc, bounds=(0.0, 1.0), norm=norm, perturb=noise, guard=False)


def test_dense1000_noisy_stop_matches_printed_iterations():
    spec = json.load(open(os.path.join(GOLDEN, "dense1000_noise_stop.json")))
    rf = _dense1000_run("fro", spec)
    rs = _dense1000_run("spectral", spec)
    assert rf.stop_reason == o.STOP_ORDER and rs.stop_reason == o.STOP_ORDER
    assert rs.n - rf.n == spec["printed_stop_spectral"] - spec["printed_stop_frobenius"]
    assert rf.n + 1 == spec["printed_stop_frobenius"]
    assert rs.n + 1 == spec["printed_stop_spectral"]


# ---- planted mistakes: the pins above must catch them ----------------------------------

def test_planted_sign_error_in_scaling_is_caught(monkeypatch):
    # X_0 = (F - lmin I)/(lmax - lmin) (a sign slip) drives X towards the projector on
    # the virtual space: the Jacobi-definition pin fails.
    case = inputs.dense_gapped(17, 9, gap=0.2, seed=17)
    F = case.F.numpy()
    real = o.initial_scaling
    monkeypatch.setattr(o, "initial_scaling", lambda F_, a, b: np.eye(F_.shape[0]) - real(F_, a, b))
    res = o.sp2(F, 9)
    assert o.rel_error(res.D, density_by_definition(F, 9), 9) > 0.1


def test_planted_wrong_lag_is_caught():
    # Comparing v_i with v_{i-1} instead of v_{i-2} moves the stop of the printed
    # example (or removes it): the printed-iteration pin fails.
    spec = json.load(open(os.path.join(GOLDEN, "dense1000_noise_stop.json")))
    r = _dense1000_run("fro", dict(spec, N=300, nocc=150))
    wrong = None
    for i in range(2, len(r.v)):
        if r.p[i] != r.p[i - 1] and o.order_test_stops(r.v[i], r.v[i - 1]):
            wrong = i
            break
    assert wrong != r.n


# ---- the mixed norm of §2 ---------------------------------------------------------------------

def test_mixed_norm_between_spectral_and_frobenius():
    g = np.random.Generator(np.random.PCG64(31))
    for N, b in [(50, 8), (64, 16), (100, 128), (96, 1)]:
        A = g.standard_normal((N, N))
        A = A + A.T
        e = float(np.linalg.norm(A, 2))
        m = o.mixed_norm(A, b)
        v = float(np.linalg.norm(A, "fro"))
        assert e <= m * (1 + 1e-12) and m <= v * (1 + 1e-12)


def test_mixed_norm_special_block_sizes():
    g = np.random.Generator(np.random.PCG64(32))
    A = g.standard_normal((40, 40))
    assert o.mixed_norm(A, 1) == pytest.approx(float(np.linalg.norm(np.abs(A), 2)), rel=1e-12)
    assert o.mixed_norm(A, 40) == pytest.approx(float(np.linalg.norm(A, "fro")), rel=1e-12)
    assert o.mixed_norm(A, 64) == pytest.approx(float(np.linalg.norm(A, "fro")), rel=1e-12)   # padded
    # block-diagonal with equal blocks: the largest block's Frobenius norm
    B = np.kron(np.eye(4), np.full((8, 8), 0.5))
    assert o.mixed_norm(B, 8) == pytest.approx(4.0, rel=1e-12)


def test_mixed_norm_stop_on_dense_case():
    # the stop with m_i in place of v_i reaches the same projector; for this size the mixed
    # norm lies between e_i and v_i at every step
    case = inputs.dense_gapped(300, 150, gap=0.05, seed=4)
    F = case.F.numpy()
    rm = o.sp2(F, 150, norm="mixed", block=64)
    rs = o.sp2(F, 150, norm="spectral")
    rf = o.sp2(F, 150)
    for r in (rm, rs, rf):
        assert o.rel_error(r.D, case.D_exact.numpy() if case.D_exact is not None else rf.D, 150) < 1e-12
    k = min(len(rm.v), len(rs.v), len(rf.v))
    assert all(rs.v[i] <= rm.v[i] * (1 + 1e-9) and rm.v[i] <= rf.v[i] * (1 + 1e-9) for i in range(k))
    assert rf.n <= rm.n <= rs.n + 1

"""Cyclic Jacobi eigensolver and the density matrix by its definition --
TEST INFRASTRUCTURE ONLY (imported by the tests, never by the library).

For tiny N this gives the density matrix straight from its definition in §1,
D = sum_{i <= nocc} x_i x_i^T over the eigenvectors of the nocc smallest
eigenvalues, without any purification, so the SP2 oracle can be checked against
it.  The eigensolver is the textbook cyclic-by-row Jacobi method: each sweep
visits every off-diagonal pair (p, q) and applies the plane rotation that zeroes
A[p, q], until the off-diagonal mass is below tol * ||A||_F.
"""
from __future__ import annotations

import math

import numpy as np


def jacobi_eigh(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Eigenvalues (ascending) and orthonormal eigenvectors (columns) of symmetric A."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    scale = np.linalg.norm(A, "fro")
    for _ in range(max_sweeps):
        off = float(np.linalg.norm(A - np.diag(np.diag(A)), "fro"))
        if off <= tol * scale:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                # Rotation J with J[p,p]=J[q,q]=c, J[p,q]=s, J[q,p]=-s chosen so that
                # (J^T A J)[p,q] = 0: t = tan(theta) is the smaller root of
                # t^2 + 2 tau t - 1 = 0 with tau = (a_qq - a_pp) / (2 a_pq).
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                if abs(tau) > 1e150:
                    t = 0.5 / tau  # the smaller root, without overflowing tau^2
                else:
                    t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + math.sqrt(1.0 + tau * tau))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = t * c
                colp = A[:, p].copy()
                colq = A[:, q].copy()
                A[:, p] = c * colp - s * colq
                A[:, q] = s * colp + c * colq
                rowp = A[p, :].copy()
                rowq = A[q, :].copy()
                A[p, :] = c * rowp - s * rowq
                A[q, :] = s * rowp + c * rowq
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    w = np.diag(A).copy()
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


def density_by_definition(F: np.ndarray, nocc: int) -> np.ndarray:
    """D = sum over the nocc smallest eigenpairs of x_i x_i^T (§1, definition of D)."""
    _, V = jacobi_eigh(F)
    Vo = V[:, :nocc]
    return Vo @ Vo.T

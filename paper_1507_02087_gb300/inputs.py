"""Seeded synthetic Fock matrices for SP2 density-matrix purification.

The paper's own matrices (the alkane Hartree-Fock Fock matrix of §5 and the
water-cluster SCF matrices of §6) are not available, so these generators stand
in for them: dense symmetric matrices with a prescribed gapped spectrum and a
random orthogonal eigenbasis (the construction the paper uses for its dense
tests in §4.1 and §5), and a gapped three-dimensional tight-binding
Hamiltonian whose density matrix decays exponentially like an insulator's.

This module holds none of the purification's arithmetic.  It only draws random
numbers and builds F = Q diag(lam) Q^T, together with the exact density matrix
D = Q[:, :nocc] Q[:, :nocc]^T that the construction fixes (the definition of D
in §1: the projector onto the eigenvectors of the nocc smallest eigenvalues).
Both the CPU oracle and the GPU path are fed from here.

Random numbers come from numpy's PCG64 generator with the stated seed, so a
case is the same on every machine.  Large cases may be assembled on a CUDA
device with torch (QR, matrix products); the draws themselves always happen on
the host.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch


def rng(seed: int) -> np.random.Generator:
    """PCG64 stream for a seed; every generator below draws from one of these."""
    return np.random.Generator(np.random.PCG64(seed))


@dataclasses.dataclass
class DenseCase:
    """A dense symmetric Fock matrix with a known spectral projector."""

    F: torch.Tensor           # N x N float64, exactly symmetric
    nocc: int
    lam: np.ndarray           # eigenvalues paired with Q's columns (occupied first)
    D_exact: torch.Tensor | None  # Q[:, :nocc] Q[:, :nocc]^T, or None if not asked for
    name: str = ""

    @property
    def N(self) -> int:
        return self.F.shape[0]


def gapped_eigenvalues(N: int, nocc: int, occ: tuple[float, float],
                       virt: tuple[float, float], g: np.random.Generator) -> np.ndarray:
    """nocc occupied eigenvalues uniform in `occ`, then N-nocc virtual ones uniform in `virt`."""
    if not (0 <= nocc <= N):
        raise ValueError("nocc must lie in [0, N]")
    lo = g.uniform(occ[0], occ[1], size=nocc)
    hi = g.uniform(virt[0], virt[1], size=N - nocc)
    return np.concatenate([lo, hi])


def _symmetrize(F: torch.Tensor) -> torch.Tensor:
    # Exact symmetry: both triangles hold the same rounded value.
    return 0.5 * (F + F.T)


def dense_from_spectrum(lam: np.ndarray, nocc: int, seed: int, device: str | torch.device = "cpu",
                        want_exact: bool = True, name: str = "") -> DenseCase:
    """F = Q diag(lam) Q^T with Q the orthogonal factor of a QR factorisation of a
    seeded N x N standard-Gaussian matrix (the eigenvector construction of the
    paper's dense tests, §4.1 and §5)."""
    N = lam.shape[0]
    G = rng(seed).standard_normal((N, N))
    Gt = torch.from_numpy(G).to(device)
    del G
    Q, _ = torch.linalg.qr(Gt)
    del Gt
    lam_t = torch.from_numpy(lam).to(device=Q.device, dtype=torch.float64)
    F = _symmetrize((Q * lam_t) @ Q.T)
    D = None
    if want_exact:
        Qo = Q[:, :nocc]
        D = _symmetrize(Qo @ Qo.T)
    return DenseCase(F=F, nocc=nocc, lam=lam, D_exact=D, name=name)


def dense_gapped(N: int, nocc: int, *, gap: float, width: float = 1.0, seed: int = 0,
                 device: str | torch.device = "cpu", want_exact: bool = True,
                 name: str = "") -> DenseCase:
    """Occupied eigenvalues uniform in [-width, -gap/2], virtual ones uniform in
    [gap/2, width]: a homo-lumo gap `gap` centred at zero (so kappa = 2 width / gap)."""
    g = rng(seed)
    lam = gapped_eigenvalues(N, nocc, (-width, -gap / 2), (gap / 2, width), g)
    # The eigenvector draw uses its own stream so that lam and Q are independent.
    return dense_from_spectrum(lam, nocc, seed + 1_000_003, device, want_exact, name)


# ---- the named workloads -------------------------------------------------------------

def dense_n400(device="cpu", want_exact=True) -> DenseCase:
    """N=400, nocc=200, occupied in [-1,-0.05], virtual in [0.05,1] (gap 0.1), seed 0."""
    return dense_gapped(400, 200, gap=0.1, seed=0, device=device, want_exact=want_exact,
                        name="dense N=400 nocc=200 gap=0.1")


def dense_equidistant_noisy(N: int, nocc: int, occupied: tuple[float, float], unoccupied: tuple[float, float],
                            noise_norm: float, count: int, seed: int = 0,
                            noise_seed: int = 7) -> tuple[np.ndarray, np.ndarray]:
    """The dense example of §4.1: equidistant occupied and unoccupied eigenvalues, eigenvectors
    from the QR factorisation of a Gaussian matrix (PCG64(seed)), and `count` symmetric Gaussian
    perturbations E_0, E_1, ... of spectral norm `noise_norm` (PCG64(noise_seed), drawn in that
    order, each (G + G^T)/2 rescaled by its largest |eigenvalue|).  Returns (F, E) as float64
    numpy arrays, E of shape (count, N, N)."""
    g = rng(seed)
    lam = np.concatenate([np.linspace(*occupied, nocc), np.linspace(*unoccupied, N - nocc)])
    Q, _ = np.linalg.qr(g.standard_normal((N, N)))
    F = (Q * lam) @ Q.T
    F = 0.5 * (F + F.T)
    gn = rng(noise_seed)
    E = np.empty((count, N, N))
    for i in range(count):
        G = gn.standard_normal((N, N))
        G = 0.5 * (G + G.T)
        E[i] = G * (noise_norm / np.max(np.abs(np.linalg.eigvalsh(G))))
    return F, E


def dense_n8192(device="cpu", want_exact=True) -> DenseCase:
    """N=8192, nocc=4096, spectrum in [-1,1] with gap 0.01 at nocc, seed 0."""
    return dense_gapped(8192, 4096, gap=0.01, seed=0, device=device, want_exact=want_exact,
                        name="dense N=8192 nocc=4096 gap=0.01")


def batch_sizes(count: int = 64, nmin: int = 128, nmax: int = 2048, seed: int = 1):
    """Sizes log-uniform in [nmin, nmax], nocc = floor(N/2), gap uniform in [0.005, 0.1]."""
    g = rng(seed)
    logs = g.uniform(math.log(nmin), math.log(nmax), size=count)
    Ns = np.clip(np.rint(np.exp(logs)).astype(np.int64), nmin, nmax)
    gaps = g.uniform(0.005, 0.1, size=count)
    return [(int(n), int(n) // 2, float(gp)) for n, gp in zip(Ns, gaps)]


def dense_batch(count: int = 64, nmin: int = 128, nmax: int = 2048, seed: int = 1,
                device="cpu", want_exact=True) -> list[DenseCase]:
    """A batch of dense gapped matrices of uneven size, each built like dense_n400
    with its own gap and eigenvector seed (seed*100003 + index)."""
    cases = []
    for k, (N, nocc, gap) in enumerate(batch_sizes(count, nmin, nmax, seed)):
        cases.append(dense_gapped(N, nocc, gap=gap, seed=seed * 100_003 + k, device=device,
                                  want_exact=want_exact,
                                  name=f"batch[{k}] N={N} nocc={nocc} gap={gap:.4f}"))
    return cases


def householder_gapped(N: int, nocc: int, *, gap: float, n_reflectors: int = 64, seed: int = 3,
                       device="cpu", want_exact=True, name: str = "") -> DenseCase:
    """Spectrum as in dense_gapped, eigenvectors Q = H_1 H_2 ... H_m, a product of m
    seeded Householder reflectors H_k = I - 2 u_k u_k^T (|u_k| = 1).  Building F
    costs O(m N^2), which keeps very large N affordable."""
    g = rng(seed)
    lam = gapped_eigenvalues(N, nocc, (-1.0, -gap / 2), (gap / 2, 1.0), g)
    U = g.standard_normal((n_reflectors, N))
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    Ut = torch.from_numpy(U).to(device)

    def apply_q_sandwich(diag_vals: torch.Tensor) -> torch.Tensor:
        # A = Q diag Q^T, applying the reflectors from the innermost outwards:
        # A <- H_k A H_k for k = m, ..., 1.
        A = torch.diag(diag_vals)
        for k in range(n_reflectors - 1, -1, -1):
            u = Ut[k]
            Au = A @ u
            uAu = torch.dot(u, Au)
            # H A H = A - 2 u (Au)^T - 2 (Au) u^T + 4 (u^T A u) u u^T
            #       = A - 2 u w^T - 2 w u^T   with w = Au - (u^T A u) u
            w = Au - uAu * u
            A -= 2.0 * torch.outer(u, w)
            A -= 2.0 * torch.outer(w, u)
        return _symmetrize(A)

    lam_t = torch.from_numpy(lam).to(device=Ut.device, dtype=torch.float64)
    F = apply_q_sandwich(lam_t)
    D = None
    if want_exact:
        occ = torch.zeros(N, dtype=torch.float64, device=Ut.device)
        occ[:nocc] = 1.0
        D = apply_q_sandwich(occ)
    return DenseCase(F=F, nocc=nocc, lam=lam, D_exact=D, name=name)


def householder_n32768(device="cuda", want_exact=True) -> DenseCase:
    """N=32768, nocc=16384, gap 1e-3 (kappa ~ 2e3), Q from 64 reflectors, seed 3."""
    return householder_gapped(32768, 16384, gap=1e-3, n_reflectors=64, seed=3, device=device,
                              want_exact=want_exact, name="householder N=32768 gap=1e-3")


# ---- gapped tight-binding model ------------------------------------------------------

@dataclasses.dataclass
class TightBinding:
    """Simple-cubic Lx x Ly x Lz lattice, one orbital per site, periodic boundaries.
    Site index s = x + Lx y + Lx Ly z.  Onsite +delta where x+y+z is even, -delta where
    odd, plus Gaussian disorder sigma; nearest-neighbour hopping -t.  With Lx = 32 the
    32 x 32 blocks of F are the x-lines of the lattice."""

    dims: tuple
    onsite: np.ndarray        # length N
    rows: np.ndarray          # COO of the off-diagonal hopping (both directions, no duplicates)
    cols: np.ndarray
    hop: float
    nocc: int

    @property
    def N(self) -> int:
        return int(np.prod(self.dims))

    def dense(self, device="cpu", dtype=torch.float64) -> torch.Tensor:
        F = torch.zeros(self.N, self.N, dtype=dtype, device=device)
        idx = torch.arange(self.N, device=device)
        F[idx, idx] = torch.from_numpy(self.onsite).to(device=device, dtype=dtype)
        r = torch.from_numpy(self.rows).to(device)
        c = torch.from_numpy(self.cols).to(device)
        F[r, c] = -self.hop
        return F

    def bsr(self, b: int = 32):
        """Block-sparse (BSR) form with b x b blocks: int32 row_ptr [N/b + 1], int32
        col_idx [nnzb] (sorted in each block row), float64 vals [nnzb, b, b]."""
        if self.N % b:
            raise ValueError("N must be a multiple of the block size")
        nb = self.N // b
        Lx, Ly, Lz = self.dims
        if Lx == b:
            # blocks are x-lines: the diagonal block holds the onsite terms and the hopping
            # along the line, the off-diagonal blocks the hopping to the neighbouring lines
            # (-t on the diagonal of the block); no dense matrix is formed
            cols, vals = [], []
            ring = np.zeros((b, b))
            for x in range(b):
                for dx in (1, -1):
                    if Lx >= 2 and (x + dx) % Lx != x:
                        ring[x, (x + dx) % Lx] = -self.hop
            row_ptr = np.zeros(nb + 1, dtype=np.int32)
            for I in range(nb):
                y, z = I % Ly, I // Ly
                nbrs = set()
                for yy, zz in (((y + 1) % Ly, z), ((y - 1) % Ly, z), (y, (z + 1) % Lz), (y, (z - 1) % Lz)):
                    J = yy + Ly * zz
                    if J != I:
                        nbrs.add(J)
                row = sorted(nbrs | {I})
                for J in row:
                    if J == I:
                        blk = ring + np.diag(self.onsite[I * b:(I + 1) * b])
                    else:
                        blk = -self.hop * np.eye(b)
                    cols.append(J)
                    vals.append(blk)
                row_ptr[I + 1] = len(cols)
            return row_ptr, np.array(cols, dtype=np.int32), np.ascontiguousarray(np.stack(vals))
        F = self.dense().numpy()
        blocks = F.reshape(nb, b, nb, b).transpose(0, 2, 1, 3)
        nz = np.abs(blocks).sum(axis=(2, 3)) > 0
        np.fill_diagonal(nz, True)
        row_ptr = np.zeros(nb + 1, dtype=np.int32)
        row_ptr[1:] = np.cumsum(nz.sum(axis=1))
        I, J = np.nonzero(nz)
        return row_ptr, J.astype(np.int32), np.ascontiguousarray(blocks[I, J])


def tight_binding(L: int = 32, delta: float = 1.0, t: float = 0.3, sigma: float = 0.05, seed: int = 2,
                  dims: tuple | None = None) -> TightBinding:
    """dims = (Lx, Ly, Lz), default (L, L, L); nocc = N/2 (the lower band)."""
    Lx, Ly, Lz = dims if dims is not None else (L, L, L)
    N = Lx * Ly * Lz
    g = rng(seed)
    s = np.arange(N)
    x, y, z = s % Lx, (s // Lx) % Ly, s // (Lx * Ly)
    parity = (x + y + z) % 2
    onsite = np.where(parity == 0, delta, -delta) + sigma * g.standard_normal(N)
    site = lambda a, b_, c: (a % Lx) + Lx * (b_ % Ly) + Lx * Ly * (c % Lz)
    pairs = set()
    for dx, dy, dz, Ld in ((1, 0, 0, Lx), (0, 1, 0, Ly), (0, 0, 1, Lz)):
        if Ld < 2:
            continue
        dst = site(x + dx, y + dy, z + dz)
        for a_, b_ in zip(s.tolist(), dst.tolist()):
            if a_ != b_:
                pairs.add((a_, b_))
                pairs.add((b_, a_))
    pr = np.array(sorted(pairs), dtype=np.int64).reshape(-1, 2)
    return TightBinding(dims=(Lx, Ly, Lz), onsite=onsite, rows=pr[:, 0], cols=pr[:, 1], hop=t, nocc=N // 2)

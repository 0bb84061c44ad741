"""Matrix-dependent semicoarsening (MDSC) two-level preconditioner (TEST INFRASTRUCTURE ONLY).

Paper Sec. 4.4: the multigrid preconditioner of the first-order Stokes solve coarsens the extruded
mesh in the vertical direction first: a prolongation built from per-vertical-line solves of the
Jacobian maps a single-layer (plane) field to the whole column, and the plane problem is solved
by a 2D method.  This file states one two-level version of it from its definitions, with dense
per-column solves and sparse products (library primitives), for checking the GPU implementation.

Definitions (dof = 2 (a (L + 1) + l) + c, vertex a, level l, component c):
* T: the column block-tridiagonal part of J (J restricted to the dofs of each column);
* prolongation P (ndof x 2 nv), semicoarsening to the top level: in column a, P_a = [X_a; I] with
  X_a = -T_a[low, low]^-1 T_a[low, top] (the harmonic extension of the top value down the column:
  the column rows below the top are satisfied with zero right-hand side);
* plane operator A_c = P^T J P (Galerkin);
* plane solve B_c: K steps of Chebyshev acceleration of block-Jacobi on A_c (D = the 2 x 2
  diagonal blocks of A_c) over [lam_hi / ratio, lam_hi], lam_hi the Gershgorin bound of D^-1 A_c;
* smoother S = omega T^-1;
* one symmetric cycle: z1 = S r; z2 = z1 + P B_c P^T (r - J z1); z = z2 + S (r - J z2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

OMEGA = 0.7        # smoother damping (undamped, the block-Jacobi smoother makes the cycle indefinite)
CHEB_STEPS = 8     # Chebyshev steps of the plane solve
CHEB_RATIO = 30.0  # lam_hi / lam_lo of the Chebyshev interval


def column_dofs(nv: int, L: int, a: int) -> np.ndarray:
    return np.arange(2 * a * (L + 1), 2 * (a + 1) * (L + 1))


def column_blocks(J: sp.csr_matrix, nv: int, L: int) -> list:
    """Dense T_a = J[col a, col a] for every column."""
    J = J.tocsr()
    return [J[column_dofs(nv, L, a)][:, column_dofs(nv, L, a)].toarray() for a in range(nv)]


def prolongation(J: sp.csr_matrix, nv: int, L: int) -> sp.csr_matrix:
    """P (ndof x 2 nv): harmonic extension of the top-level value down each column."""
    rows, cols, vals = [], [], []
    for a, T in enumerate(column_blocks(J, nv, L)):
        low, top = slice(0, 2 * L), slice(2 * L, 2 * L + 2)
        Pa = np.zeros((2 * (L + 1), 2))
        Pa[top] = np.eye(2)
        if L > 0:
            Pa[low] = -np.linalg.solve(T[low, low], T[low, top])
        d = column_dofs(nv, L, a)
        for i in range(2 * (L + 1)):
            for c in range(2):
                rows.append(d[i])
                cols.append(2 * a + c)
                vals.append(Pa[i, c])
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nv * (L + 1), 2 * nv))


def plane_operator(J: sp.csr_matrix, P: sp.csr_matrix) -> sp.csr_matrix:
    return (P.T @ J @ P).tocsr()


def block_diag_inverse(Ac: sp.csr_matrix) -> sp.csr_matrix:
    """D^-1 for the 2 x 2 diagonal blocks of the plane operator."""
    Ac = Ac.tocsr()
    n = Ac.shape[0] // 2
    blocks = [sp.csr_matrix(np.linalg.inv(Ac[2 * a:2 * a + 2, 2 * a:2 * a + 2].toarray())) for a in range(n)]
    return sp.block_diag(blocks, format="csr")


def gershgorin_bound(Ac: sp.csr_matrix, Dinv: sp.csr_matrix) -> float:
    """max_i sum_j |(D^-1 A_c)_ij|, an upper bound of the spectrum of D^-1 A_c."""
    M = (Dinv @ Ac).tocsr()
    return float(np.max(np.asarray(abs(M).sum(axis=1)).ravel()))


def chebyshev(Ac: sp.csr_matrix, Dinv: sp.csr_matrix, b: np.ndarray, lam_lo: float, lam_hi: float,
              steps: int) -> np.ndarray:
    """Chebyshev acceleration of the preconditioned Richardson iteration x <- x + D^-1 (b - A x),
    from x = 0, over the interval [lam_lo, lam_hi] of the spectrum of D^-1 A (Saad, Iterative
    Methods for Sparse Linear Systems, Sec. 12.3, Chebyshev acceleration)."""
    theta = 0.5 * (lam_hi + lam_lo)
    delta = 0.5 * (lam_hi - lam_lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(b)
    r = b.copy()
    d = (Dinv @ r) / theta
    for _ in range(steps):
        x = x + d
        r = r - Ac @ d
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (Dinv @ r)
        rho = rho_new
    return x


class TwoLevel:
    """The symmetric two-level cycle for one Jacobian."""

    def __init__(self, J: sp.csr_matrix, nv: int, L: int, omega: float = OMEGA, steps: int = CHEB_STEPS,
                 ratio: float = CHEB_RATIO):
        self.J = J.tocsr()
        self.nv, self.L = nv, L
        self.omega, self.steps = omega, steps
        self.T = column_blocks(self.J, nv, L)
        self.Tinv = [np.linalg.inv(T) for T in self.T]
        self.P = prolongation(self.J, nv, L)
        self.Ac = plane_operator(self.J, self.P)
        self.Dinv = block_diag_inverse(self.Ac)
        self.lam_hi = gershgorin_bound(self.Ac, self.Dinv)
        self.lam_lo = self.lam_hi / ratio

    def smooth(self, r: np.ndarray) -> np.ndarray:
        z = np.empty_like(r)
        for a, Ti in enumerate(self.Tinv):
            d = column_dofs(self.nv, self.L, a)
            z[d] = Ti @ r[d]
        return self.omega * z

    def plane_solve(self, rc: np.ndarray) -> np.ndarray:
        return chebyshev(self.Ac, self.Dinv, rc, self.lam_lo, self.lam_hi, self.steps)

    def apply(self, r: np.ndarray) -> np.ndarray:
        z1 = self.smooth(r)
        z2 = z1 + self.P @ self.plane_solve(self.P.T @ (r - self.J @ z1))
        return z2 + self.smooth(r - self.J @ z2)


def pcg(J: sp.csr_matrix, b: np.ndarray, apply, tol: float, maxit: int = 10000):
    """Preconditioned CG from x = 0 to ||r|| <= tol ||b||; returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = apply(r)
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    for k in range(1, maxit + 1):
        q = J @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= tol * nb:
            return x, k
        z = apply(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit

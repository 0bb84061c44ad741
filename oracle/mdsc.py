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
With `TwoLevelAMG` the plane solve B_c is one V-cycle of smoothed-aggregation multigrid on A_c
(`PlaneAMG`, stated below).  Parity status: pinned by tests/test_oracle_mdsc.py (harmonic extension,
Galerkin projection, Chebyshev extremal errors, aggregation by hand, null-space preservation of the
smoothed prolongation, V-cycle symmetry and grid-independent contraction).
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


# ---------------------------------------------------------------- smoothed-aggregation plane hierarchy
# Paper Sec. 4.4 / Sec. 3.1: after the vertical semicoarsening to one layer, the plane problem is
# solved by smoothed-aggregation algebraic multigrid with a Chebyshev smoother.  Statement used here
# (Vanek, Mandel and Brezina 1996, "Algebraic multigrid by smoothed aggregation"), on 2 x 2 blocks
# (u, v per vertex):
# * aggregation of the block graph G (the sparsity pattern of A, a vertex adjacent to itself):
#   pass 1, vertices in index order: a vertex whose whole neighbourhood is still free starts a new
#   aggregate made of that neighbourhood; pass 2: every vertex still free joins the aggregate (from
#   pass 1) of its lowest-numbered neighbour that pass 1 aggregated;
# * tentative prolongation Pt: block (i, agg(i)) = I (the two translations, the near-null space of
#   the plane operator);
# * smoothed prolongation P = (I - omega D^-1 A) Pt with omega = 4 / (3 lam), lam the Gershgorin bound
#   of D^-1 A (D the 2 x 2 diagonal blocks);
# * coarse operator P^T A P (Galerkin); its pattern is the next graph;
# * coarsening stops when a level has at most AMG_COARSE vertices, when it shrinks by less than
#   AMG_MIN_RATIO, or after AMG_MAX_LEVELS levels; the coarsest level is solved exactly;
# * V-cycle: AMG_SMOOTH Chebyshev steps (block Jacobi over [lam / CHEB_RATIO, lam], from zero) as
#   pre-smoother, coarse correction, the same polynomial applied to the new residual as post-smoother
#   (symmetric positive definite for CG).

AMG_COARSE = 64
AMG_MIN_RATIO = 0.8
AMG_MAX_LEVELS = 8
AMG_SMOOTH = 3


def block_pattern(A: sp.csr_matrix) -> list:
    """Neighbour lists (sorted, a vertex included) of the 2 x 2 block graph of A (structural)."""
    A = A.tocsr()
    n = A.shape[0] // 2
    out = []
    for a in range(n):
        cols = set()
        for row in (2 * a, 2 * a + 1):
            cols.update(int(c) // 2 for c in A.indices[A.indptr[row]:A.indptr[row + 1]])
        cols.add(a)
        out.append(np.array(sorted(cols), dtype=np.int64))
    return out


def aggregate(nbrs: list) -> np.ndarray:
    """Aggregate index of every vertex (the two passes above)."""
    n = len(nbrs)
    agg = np.full(n, -1, dtype=np.int64)
    count = 0
    for a in range(n):
        if all(agg[b] < 0 for b in nbrs[a]):
            agg[nbrs[a]] = count
            count += 1
    first = agg.copy()  # pass-1 assignments
    for a in range(n):
        if agg[a] < 0:
            joined = [b for b in nbrs[a] if first[b] >= 0]
            agg[a] = first[min(joined)]
    return agg


def tentative(agg: np.ndarray) -> sp.csr_matrix:
    n = agg.shape[0]
    nc = int(agg.max()) + 1
    rows = np.arange(2 * n)
    cols = 2 * np.repeat(agg, 2) + np.tile([0, 1], n)
    return sp.csr_matrix((np.ones(2 * n), (rows, cols)), shape=(2 * n, 2 * nc))


def structural(M: sp.csr_matrix) -> sp.csr_matrix:
    """The same pattern with every stored entry 1 (explicit zeros kept)."""
    M = M.tocsr().copy()
    M.data[:] = 1.0
    return M


class AmgLevel:
    def __init__(self, A: sp.csr_matrix, nbrs: list):
        self.A = A.tocsr()
        self.nbrs = nbrs
        self.Dinv = block_diag_inverse(self.A)
        self.lam = gershgorin_bound(self.A, self.Dinv)


class PlaneAMG:
    """The smoothed-aggregation hierarchy of the plane operator and its V-cycle."""

    def __init__(self, Ac: sp.csr_matrix, nbrs0: list, smooth: int = AMG_SMOOTH):
        self.smooth = smooth
        self.levels = [AmgLevel(Ac, nbrs0)]
        self.P, self.agg = [], []
        while True:
            lv = self.levels[-1]
            n = len(lv.nbrs)
            if n <= AMG_COARSE or len(self.levels) >= AMG_MAX_LEVELS:
                break
            agg = aggregate(lv.nbrs)
            nc = int(agg.max()) + 1
            if nc > AMG_MIN_RATIO * n:
                break
            Pt = tentative(agg)
            omega = 4.0 / (3.0 * lv.lam)
            P = (Pt - omega * (lv.Dinv @ (lv.A @ Pt))).tocsr()
            # pattern: structural product (no entry dropped where values cancel)
            Ppat = structural(Pt + structural(lv.Dinv) @ structural(lv.A) @ Pt)
            P = (P + 0.0 * Ppat).tocsr()
            P.sort_indices()
            Anext = (P.T @ lv.A @ P).tocsr()
            Apat = structural(structural(P).T @ structural(lv.A) @ structural(P))
            Anext = (Anext + 0.0 * Apat).tocsr()
            Anext.sort_indices()
            self.P.append(P)
            self.agg.append(agg)
            self.levels.append(AmgLevel(Anext, block_pattern(Anext)))
        self.coarse = self.levels[-1].A.toarray()

    def sizes(self):
        return [len(lv.nbrs) for lv in self.levels]

    def vcycle(self, b: np.ndarray, k: int = 0) -> np.ndarray:
        lv = self.levels[k]
        if k == len(self.levels) - 1:
            return np.linalg.solve(self.coarse, b)
        lo = lv.lam / CHEB_RATIO
        x = chebyshev(lv.A, lv.Dinv, b, lo, lv.lam, self.smooth)
        P = self.P[k]
        x = x + P @ self.vcycle(P.T @ (b - lv.A @ x), k + 1)
        return x + chebyshev(lv.A, lv.Dinv, b - lv.A @ x, lo, lv.lam, self.smooth)


def plane_neighbours(nv: int, tri: np.ndarray) -> list:
    """Closed neighbourhoods of the base vertices (the pattern of the plane operator)."""
    nb = [set([a]) for a in range(nv)]
    for t in tri:
        for a in t:
            nb[int(a)].update(int(x) for x in t)
    return [np.array(sorted(s), dtype=np.int64) for s in nb]


class TwoLevelAMG(TwoLevel):
    """The semicoarsening cycle of TwoLevel with the plane problem solved by one SA-AMG V-cycle."""

    def __init__(self, J: sp.csr_matrix, nv: int, L: int, tri: np.ndarray, omega: float = OMEGA,
                 smooth: int = AMG_SMOOTH):
        super().__init__(J, nv, L, omega=omega)
        self.amg = PlaneAMG(self.Ac, plane_neighbours(nv, tri), smooth)

    def plane_solve(self, rc: np.ndarray) -> np.ndarray:
        return self.amg.vcycle(rc)

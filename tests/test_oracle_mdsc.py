"""Pins of the oracle's MDSC two-level preconditioner (paper Sec. 4.4), on CPU.

Each pin checks a property that a plausible mistake breaks: the harmonic extension (a wrong column
block or sign), the Galerkin plane operator (a transposed product), the Chebyshev recurrence (any
wrong coefficient changes the error at the extremal points of the Chebyshev polynomial), and the
symmetry / positivity of the whole cycle that CG needs."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import mdsc
from paper_2204_04321_b300 import synth


@pytest.fixture(scope="module")
def system():
    mesh = synth.dome_mesh(10, 4, 51, 52, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    J, R = om.jacobian_scipy(om.sia())
    return mesh, J.tocsr(), R


def test_prolongation_is_the_harmonic_extension_of_the_top_level(system):
    mesh, J, _ = system
    L = mesh.nlayers
    P = mdsc.prolongation(J, mesh.nv, L).toarray()
    for a in range(0, mesh.nv, 5):
        d = mdsc.column_dofs(mesh.nv, L, a)
        Pa = P[d][:, 2 * a:2 * a + 2]
        assert np.allclose(Pa[2 * L:], np.eye(2), atol=0)           # top level: identity
        T = J[d][:, d].toarray()
        # the column rows below the top are satisfied with zero right-hand side
        assert np.abs((T @ Pa)[:2 * L]).max() <= 1e-12 * np.abs(T).max()
        # and P touches no other column
        assert np.count_nonzero(np.delete(P[d], [2 * a, 2 * a + 1], axis=1)) == 0


def test_galerkin_coarse_correction_is_a_J_orthogonal_projection(system):
    """E = I - P A_c^-1 P^T J with A_c = P^T J P: E E = E and J E symmetric.  A plane operator formed
    any other way (P J P^T, a dropped block) breaks both."""
    mesh, J, _ = system
    P = mdsc.prolongation(J, mesh.nv, mesh.nlayers)
    Ac = mdsc.plane_operator(J, P).toarray()
    Pd, Jd = P.toarray(), J.toarray()
    E = np.eye(Jd.shape[0]) - Pd @ np.linalg.solve(Ac, Pd.T @ Jd)
    assert np.abs(E @ E - E).max() <= 1e-8
    JE = Jd @ E
    assert np.abs(JE - JE.T).max() <= 1e-8 * np.abs(Jd).max()


@pytest.mark.parametrize("k", [1, 3, 8])
def test_chebyshev_error_at_the_extremal_points_is_one_over_Tk(k):
    """For A = diag(lambda) with lambda at the extrema of the shifted Chebyshev polynomial, the
    semi-iterative error after k steps is exactly T_k(sigma)^-1 times the initial error in every
    component (sigma = theta / delta): a textbook identity that every recurrence coefficient
    enters."""
    lo, hi = 0.05, 2.0
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    lam = theta + delta * np.cos(np.arange(k + 1) * np.pi / k)
    A = sp.diags(lam).tocsr()
    I = sp.identity(k + 1, format="csr")
    b = np.linspace(1.0, 2.0, k + 1)
    x = mdsc.chebyshev(A, I, b, lo, hi, k)
    e0 = b / lam
    ratio = np.abs((e0 - x) / e0)
    Tk = np.cosh(k * np.arccosh(theta / delta))
    assert np.allclose(ratio, 1.0 / Tk, rtol=1e-9, atol=0)


def test_chebyshev_one_step_is_scaled_jacobi():
    rng = np.random.default_rng(3)
    M = rng.normal(size=(6, 6))
    A = sp.csr_matrix(M @ M.T + 6 * np.eye(6))
    Dinv = sp.diags(1.0 / A.diagonal()).tocsr()
    b = rng.normal(size=6)
    x = mdsc.chebyshev(A, Dinv, b, 0.1, 3.0, 1)
    assert np.allclose(x, (Dinv @ b) / 1.55, rtol=1e-14)


def test_cycle_is_symmetric_positive_definite(system):
    mesh, J, _ = system
    tl = mdsc.TwoLevel(J, mesh.nv, mesh.nlayers)
    rng = np.random.default_rng(5)
    for _ in range(4):
        x, y = rng.normal(size=J.shape[0]), rng.normal(size=J.shape[0])
        xy, yx = x @ tl.apply(y), y @ tl.apply(x)
        assert abs(xy - yx) <= 1e-10 * (abs(xy) + abs(yx))
        assert x @ tl.apply(x) > 0


def test_gershgorin_bound_covers_the_spectrum(system):
    mesh, J, _ = system
    tl = mdsc.TwoLevel(J, mesh.nv, mesh.nlayers)
    ev = np.linalg.eigvals((tl.Dinv @ tl.Ac).toarray()).real
    assert ev.max() <= tl.lam_hi * (1 + 1e-12) and ev.min() > 0


def test_mdsc_takes_fewer_cg_iterations_than_the_column_solve():
    mesh = synth.dome_mesh(24, 5, 51, 52, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    J, R = om.jacobian_scipy(om.sia())
    tl = mdsc.TwoLevel(J, mesh.nv, mesh.nlayers)
    x, km = mdsc.pcg(J, -R, tl.apply, 1e-6)
    _, kc = mdsc.pcg(J, -R, lambda r: tl.smooth(r) / tl.omega, 1e-6)
    assert np.linalg.norm(J @ x + R) <= 1e-6 * np.linalg.norm(R)
    assert km <= 0.7 * kc, (km, kc)


# ---------------------------------------------------------------- smoothed-aggregation plane hierarchy

def _grid_laplacian(n, shift=0.0):
    """2D 5-point graph Laplacian on an n x n grid, times I_2 (u and v), plus shift * I."""
    N = n * n
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in range(n):
            a = i * n + j
            deg = 0
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n:
                    b = ii * n + jj
                    rows.append(a), cols.append(b), vals.append(-1.0)
                    deg += 1
            rows.append(a), cols.append(a), vals.append(deg + shift)
    Ls = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    return sp.kron(Ls, sp.identity(2), format="csr")


def test_aggregation_of_a_path_graph_by_hand():
    # path 0-1-2-3-4-5-6: roots 0 ({0,1}), 3 ({2,3,4}), 6 ({5,6}); nobody is left for pass 2
    nbrs = [np.array(sorted({max(0, a - 1), a, min(6, a + 1)})) for a in range(7)]
    assert list(mdsc.aggregate(nbrs)) == [0, 0, 1, 1, 1, 2, 2]
    # a star whose centre is taken by the first leaf's neighbourhood: the other leaves join it in pass 2
    nbrs = [np.array([0, 1]), np.array([0, 1, 2, 3]), np.array([1, 2]), np.array([1, 3])]
    assert list(mdsc.aggregate(nbrs)) == [0, 0, 0, 0]


def test_aggregation_covers_every_vertex_with_disjoint_root_neighbourhoods():
    nbrs = mdsc.plane_neighbours(*(lambda m: (m.nv, m.tri))(synth.dome_mesh(20, 1, 3, 4)))
    agg = mdsc.aggregate(nbrs)
    assert agg.min() == 0 and len(np.unique(agg)) == agg.max() + 1
    for a, nb in enumerate(nbrs):   # every vertex sits next to (or in) a vertex of its own aggregate
        assert any(agg[b] == agg[a] for b in nb if b != a) or len(nb) == 1


def test_smoothed_prolongation_keeps_the_translations_of_a_singular_operator():
    """For A with the two translations in its null space (a graph Laplacian times I_2), the tentative
    prolongation reproduces them and smoothing (I - omega D^-1 A) keeps them exactly; the Galerkin
    operator then has them in its null space too."""
    A = _grid_laplacian(12)
    lv = mdsc.AmgLevel(A, mdsc.block_pattern(A))
    agg = mdsc.aggregate(lv.nbrs)
    Pt = mdsc.tentative(agg)
    nc = agg.max() + 1
    for c in range(2):
        e = np.zeros(2 * nc)
        e[c::2] = 1.0
        t = np.zeros(A.shape[0])
        t[c::2] = 1.0
        assert np.array_equal(Pt @ e, t)
        P = Pt - (4.0 / (3.0 * lv.lam)) * (lv.Dinv @ (A @ Pt))
        assert np.abs(P @ e - t).max() <= 1e-14
        assert np.abs((P.T @ A @ P) @ e).max() <= 1e-12


def test_vcycle_is_symmetric_positive_definite_and_contracts_independently_of_the_grid():
    rates = []
    for n in (16, 32):
        A = _grid_laplacian(n, shift=1e-3)
        amg = mdsc.PlaneAMG(A, mdsc.block_pattern(A))
        assert len(amg.sizes()) >= 2 and amg.sizes()[-1] <= mdsc.AMG_COARSE
        rng = np.random.default_rng(n)
        x, y = rng.normal(size=A.shape[0]), rng.normal(size=A.shape[0])
        xy, yx = x @ amg.vcycle(y), y @ amg.vcycle(x)
        assert abs(xy - yx) <= 1e-10 * (abs(xy) + abs(yx))
        assert x @ amg.vcycle(x) > 0
        # as a stationary solver: the error shrinks by a grid-independent factor per cycle
        b = rng.normal(size=A.shape[0])
        u = np.zeros_like(b)
        rn = [np.linalg.norm(b)]
        for _ in range(6):
            u = u + amg.vcycle(b - A @ u)
            rn.append(np.linalg.norm(b - A @ u))
        rate = (rn[-1] / rn[1]) ** (1 / 5)
        assert rate < 0.45, (n, rate)
        rates.append(rate)
        for lv, P in zip(amg.levels[1:], amg.P):   # Galerkin operators stay SPD
            ev = np.linalg.eigvalsh(lv.A.toarray())
            assert ev.min() > 0
    assert rates[1] <= 1.15 * rates[0]   # four times the unknowns, (nearly) the same contraction


def test_mdsc_with_amg_plane_solve_is_spd_and_solves(system):
    mesh, J, R = system
    tl = mdsc.TwoLevelAMG(J, mesh.nv, mesh.nlayers, mesh.tri)
    rng = np.random.default_rng(6)
    for _ in range(3):
        x, y = rng.normal(size=J.shape[0]), rng.normal(size=J.shape[0])
        xy, yx = x @ tl.apply(y), y @ tl.apply(x)
        assert abs(xy - yx) <= 1e-10 * (abs(xy) + abs(yx))
        assert x @ tl.apply(x) > 0
    x, k = mdsc.pcg(J, -R, tl.apply, 1e-8)
    assert np.linalg.norm(J @ x + R) <= 1e-8 * np.linalg.norm(R)

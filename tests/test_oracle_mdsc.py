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

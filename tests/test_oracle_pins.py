"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test ties one part of the oracle to a fact that does not come from the oracle itself:
closed forms, invariants of the basis, finite differences, Glen's law in simple shear and
the exact first-order solution for an inclined slab.  A plausible slip in the oracle (a
dropped term, a wrong sign, a transposed index, a wrong measure) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.optimize

import oracle
from paper_2204_04321_b300 import synth


def tiny_mesh(m=2, L=2, seed=5, bed="sinusoidal", H0=1500.0, half_width=3e3, delta=1e-10):
    xy, tri = synth.jittered_grid(m, seed, half_width=half_width)
    rng = np.random.default_rng(seed + 1)
    thick = rng.uniform(300.0, 900.0, size=xy.shape[0])
    b = rng.uniform(-100.0, 100.0, size=xy.shape[0]) if bed == "sinusoidal" else np.zeros(xy.shape[0])
    beta = rng.uniform(200.0, 2000.0, size=xy.shape[0])
    mesh = synth.Mesh(xy=xy, tri=tri, bed=b, thick=thick, beta=beta,
                      sigma=np.sort(np.concatenate([[0.0, 1.0], rng.uniform(0.1, 0.9, L - 1)])),
                      name="tiny")
    mesh.params.delta = delta
    return mesh


def random_wedge(rng):
    """Wedge with vertical edges, non-parallel (tilted) bottom and top faces."""
    x = rng.uniform(-1e3, 1e3, 3)
    y = rng.uniform(-1e3, 1e3, 3)
    if (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]) < 0:
        x[[1, 2]] = x[[2, 1]]
        y[[1, 2]] = y[[2, 1]]
    zb = rng.uniform(-50.0, 50.0, 3)
    zt = zb + rng.uniform(50.0, 400.0, 3)
    X = np.zeros((6, 3))
    X[:3, 0] = X[3:, 0] = x
    X[:3, 1] = X[3:, 1] = y
    X[:3, 2] = zb
    X[3:, 2] = zt
    return X


REF_NODES = [(0, 0, -1), (1, 0, -1), (0, 1, -1), (0, 0, 1), (1, 0, 1), (0, 1, 1)]


# ------------------------------------------------------------------ basis (Sec. 3.1, low-order prismatic)

def test_basis_kronecker_property():
    rng = np.random.default_rng(0)
    X = random_wedge(rng)
    for j, (xi, eta, zeta) in enumerate(REF_NODES):
        N, _, _ = oracle.basis_at(X, xi, eta, zeta)
        np.testing.assert_allclose(N, np.eye(6)[j], atol=1e-15)


def test_basis_partition_of_unity_and_zero_gradient_sum():
    rng = np.random.default_rng(1)
    for _ in range(20):
        X = random_wedge(rng)
        for q in range(6):
            xi, eta, zeta, _ = oracle.quadrature_point(q)
            N, gN, det = oracle.basis_at(X, xi, eta, zeta)
            assert det > 0
            assert abs(N.sum() - 1.0) < 1e-14
            scale = np.abs(gN).max()
            assert np.abs(gN.sum(axis=0)).max() < 1e-13 * scale


def test_basis_gradient_reproduces_linear_fields():
    """sum_i f(X_i) grad N_i = grad f for every affine f (iso-parametric map of an extruded wedge)."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        X = random_wedge(rng)
        g = rng.normal(size=3)
        c = rng.normal()
        f = c + X @ g
        for xi, eta, zeta in rng.uniform(0.0, 0.5, size=(5, 3)):
            _, gN, _ = oracle.basis_at(X, xi, eta, 2 * zeta - 0.5)
            np.testing.assert_allclose(f @ gN, g, rtol=1e-10, atol=1e-12 * np.abs(g).max())


def test_quadrature_volume_is_exact_wedge_volume():
    """Sum_q w_q det J_q = area * (h0 + h1 + h2) / 3 (volume of a wedge with vertical edges, planar faces)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        X = random_wedge(rng)
        vol = 0.0
        for q in range(6):
            xi, eta, zeta, w = oracle.quadrature_point(q)
            vol += w * oracle.basis_at(X, xi, eta, zeta)[2]
        x, y = X[:3, 0], X[:3, 1]
        area = 0.5 * ((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]))
        h = X[3:, 2] - X[:3, 2]
        assert vol == pytest.approx(area * h.mean(), rel=1e-13)


def test_quadrature_rule_weights():
    pts = [oracle.quadrature_point(q) for q in range(6)]
    assert sum(p[3] for p in pts) == pytest.approx(1.0)       # ref wedge volume = 1/2 * 2
    zs = sorted({round(p[2], 15) for p in pts})
    assert zs == pytest.approx([-1 / math.sqrt(3), 1 / math.sqrt(3)])


# ------------------------------------------------------------------ strain rate and viscosity (Sec. 2)

def linear_velocity(mesh, G, c):
    """u = c0 + G[0] . x, v = c1 + G[1] . x at every node (x = (x, y, z))."""
    L = mesh.nlayers
    U = np.empty(mesh.ndof)
    for l in range(L + 1):
        z = mesh.bed + mesh.sigma[l] * mesh.thick
        X = np.stack([mesh.xy[:, 0], mesh.xy[:, 1], z], 1)
        for comp in range(2):
            U[mesh.dof(np.arange(mesh.nv), l, comp)] = c[comp] + X @ G[comp]
    return U


def test_linear_velocity_gives_exact_constant_gradient():
    mesh = tiny_mesh(m=3, L=3)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(4)
    G = rng.normal(scale=1e-2, size=(2, 3))
    U = linear_velocity(mesh, G, c=[3.0, -2.0])
    for t in range(mesh.ntri):
        for l in range(mesh.nlayers):
            for q in range(6):
                st = om.qp_state(U, t, l, q)
                np.testing.assert_allclose(st["grad_u"], G[0], rtol=1e-9, atol=1e-13)
                np.testing.assert_allclose(st["grad_v"], G[1], rtol=1e-9, atol=1e-13)


def test_effective_strain_rate_is_second_invariant_of_incompressible_tensor():
    """eps_e^2 = (1/2) eps_ij eps_ij of the full strain-rate tensor with eps_zz = -(u_x + v_y)
    (incompressibility) and the first-order shear terms eps_xz = u_z/2, eps_yz = v_z/2."""
    mesh = tiny_mesh(m=2, L=2)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(21)
    for _ in range(10):
        G = rng.normal(scale=1e-2, size=(2, 3))
        st = om.qp_state(linear_velocity(mesh, G, [0.0, 0.0]), 2, 1, 1)
        (ux, uy, uz), (vx, vy, vz) = G
        E = np.array([[ux, 0.5 * (uy + vx), 0.5 * uz],
                      [0.5 * (uy + vx), vy, 0.5 * vz],
                      [0.5 * uz, 0.5 * vz, -(ux + vy)]])
        assert st["eps2"] == pytest.approx(0.5 * np.sum(E * E), rel=1e-9)


@pytest.mark.parametrize("kind", ["xz", "yz", "xy"])
def test_glen_flow_law_in_simple_shear(kind):
    """Simple shear: the shear strain rate equals A tau^n with tau = 2 mu eps (Glen's law, delta = 0)."""
    mesh = tiny_mesh(m=2, L=2, delta=0.0)
    om = oracle.OracleMesh(mesh)
    gam = 3e-2
    G = np.zeros((2, 3))
    if kind == "xz":
        G[0, 2] = gam        # u = gam z: eps_xz = gam / 2
    elif kind == "yz":
        G[1, 2] = gam
    else:
        G[0, 1] = gam        # u = gam y: eps_xy = gam / 2
    U = linear_velocity(mesh, G, c=[0.0, 0.0])
    st = om.qp_state(U, 1, 0, 2)
    eps = gam / 2.0
    tau = 2.0 * st["mu"] * eps
    assert eps == pytest.approx(mesh.params.A * tau ** 3, rel=1e-12)
    assert st["eps2"] == pytest.approx(eps ** 2, rel=1e-12)


def test_glen_flow_law_pure_stretching():
    """Uniaxial plane stretching u = g x (v = 0): eps_e^2 = g^2, deviatoric xx stress 2 mu (2 exx + eyy)
    equals 2 A^(-1/3) g^(1/3) (Glen's law with the first-order eps_1 convention)."""
    mesh = tiny_mesh(m=2, L=2, delta=0.0)
    om = oracle.OracleMesh(mesh)
    g = 2e-3
    G = np.zeros((2, 3))
    G[0, 0] = g
    st = om.qp_state(linear_velocity(mesh, G, [0.0, 0.0]), 0, 1, 4)
    assert st["eps2"] == pytest.approx(g * g, rel=1e-12)
    A = mesh.params.A
    assert 2 * st["mu"] * 2 * g == pytest.approx(2 * A ** (-1 / 3) * g ** (1 / 3), rel=1e-12)


# ------------------------------------------------------------------ residual closed forms

def _tri_area(xy, tri):
    p = xy[tri]
    return 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                  - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))


def _p1_grad(xy, tri, f):
    p = xy[tri]
    ax, ay = p[:, 1, 0] - p[:, 0, 0], p[:, 1, 1] - p[:, 0, 1]
    bx, by = p[:, 2, 0] - p[:, 0, 0], p[:, 2, 1] - p[:, 0, 1]
    det = ax * by - ay * bx
    d1, d2 = f[tri[:, 1]] - f[tri[:, 0]], f[tri[:, 2]] - f[tri[:, 0]]
    return (d1 * by - d2 * ay) / det, (ax * d2 - bx * d1) / det


def closed_form_constant_velocity_residual(mesh, c):
    """R for U = const (c_u, c_v): no strain, so R = driving + basal friction, both in closed form.

    Driving: rho g grad s . int N_{a,k}; over a wedge with vertical edges,
             int lambda_a psi_k dV = (1/2) int lambda_a h dA = A_t/24 (h_a + sum_b h_b).
    Friction: beta linear on the (planar) basal face of true area A_f:
             int beta lambda_a dGamma = A_f/12 (beta_a + sum_b beta_b).
    """
    R = np.zeros(mesh.ndof)
    tri = mesh.tri
    area = _tri_area(mesh.xy, tri)
    s = mesh.bed + mesh.thick
    sx, sy = _p1_grad(mesh.xy, tri, s)
    rg = mesh.params.rho * mesh.params.g
    for l in range(mesh.nlayers):
        h = (mesh.sigma[l + 1] - mesh.sigma[l]) * mesh.thick[tri]          # [T, 3]
        intN = area[:, None] / 24.0 * (h + h.sum(1, keepdims=True))         # same for bottom and top
        for k in (0, 1):
            for a in range(3):
                np.add.at(R, mesh.dof(tri[:, a], l + k, 0), rg * sx * intN[:, a])
                np.add.at(R, mesh.dof(tri[:, a], l + k, 1), rg * sy * intN[:, a])
    # true area of the basal triangle
    P = np.stack([mesh.xy[tri][..., 0], mesh.xy[tri][..., 1], mesh.bed[tri]], -1)
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    Af = 0.5 * np.linalg.norm(cr, axis=1)
    bt = mesh.beta[tri]
    for a in range(3):
        ib = Af / 12.0 * (bt[:, a] + bt.sum(1))
        np.add.at(R, mesh.dof(tri[:, a], 0, 0), ib * c[0])
        np.add.at(R, mesh.dof(tri[:, a], 0, 1), ib * c[1])
    return R


@pytest.mark.parametrize("c", [(0.0, 0.0), (37.0, -12.5)])
def test_constant_velocity_residual_closed_form(c):
    mesh = tiny_mesh(m=4, L=3)
    om = oracle.OracleMesh(mesh)
    U = np.empty(mesh.ndof)
    U[0::2], U[1::2] = c
    R = om.residual(U)
    Rc = closed_form_constant_velocity_residual(mesh, c)
    assert np.abs(R - Rc).max() <= 1e-12 * np.abs(Rc).max()


def test_global_force_balance():
    """Sum over nodes of R^u = int rho g s_x dV + int_bed beta u dGamma (stress terms sum to zero)."""
    mesh = tiny_mesh(m=4, L=3)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(9)
    U = rng.uniform(-100, 100, mesh.ndof)
    R = om.residual(U)
    tri = mesh.tri
    area = _tri_area(mesh.xy, tri)
    sx, sy = _p1_grad(mesh.xy, tri, mesh.bed + mesh.thick)
    vol = area * mesh.thick[tri].mean(1)
    rg = mesh.params.rho * mesh.params.g
    P = np.stack([mesh.xy[tri][..., 0], mesh.xy[tri][..., 1], mesh.bed[tri]], -1)
    Af = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    bt = mesh.beta[tri]
    for comp, g in ((0, sx), (1, sy)):
        ub = U[mesh.dof(tri, 0, comp)]
        # int of the product of two linear functions over a triangle: A/12 (sum_a b_a u_a + sum_a b_a sum_b u_b)
        fric = Af / 12.0 * ((bt * ub).sum(1) + bt.sum(1) * ub.sum(1))
        expected = (rg * g * vol).sum() + fric.sum()
        scale = np.abs(R[comp::2]).sum()
        assert abs(R[comp::2].sum() - expected) <= 1e-11 * scale


# ------------------------------------------------------------------ energy and derivatives

def test_residual_is_gradient_of_energy():
    mesh = tiny_mesh(m=2, L=2)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(11)
    U = rng.uniform(-100, 100, mesh.ndof)
    R = om.residual(U)
    for j in rng.choice(mesh.ndof, 12, replace=False):
        h = 1e-3 * max(1.0, abs(U[j]))
        Up, Um = U.copy(), U.copy()
        Up[j] += h
        Um[j] -= h
        fd = (om.energy(Up) - om.energy(Um)) / (2 * h)
        assert fd == pytest.approx(R[j], rel=1e-6, abs=1e-9 * np.abs(R).max())


def _dense(om, U):
    J, R = om.jacobian_scipy(U)
    return J.toarray(), R


def test_jacobian_matches_central_differences():
    mesh = tiny_mesh(m=2, L=2)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(12)
    U = rng.uniform(-100, 100, mesh.ndof)
    J, R0 = _dense(om, U)
    np.testing.assert_allclose(R0, om.residual(U), rtol=0, atol=1e-12 * np.abs(R0).max())
    FD = np.empty_like(J)
    for j in range(mesh.ndof):
        h = 1e-6 * max(1.0, abs(U[j]))
        Up, Um = U.copy(), U.copy()
        Up[j] += h
        Um[j] -= h
        FD[:, j] = (om.residual(Up) - om.residual(Um)) / (2 * h)
    assert np.abs(FD - J).max() <= 1e-7 * np.abs(J).max()


def test_jacobian_symmetric_positive_definite():
    """J is the Hessian of a convex energy: symmetric, and positive definite with beta > 0."""
    mesh = tiny_mesh(m=2, L=3)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(13)
    for U in (rng.uniform(-100, 100, mesh.ndof), np.zeros(mesh.ndof)):
        J, _ = _dense(om, U)
        assert np.abs(J - J.T).max() <= 1e-13 * np.abs(J).max()
        np.linalg.cholesky(J)


def test_element_jacobian_matches_global_assembly():
    mesh = tiny_mesh(m=2, L=2)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(14)
    U = rng.uniform(-100, 100, mesh.ndof)
    J = np.zeros((mesh.ndof, mesh.ndof))
    R = np.zeros(mesh.ndof)
    for t in range(mesh.ntri):
        for l in range(mesh.nlayers):
            Re, Ke = om.element(U, t, l)
            d = np.array([mesh.dof(mesh.tri[t, a], l + k, c) for k in (0, 1) for a in range(3)
                          for c in (0, 1)])
            J[np.ix_(d, d)] += Ke
            R[d] += Re
    Jg, Rg = _dense(om, U)
    assert np.abs(J - Jg).max() <= 1e-13 * np.abs(Jg).max()
    assert np.abs(R - Rg).max() <= 1e-13 * np.abs(Rg).max()


# ------------------------------------------------------------------ pattern

def test_pattern_matches_definition_and_closed_form_count():
    """Columns of row (a, l, c): all (b, l', c') with b == a or b ~ a in the base mesh, |l - l'| <= 1."""
    mesh = tiny_mesh(m=3, L=3)
    om = oracle.OracleMesh(mesh)
    rowptr, colidx = om.pattern()
    assert colidx.shape[0] == mesh.expected_nnz()
    nbr = {a: {a} for a in range(mesh.nv)}
    for t in mesh.tri:
        for a in t:
            nbr[int(a)].update(int(b) for b in t)
    L = mesh.nlayers
    for a in range(mesh.nv):
        for l in range(L + 1):
            for c in (0, 1):
                r = mesh.dof(a, l, c)
                want = sorted(int(mesh.dof(b, lp, cp)) for b in nbr[a]
                              for lp in range(max(0, l - 1), min(L, l + 1) + 1) for cp in (0, 1))
                assert list(colidx[rowptr[r]:rowptr[r + 1]]) == want


def test_small_config_pattern_size():
    mesh = synth.config_small()
    assert (mesh.ntri, mesh.nv, mesh.nwedges, mesh.ndof) == (2048, 1089, 10240, 13068)
    assert mesh.expected_nnz() == 471104


# ------------------------------------------------------------------ inclined slab (exact FO solution)

def slab_exact(alpha, H, beta, A, rho, g, delta):
    """Exact first-order solution u(d), d = depth below the surface, for an infinite slab of slope alpha.

    With u = f(d): exx = alpha f', exz = -f'/2, so eps_e^2 = f'^2 (1 + 4 alpha^2)/4 and the x-momentum
    equation integrates to mu f' = rho g alpha d / (1 + 4 alpha^2) (stress-free surface).  The bed
    traction 2 mu eps_1 . n = rho g alpha H / sqrt(1 + alpha^2) fixes u(H) = -rho g alpha H /(beta sqrt(1+alpha^2)).
    f' is found pointwise by a bracketing root solve and integrated by adaptive quadrature.
    """
    k = (1.0 + 4 * alpha ** 2) / 4.0
    rg = rho * g

    def fprime(d):
        M = rg * alpha * d / (1.0 + 4 * alpha ** 2)
        if M == 0.0:
            return 0.0
        phi = lambda y: 0.5 * A ** (-1 / 3) * y * (k * y * y + delta) ** (-1 / 3) - M
        hi = 1.0
        while phi(hi) < 0:
            hi *= 2.0
        return scipy.optimize.brentq(phi, 0.0, hi, xtol=1e-300, rtol=1e-15, maxiter=500)

    ub = -rg * alpha * H / (beta * math.sqrt(1.0 + alpha ** 2))

    def u(d):
        val, _ = scipy.integrate.quad(fprime, d, H, epsabs=0, epsrel=1e-13, limit=200)
        return ub - val

    return u


def slab_residual_error(L, alpha=0.02, H=1000.0, beta=500.0, delta=1e-4, m=4):
    """(max over levels 1..L of |R_i| / own load, max at the bed of |R_i| / column load)."""
    mesh = synth.slab_mesh(m, L, slope=alpha, thickness=H, beta=beta, half_width=10e3, jitter=0.2)
    mesh.params.delta = delta
    p = mesh.params
    u = slab_exact(alpha, H, beta, p.A, p.rho, p.g, delta)
    U = np.zeros(mesh.ndof)
    for l in range(L + 1):
        U[mesh.dof(np.arange(mesh.nv), l, 0)] = u((1.0 - mesh.sigma[l]) * H)
    om = oracle.OracleMesh(mesh)
    R = om.residual(U)
    load = np.abs(om.residual(np.zeros(mesh.ndof)))
    ij = np.stack(np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="xy"), -1).reshape(-1, 2)
    interior = np.where((ij[:, 0] > 0) & (ij[:, 0] < m) & (ij[:, 1] > 0) & (ij[:, 1] < m))[0]
    column_load = sum(load[mesh.dof(interior, l, 0)] for l in range(L + 1))
    e_levels = 0.0
    for l in range(1, L + 1):
        du, dv = mesh.dof(interior, l, 0), mesh.dof(interior, l, 1)
        e_levels = max(e_levels, np.max(np.abs(R[du]) / load[du]), np.max(np.abs(R[dv]) / load[du]))
    d0u, d0v = mesh.dof(interior, 0, 0), mesh.dof(interior, 0, 1)
    e_bed = max(np.max(np.abs(R[d0u]) / column_load), np.max(np.abs(R[d0v]) / column_load))
    return e_levels, e_bed


def test_inclined_slab_residual_consistency_second_order():
    """The nodal residual of the exact slab profile vanishes at O(dz^2): at levels 1..L relative to
    the node's own load, at the bed (one element only, Robin term) relative to the column's load."""
    e = np.array([slab_residual_error(L) for L in (8, 16, 32)])
    assert e[2, 0] < 5e-3 and e[2, 1] < 1e-3, e
    assert np.all(e[0] / e[1] > 3.0) and np.all(e[1] / e[2] > 3.0), e


def test_sia_guess_matches_slab_solution_at_small_slope():
    """On a slab, the shallow-ice + sliding guess equals the exact profile up to O(alpha^2)."""
    alpha, H, beta = 1e-3, 800.0, 2e3
    mesh = synth.slab_mesh(3, 6, slope=alpha, thickness=H, beta=beta)
    mesh.params.delta = 0.0
    p = mesh.params
    U = oracle.OracleMesh(mesh).sia()
    rg = p.rho * p.g
    for l in range(mesh.nlayers + 1):
        d = (1 - mesh.sigma[l]) * H
        u_exact = -rg * alpha * H / (beta * math.sqrt(1 + alpha ** 2)) \
            - p.A / 2 * (rg * alpha) ** 3 * (H ** 4 - d ** 4) / (1 + 4 * alpha ** 2) ** 2
        got = U[mesh.dof(np.arange(mesh.nv), l, 0)]
        np.testing.assert_allclose(got, u_exact, rtol=5 * alpha ** 2)
        assert np.abs(U[mesh.dof(np.arange(mesh.nv), l, 1)]).max() <= 1e-12 * abs(u_exact)


# ------------------------------------------------------------------ Newton (plain, sparse direct)

def test_oracle_newton_converges_quadratically_to_unique_minimiser():
    from oracle.newton import newton
    mesh = tiny_mesh(m=3, L=3)
    om = oracle.OracleMesh(mesh)
    U1, info1 = newton(om, np.zeros(mesh.ndof), rtol=1e-10)
    U2, info2 = newton(om, om.sia(), rtol=1e-10)
    assert info1["converged"] and info2["converged"]
    assert np.abs(U1 - U2).max() <= 1e-6 * np.abs(U1).max()
    h = info1["history"]
    # quadratic tail: the last reduction is at least the square of the previous ratio (loosely)
    assert h[-1] <= 1e-10 and h[-1] <= 10 * h[-2] ** 1.5


# ------------------------------------------------------------------ ocean margin condition (Sec. 2, lateral BC)

def _margin(mesh, rho_w):
    mesh.params.margin = 1
    mesh.params.rho_w = rho_w
    return mesh


@pytest.mark.parametrize("m,L", [(2, 2), (5, 3)])
def test_margin_cryostatic_load_balances_driving_stress_on_flat_bed(m, L):
    """With rho_w = 0 the margin load is -int rho g (s - z) n_c N_i.  At U = 0 (no stress, no
    friction) the residual is the load, and its sum over nodes is the total force
    int rho g grad s dV - oint_lateral rho g (s - z) n dGamma, which the divergence theorem sets to
    zero on a flat bed (s - z vanishes on the surface, n_c on the bed): the pin checks the face
    geometry, the outward normal, the sign and the rule (exact here) against the volume term."""
    mesh = _margin(tiny_mesh(m=m, L=L, bed="flat"), 0.0)
    om = oracle.OracleMesh(mesh)
    R = om.residual(np.zeros(mesh.ndof))
    mesh.params.margin = 0
    drive = oracle.OracleMesh(mesh).residual(np.zeros(mesh.ndof))
    for c in (0, 1):
        assert abs(R[c::2].sum()) <= 1e-12 * np.abs(drive[c::2]).sum()
        assert np.abs(drive[c::2].sum()) > 1e-3 * np.abs(drive[c::2]).sum()  # the driving force is not zero


@pytest.mark.parametrize("bed,rho_w", [(100.0, 1028.0), (-1500.0, 1028.0), (-1500.0, 0.0)])
def test_margin_side_force_of_a_slab_closed_form(bed, rho_w):
    """Slab of constant thickness on a flat bed at `bed` (all above, or all below sea level): the
    x-force on the side x = +W is -2W (rho g H^2 / 2 - rho_w g int_b^s max(-z, 0) dz); nodes of that
    side receive it all (the y-sides have n_x = 0) and the interior none (grad s = 0)."""
    H = 1000.0
    mesh = synth.slab_mesh(4, 3, slope=0.0, thickness=H, beta=1e3, half_width=5e3, jitter=0.0)
    mesh.bed = np.full(mesh.nv, bed)
    _margin(mesh, rho_w)
    R = oracle.OracleMesh(mesh).residual(np.zeros(mesh.ndof))
    s = bed + H
    rg, wg = mesh.params.rho * mesh.params.g, rho_w * mesh.params.g
    submerged = (max(-bed, 0.0) ** 2 - max(-s, 0.0) ** 2) / 2.0  # int_b^s max(-z, 0) dz
    expected = -2 * 5e3 * (rg * H * H / 2.0 - wg * submerged)
    right = np.abs(mesh.xy[:, 0] - 5e3) < 1e-6
    rows = np.concatenate([mesh.dof(np.nonzero(right)[0], l, 0) for l in range(mesh.nlayers + 1)])
    assert R[rows].sum() == pytest.approx(expected, rel=1e-12)
    left = np.abs(mesh.xy[:, 0] + 5e3) < 1e-6
    rows_l = np.concatenate([mesh.dof(np.nonzero(left)[0], l, 0) for l in range(mesh.nlayers + 1)])
    assert R[rows_l].sum() == pytest.approx(-expected, rel=1e-12)   # opposite normal
    inner = ~(right | left)
    rows_i = np.concatenate([mesh.dof(np.nonzero(inner)[0], l, 0) for l in range(mesh.nlayers + 1)])
    assert np.abs(R[rows_i]).max() <= 1e-9 * abs(expected)


def test_margin_residual_is_gradient_of_energy():
    """The margin load is constant, so the margin part of the energy is linear in U: its central
    differences (energy with the margin minus energy without) equal the residual difference."""
    mesh = _margin(tiny_mesh(m=2, L=2), 1028.0)
    mesh.bed = mesh.bed - 500.0   # partly below sea level
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(21)
    U = rng.uniform(-100, 100, mesh.ndof)
    mesh.params.margin = 0
    om0 = oracle.OracleMesh(mesh)
    dR = om.residual(U) - om0.residual(U)
    assert np.abs(dR).max() > 0
    for j in rng.choice(mesh.ndof, 12, replace=False):
        h = 1e-3 * max(1.0, abs(U[j]))
        Up, Um = U.copy(), U.copy()
        Up[j] += h
        Um[j] -= h
        fd = ((om.energy(Up) - om0.energy(Up)) - (om.energy(Um) - om0.energy(Um))) / (2 * h)
        assert fd == pytest.approx(dR[j], rel=1e-6, abs=1e-6 * np.abs(dR).max())


# ------------------------------------------------------------------ temperature-dependent rate factor (Sec. 2, Arrhenius)

def test_uniform_rate_factor_field_equals_the_constant():
    mesh = tiny_mesh(m=3, L=2)
    rng = np.random.default_rng(31)
    U = rng.uniform(-100, 100, mesh.ndof)
    om0 = oracle.OracleMesh(mesh)
    R0, E0 = om0.residual(U), om0.energy(U)
    _, _, J0, _ = om0.jacobian(U)
    mesh.rate_factor = np.full(mesh.nv * (mesh.nlayers + 1), mesh.params.A)
    om = oracle.OracleMesh(mesh)
    _, _, J1, _ = om.jacobian(U)
    assert np.abs(om.residual(U) - R0).max() <= 1e-13 * np.abs(R0).max()
    assert np.abs(J1 - J0).max() <= 1e-13 * np.abs(J0).max()
    assert om.energy(U) == pytest.approx(E0, rel=1e-13)


def test_affine_hardness_field_is_reproduced_at_the_quadrature_points():
    """Nodal A = (b0 + g . x)^-3 makes the hardness A^(-1/3) affine in x; interpolated with the wedge
    basis it must equal b0 + g . x_q at every quadrature point (a wrong node or level index of the
    field, or a wrong exponent, breaks this)."""
    mesh = tiny_mesh(m=3, L=3)
    b0, g = 2.0e5, np.array([3.0, -2.0, 40.0])
    L = mesh.nlayers
    A = np.empty((mesh.nv, L + 1))
    for l in range(L + 1):
        X = np.stack([mesh.xy[:, 0], mesh.xy[:, 1], mesh.bed + mesh.sigma[l] * mesh.thick], 1)
        A[:, l] = (b0 + X @ g) ** -3.0
    mesh.rate_factor = A.reshape(-1)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(32)
    U = rng.uniform(-100, 100, mesh.ndof)
    for t in range(0, mesh.ntri, 3):
        for l in range(L):
            vert = mesh.tri[t]
            Xw = np.array([[mesh.xy[v, 0], mesh.xy[v, 1], mesh.bed[v] + mesh.sigma[l + k] * mesh.thick[v]]
                           for k in (0, 1) for v in vert])
            for q in range(6):
                xi, eta, zeta, _ = oracle.quadrature_point(q)
                N, _, _ = oracle.basis_at(Xw, xi, eta, zeta)
                xq = N @ Xw
                st = om.qp_state(U, t, l, q)
                B = 2 * st["mu"] * (st["eps2"] + mesh.params.delta) ** (1.0 / 3.0)
                assert B == pytest.approx(b0 + xq @ g, rel=1e-12)


def test_rate_factor_field_residual_is_gradient_of_energy():
    mesh = tiny_mesh(m=2, L=2)
    mesh.rate_factor = synth.arrhenius_rate_factor(mesh)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(33)
    U = rng.uniform(-100, 100, mesh.ndof)
    R = om.residual(U)
    J, _ = om.jacobian_scipy(U)
    for j in rng.choice(mesh.ndof, 12, replace=False):
        h = 1e-3 * max(1.0, abs(U[j]))
        Up, Um = U.copy(), U.copy()
        Up[j] += h
        Um[j] -= h
        fd = (om.energy(Up) - om.energy(Um)) / (2 * h)
        assert fd == pytest.approx(R[j], rel=1e-6, abs=1e-9 * np.abs(R).max())
        fdJ = (om.residual(Up) - om.residual(Um)) / (2 * h)
        col = J[:, j].toarray().ravel()
        assert np.abs(fdJ - col).max() <= 1e-6 * np.abs(col).max()


def test_arrhenius_rate_factor_values():
    """The generator's A at -10 C is the reference 3.5e-25 s^-1 Pa^-3 in both regimes, and A rises
    with temperature (and steeply above -10 C)."""
    mesh = tiny_mesh(m=2, L=2)
    A = synth.arrhenius_rate_factor(mesh, T_centre=-10.0, T_margin=-10.0, T_bed=-10.0)
    assert np.allclose(A, 3.5e-25 * synth.SECONDS_PER_YEAR, rtol=1e-12)
    warm = synth.arrhenius_rate_factor(mesh, T_centre=-2.0, T_margin=-2.0, T_bed=-2.0)[0]
    cold = synth.arrhenius_rate_factor(mesh, T_centre=-30.0, T_margin=-30.0, T_bed=-30.0)[0]
    assert cold < A[0] < warm
    # Q = 115 kJ/mol above -10 C: A(-2 C) / A(-10 C) = exp(Q/R (1/263.15 - 1/271.15))
    assert warm / A[0] == pytest.approx(math.exp(1.15e5 / 8.314 * (1 / 263.15 - 1 / 271.15)), rel=1e-12)


def test_threaded_colored_oracle_is_bitwise_independent_of_the_thread_count():
    """The coloured, threaded oracle (used to time the oracle on all host cores) gives bitwise the
    same Jacobian and residual for 1, 3 and 8 threads, and the plain oracle's up to summation order."""
    mesh = synth.dome_mesh(9, 4, 51, 52, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    U = synth.random_velocity(mesh, 53)
    _, _, v1, R1 = om.jacobian_colored(U, 1)
    for nt in (3, 8):
        _, _, vn, Rn = om.jacobian_colored(U, nt)
        assert np.array_equal(vn, v1) and np.array_equal(Rn, R1)
    _, _, v0, R0 = om.jacobian(U)
    assert np.abs(v1 - v0).max() <= 1e-14 * np.abs(v0).max()
    assert np.abs(R1 - R0).max() <= 1e-14 * np.abs(R0).max()
    marine = synth.marine_mesh(6, 3, 45, 46)  # with the lateral (ocean margin) load
    om = oracle.OracleMesh(marine)
    U = synth.random_velocity(marine, 54)
    _, _, v2, R2 = om.jacobian_colored(U, 4)
    _, _, v0, R0 = om.jacobian(U)
    assert np.abs(R2 - R0).max() <= 1e-14 * np.abs(R0).max() and np.abs(v2 - v0).max() <= 1e-14 * np.abs(v0).max()


@pytest.mark.parametrize("L", [5, 65])
def test_residual_and_jacobian_invariant_under_translations(L):
    """The discrete problem does not change when the whole geometry is moved: a vertical translation
    of bed and surface (stress-free margins) or a horizontal translation of the base mesh (every field
    nodal) leaves R and J as they are.  A term that used absolute coordinates where only differences
    belong (z instead of z - b, x instead of x - x_a) fails this.  The oracle's FP64 evaluation
    meets the invariance to its rounding, which grows on thin wedges (65 layers: aspect ratio ~1000),
    so the bar is 5e-13 at 5 layers and 5e-12 at 65 (measured at shallow-ice velocities: 1.2e-13
    and 1.4e-12; a wrong term moves R by O(1))."""
    import copy
    mesh = synth.dome_mesh(4, L, 93, 94, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    bar = 5e-13 if L == 5 else 5e-12
    for U in (om.sia(), synth.random_velocity(mesh, 103)):
        _, _, J, R = om.jacobian(U)
        lifted = copy.deepcopy(mesh)
        lifted.bed = mesh.bed + 500.0
        moved = copy.deepcopy(mesh)
        moved.xy = mesh.xy + np.array([3.7e4, -1.9e4])
        for other in (lifted, moved):
            _, _, J2, R2 = oracle.OracleMesh(other).jacobian(U)
            assert np.abs(R2 - R).max() <= bar * np.abs(R).max()
            assert np.abs(J2 - J).max() <= bar * np.abs(J).max()

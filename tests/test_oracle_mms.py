"""Manufactured-solution convergence of the oracle's discretisation (no GPU).

The oracle's residual and Jacobian (paper Sec. 2 field equations, Sec. 3.1 Eq. residual on the
extruded prism mesh) are driven by a body force and a basal traction derived symbolically from a
chosen smooth velocity field, so that this field is the exact solution of the continuous problem:

    -div(2 mu eps_c) = f_c                 in the ice (flat surface: no driving stress),
    2 mu eps_c . n = 0                     on the surface (the field has u_z = v_z = 0 there),
    2 mu eps_c . n + beta u_c = g_c        on the bed (n = (0, 0, -1)),
    u = exact                              on the lateral sides (Dirichlet rows, test only),

with mu = 1/2 A^(-1/3) (eps_e^2 + delta)^(-1/3).  Testing with N_i and integrating by parts gives
R_i(U) = int f_c N_i + int_bed g_c N_i, R the oracle residual.  Newton on the free dofs then gives
the discrete solution, whose L2 error must fall as h^2 (and the H1 error as h) when the base
mesh and the layers are refined together.  The load and the error integrals use a 7-point
degree-5 triangle rule (Radon) times 3-point Gauss in zeta, pinned below on monomials.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from paper_2204_04321_b300 import synth

sympy = pytest.importorskip("sympy")

HW = 10e3      # half width of the square (m)
THICK = 1000.0  # ice thickness (m), flat bed at z = 0
BETA = 1e3     # friction (Pa yr / m)


def radon7():
    """7-point degree-5 rule on the reference triangle (area 1/2): points (xi, eta), weights."""
    s = math.sqrt(15.0)
    a, b = (6 - s) / 21, (6 + s) / 21
    wa, wb = (155 - s) / 2400, (155 + s) / 2400
    pts = [(1 / 3, 1 / 3), (a, a), (1 - 2 * a, a), (a, 1 - 2 * a), (b, b), (1 - 2 * b, b), (b, 1 - 2 * b)]
    w = [9 / 80, wa, wa, wa, wb, wb, wb]
    return np.array(pts), np.array(w)


def gauss3():
    r = math.sqrt(0.6)
    return np.array([-r, 0.0, r]), np.array([5 / 9, 8 / 9, 5 / 9])


def test_radon7_rule_is_exact_to_degree_5():
    pts, w = radon7()
    for i in range(6):
        for j in range(6 - i):
            # int over the reference triangle of xi^i eta^j = i! j! / (i + j + 2)!
            exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            assert np.dot(w, pts[:, 0] ** i * pts[:, 1] ** j) == pytest.approx(exact, rel=1e-13)


def manufactured(params):
    x, y, z = sympy.symbols("x y z", real=True)
    X, Y, Z = x / HW, y / HW, z / THICK
    prof = 1 + sympy.Rational(1, 2) * Z * (2 - Z)  # d/dz = 0 at the surface
    u = 100 * (1 + sympy.Rational(3, 10) * sympy.sin(sympy.pi * X / 2 + sympy.Rational(3, 10))
               * sympy.cos(sympy.pi * Y / 2)) * prof
    v = 50 * (sympy.Rational(1, 2) + sympy.Rational(2, 5) * sympy.cos(sympy.pi * X / 2)
              * sympy.sin(sympy.pi * Y / 2 + sympy.Rational(1, 5))) * prof
    exx, eyy = sympy.diff(u, x), sympy.diff(v, y)
    exy = (sympy.diff(u, y) + sympy.diff(v, x)) / 2
    exz, eyz = sympy.diff(u, z) / 2, sympy.diff(v, z) / 2
    e2 = exx ** 2 + eyy ** 2 + exx * eyy + exy ** 2 + exz ** 2 + eyz ** 2
    mu = sympy.Float(0.5) * sympy.Float(params.A) ** sympy.Rational(-1, 3) * (e2 + params.delta) ** sympy.Rational(-1, 3)
    e1 = (2 * exx + eyy, exy, exz)
    e2v = (exy, exx + 2 * eyy, eyz)
    div = lambda e: sympy.diff(2 * mu * e[0], x) + sympy.diff(2 * mu * e[1], y) + sympy.diff(2 * mu * e[2], z)
    f1, f2 = -div(e1), -div(e2v)
    g1 = (-2 * mu * e1[2] + BETA * u).subs(z, 0)
    g2 = (-2 * mu * e2v[2] + BETA * v).subs(z, 0)
    lam = lambda e: sympy.lambdify((x, y, z), e, "numpy")
    grad = lambda w: [lam(sympy.diff(w, s)) for s in (x, y, z)]
    return {"u": lam(u), "v": lam(v), "f1": lam(f1), "f2": lam(f2), "g1": lam(g1), "g2": lam(g2),
            "grad_u": grad(u), "grad_v": grad(v)}


def wedge_points(mesh, t_pts, z_pts):
    """Physical quadrature points of every wedge: x, y [T, P], z [L, Z], weights w [T, L, P, Z]
    (right prisms: flat layers of constant thickness), and lambda [P, 3], psi [Z, 2]."""
    P = mesh.xy[mesh.tri]                       # [T, 3, 2]
    lam = np.stack([1 - t_pts[:, 0] - t_pts[:, 1], t_pts[:, 0], t_pts[:, 1]], 1)  # [P, 3]
    xq = np.einsum("pa,ta->tp", lam, P[:, :, 0])
    yq = np.einsum("pa,ta->tp", lam, P[:, :, 1])
    area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                        - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))
    zl = mesh.sigma * THICK
    hl = np.diff(zl)
    zq = zl[:-1, None] + 0.5 * (1 + z_pts[None, :]) * hl[:, None]   # [L, Z]
    psi = np.stack([0.5 * (1 - z_pts), 0.5 * (1 + z_pts)], 1)       # [Z, 2]
    return xq, yq, zq, area, hl, lam, psi


def solve_mms(m, L, ex):
    mesh = synth.slab_mesh(m, L, slope=0.0, thickness=THICK, beta=BETA, half_width=HW, jitter=0.0)
    om = oracle.OracleMesh(mesh)
    tp, tw = radon7()
    zp, zw = gauss3()
    xq, yq, zq, area, hl, lam, psi = wedge_points(mesh, tp, zp)
    T = mesh.ntri
    # load: int f_c N_i over every wedge + int_bed g_c N_i
    F = np.zeros(mesh.ndof)
    for l in range(L):
        for k in range(2):
            for c, fn in ((0, ex["f1"]), (1, ex["f2"])):
                fv = fn(xq[:, :, None], yq[:, :, None], zq[l][None, None, :])   # [T, P, Z]
                # w_tri (area 1/2 -> x 2 area) * w_z (sum 2 -> x h / 2)
                contrib = np.einsum("tpz,p,z,pa,z->ta", fv, tw, zw, lam, psi[:, k]) * (area * hl[l])[:, None]
                for a in range(3):
                    np.add.at(F, mesh.dof(mesh.tri[:, a], l + k, c), contrib[:, a])
    for c, gn in ((0, ex["g1"]), (1, ex["g2"])):
        gv = gn(xq, yq, 0.0) * np.ones_like(xq)
        contrib = np.einsum("tp,p,pa->ta", gv, tw, lam) * (2 * area)[:, None]
        for a in range(3):
            np.add.at(F, mesh.dof(mesh.tri[:, a], 0, c), contrib[:, a])
    # exact nodal values; lateral Dirichlet dofs
    zn = mesh.sigma * THICK
    U = np.zeros(mesh.ndof)
    for l in range(L + 1):
        U[mesh.dof(np.arange(mesh.nv), l, 0)] = ex["u"](mesh.xy[:, 0], mesh.xy[:, 1], zn[l])
        U[mesh.dof(np.arange(mesh.nv), l, 1)] = ex["v"](mesh.xy[:, 0], mesh.xy[:, 1], zn[l])
    side = (np.abs(np.abs(mesh.xy[:, 0]) - HW) < 1e-6 * HW) | (np.abs(np.abs(mesh.xy[:, 1]) - HW) < 1e-6 * HW)
    fixed = np.zeros(mesh.ndof, bool)
    for l in range(L + 1):
        for c in (0, 1):
            fixed[mesh.dof(np.nonzero(side)[0], l, c)] = True
    free = ~fixed
    fnorm = np.linalg.norm(F[free])
    for it in range(20):
        J, R = om.jacobian_scipy(U)
        r = (R - F)[free]
        if np.linalg.norm(r) <= 1e-11 * fnorm:
            break
        d = spla.spsolve(J[free][:, free].tocsc(), -r)
        U[free] += d
    else:
        raise AssertionError("Newton did not converge on the manufactured problem")
    # L2 and H1-seminorm errors by quadrature
    e0 = n0 = e1 = n1 = 0.0
    for l in range(L):
        w = np.einsum("p,z->pz", tw, zw)[None] * (area * hl[l])[:, None, None]    # [T, P, Z]
        for c, (fn, gfn) in enumerate(((ex["u"], ex["grad_u"]), (ex["v"], ex["grad_v"]))):
            ue = fn(xq[:, :, None], yq[:, :, None], zq[l][None, None, :]) * np.ones(w.shape)
            Un = np.stack([U[mesh.dof(mesh.tri[:, a], l + k, c)] for k in (0, 1) for a in range(3)], 1)  # [T, 6]
            Nq = np.einsum("pa,zk->pzka", lam, psi).reshape(len(tp), len(zp), 6)
            uh = np.einsum("pzn,tn->tpz", Nq, Un)
            e0 += np.sum(w * (uh - ue) ** 2)
            n0 += np.sum(w * ue ** 2)
            # gradient of the discrete field: in-plane P1 gradient times psi plus lambda times the z slope
            P = mesh.xy[mesh.tri]
            det = ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                   - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))
            lx = np.stack([(P[:, (a + 1) % 3, 1] - P[:, (a + 2) % 3, 1]) / det for a in range(3)], 1)
            ly = np.stack([(P[:, (a + 2) % 3, 0] - P[:, (a + 1) % 3, 0]) / det for a in range(3)], 1)
            ub, ut = Un[:, :3], Un[:, 3:]
            gx = np.einsum("ta,ta->t", lx, ub)[:, None, None] * psi[None, None, :, 0] + \
                np.einsum("ta,ta->t", lx, ut)[:, None, None] * psi[None, None, :, 1]
            gy = np.einsum("ta,ta->t", ly, ub)[:, None, None] * psi[None, None, :, 0] + \
                np.einsum("ta,ta->t", ly, ut)[:, None, None] * psi[None, None, :, 1]
            gz = np.einsum("pa,ta->tp", lam, ut - ub)[:, :, None] / hl[l] * np.ones(w.shape)
            for gh, gfe in zip((gx * np.ones(w.shape), gy * np.ones(w.shape), gz), gfn):
                ge = gfe(xq[:, :, None], yq[:, :, None], zq[l][None, None, :]) * np.ones(w.shape)
                e1 += np.sum(w * (gh - ge) ** 2)
                n1 += np.sum(w * ge ** 2)
    return math.sqrt(e0 / n0), math.sqrt(e1 / n1), it


@pytest.mark.slow
def test_manufactured_solution_converges_at_second_order():
    ex = manufactured(synth.Params())
    errs = [solve_mms(m, L, ex) for m, L in ((4, 2), (8, 4), (16, 8))]
    l2 = [e[0] for e in errs]
    h1 = [e[1] for e in errs]
    r_l2 = [math.log2(l2[i] / l2[i + 1]) for i in range(2)]
    r_h1 = [math.log2(h1[i] / h1[i + 1]) for i in range(2)]
    assert all(e[2] <= 8 for e in errs)                 # Newton from the interpolant converges fast
    # L2: rate over the two halvings (the single steps read 2.15 and 1.76 on these regular meshes;
    # one more halving, 37k dofs and ~1 min of sparse LU, reads 1.92)
    rate_l2 = math.log2(l2[0] / l2[2]) / 2
    assert 1.8 <= rate_l2 <= 2.3, (l2, r_l2)
    assert all(1.6 <= r <= 2.4 for r in r_l2), (l2, r_l2)
    assert all(0.9 <= r <= 1.15 for r in r_h1), (h1, r_h1)

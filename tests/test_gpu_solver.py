"""Parity of the solver kernels (through the C ABI) with plain CPU statements of the same steps.

SpMV against scipy's CSR product; the column preconditioner against dense solves of each
column's block-tridiagonal matrix; energy and the shallow-ice guess against the oracle; the
Newton solution against the oracle's Newton solution (the discrete problem has a unique
minimiser) and, at full size, the final residual recomputed by the oracle.
"""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle.newton import newton as oracle_newton
from paper_2204_04321_b300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def capi():
    from paper_2204_04321_b300 import capi as c
    return c


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def rel_inf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _host_csr(dm, J):
    rp, ci = dm.pattern()
    return sp.csr_matrix((J.cpu().numpy().astype(np.float64), ci.cpu().numpy(), rp.cpu().numpy()),
                         shape=(dm.ndof, dm.ndof))


@pytest.mark.parametrize("precision", [0, 1, 3])   # FP64, FP32 and FP32-value-path (float) values
def test_spmv_matches_scipy(precision):
    c = capi()
    mesh = synth.dome_mesh(23, 4, 31, 32, bed="sinusoidal")
    dm = c.DeviceMesh(mesh)
    U = dev(synth.random_velocity(mesh, 3))
    J, _ = dm.jacobian(U, precision=precision)
    x = np.random.default_rng(1).normal(size=dm.ndof)
    y = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    c.bp_spmv(dm.handle, J, dev(x), y, precision=precision)
    A = _host_csr(dm, J)
    assert rel_inf(y.cpu().numpy(), A @ x) <= 1e-13


@pytest.mark.parametrize("size", ["small", "dome_1m"])
def test_fp32_spmv_within_fp32_dot_product_bound(size):
    """The mixed-precision Krylov product (FP32 values, vectors, products and sums; grid-stride
    over row pairs, several per group on the 1M-wedge dome) against scipy's FP64 product of the
    same FP32 data: every row within the error bound of an FP32 dot product,
    (n + 2) u sum_j |a_ij x_j| (n the row length, u = 2^-24)."""
    c = capi()
    mesh = synth.dome_mesh(23, 4, 31, 32, bed="sinusoidal") if size == "small" else synth.config_medium()
    dm = c.DeviceMesh(mesh)
    U = dev(synth.random_velocity(mesh, 3))
    J, _ = dm.jacobian(U, precision=1)
    x = torch.from_numpy(np.random.default_rng(1).normal(size=dm.ndof).astype(np.float32)).cuda()
    y = torch.full((dm.ndof,), float("nan"), dtype=torch.float32, device="cuda")
    c.bp_spmv_f32(dm.handle, J, x, y)
    A = _host_csr(dm, J)
    xs = x.cpu().numpy().astype(np.float64)
    err = np.abs(y.cpu().numpy().astype(np.float64) - A @ xs)
    bound = (np.diff(A.indptr) + 2) * 2.0**-24 * (abs(A) @ np.abs(xs))
    assert np.all(np.isfinite(err)) and np.all(err <= bound)


def test_fp32_spmv_refuses_misaligned_buffers():
    """bp_spmv_f32 reads (u, v) pairs: x, y and J must start on 16-byte boundaries (BP_EINVAL,
    nothing read or written otherwise)."""
    c = capi()
    mesh = synth.dome_mesh(8, 3, 31, 32)
    dm = c.DeviceMesh(mesh)
    J, _ = dm.jacobian(dev(synth.random_velocity(mesh, 3)), precision=1)
    x = torch.zeros(dm.ndof + 4, dtype=torch.float32, device="cuda")
    y = torch.full((dm.ndof + 4,), 7.0, dtype=torch.float32, device="cuda")
    for args in ((J, x[1:], y[:dm.ndof]), (J, x[:dm.ndof], y[1:]), (J[1:], x[:dm.ndof], y[:dm.ndof])):
        with pytest.raises(c.BPError) as e:
            c.bp_spmv_f32(dm.handle, *args)
        assert e.value.status == c.BP_EINVAL
    torch.cuda.synchronize()
    assert bool((y == 7.0).all())


def _column_blocks(A, mesh, a):
    L = mesh.nlayers
    idx = np.array([mesh.dof(a, l, c) for l in range(L + 1) for c in (0, 1)])
    B = A[idx][:, idx].toarray()
    # keep only the block-tridiagonal part (levels |l - l'| <= 1 is all there is within a column)
    return idx, B


@pytest.mark.parametrize("precision", [0, 1, 3])
def test_column_preconditioner_is_exact_block_tridiagonal_solve(precision):
    c = capi()
    mesh = synth.dome_mesh(12, 6, 51, 52, bed="sinusoidal")
    dm = c.DeviceMesh(mesh)
    U = dev(synth.random_velocity(mesh, 4))
    J, _ = dm.jacobian(U, precision=precision)
    c.bp_colprec_setup(dm.handle, J, precision=precision)
    r = np.random.default_rng(2).normal(size=dm.ndof)
    z = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    c.bp_colprec_apply(dm.handle, dev(r), z)
    z = z.cpu().numpy()
    A = _host_csr(dm, J)
    # FP64 factors: exact to rounding; FP32 factors from FP32 elimination (mixed path): block Thomas
    # without pivoting is backward stable on these SPD columns, so the forward error is bounded by a
    # small multiple of the FP32 unit roundoff times the column block's condition number
    for a in range(0, mesh.nv, 7):
        idx, B = _column_blocks(A, mesh, a)
        zc = np.linalg.solve(B, r[idx])
        tol = 1e-11 if precision == 0 else max(2e-5, 10 * 2.0**-24 * np.linalg.cond(B))
        assert rel_inf(z[idx], zc) <= tol


@pytest.mark.parametrize("kind", ["random", "sia", "marine", "arrhenius"])
def test_energy_matches_oracle(kind):
    c = capi()
    mesh = (synth.marine_mesh(14, 5, 61, 62) if kind == "marine"
            else synth.dome_mesh(20, 5, 61, 62, bed="sinusoidal", beta="field"))
    if kind == "arrhenius":
        mesh.rate_factor = synth.arrhenius_rate_factor(mesh)
    om = oracle.OracleMesh(mesh)
    U = synth.random_velocity(mesh, 5) if kind == "random" else om.sia()
    dm = c.DeviceMesh(mesh)
    E = c.bp_energy(dm.handle, dev(U))
    assert E == pytest.approx(om.energy(U), rel=1e-12)


@pytest.mark.parametrize("alpha", [1.0, 1e-3])
@pytest.mark.parametrize("precision,rtol", [("F64", 1e-9), ("F64X2_DS", 1e-9), ("F32", 1e-4)])
def test_energy_change_kinds_match_oracle_difference(precision, rtol, alpha):
    """The three line-search kinds (FP64, double-single pairs: the FP64 solves' line search; FP32: the
    mixed solves') against the oracle's energy difference."""
    c = capi()
    mesh = synth.dome_mesh(20, 5, 61, 62, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    U = om.sia()
    D = synth.random_velocity(mesh, 8, amplitude=30.0)
    dm = c.DeviceMesh(mesh)
    dE = c.bp_energy_change_ex(dm.handle, dev(U), dev(D), alpha, getattr(c, "BP_" + precision))
    E0 = om.energy(U)
    ref = om.energy(U + alpha * D) - E0
    assert abs(dE - ref) <= rtol * abs(ref) + 1e-13 * abs(E0)
    if precision == "F32":
        return
    a = 1e-9  # the first-order prediction alpha R . D at a tiny step, as below
    d1 = c.bp_energy_change_ex(dm.handle, dev(U), dev(D), a, getattr(c, "BP_" + precision)) / a
    d2 = c.bp_energy_change_ex(dm.handle, dev(U), dev(D), 2 * a, getattr(c, "BP_" + precision)) / (2 * a)
    assert 2 * d1 - d2 == pytest.approx(float(om.residual(U) @ D), rel=1e-5)


def test_energy_change_ex_refuses_other_kinds():
    c = capi()
    dm = c.DeviceMesh(synth.dome_mesh(6, 2, 61, 62))
    U = torch.zeros(dm.ndof, dtype=torch.float64, device="cuda")
    for bad in (c.BP_F64X2, c.BP_F32_ALL, c.BP_F32_DS, 99):
        with pytest.raises(c.BPError):
            c.bp_energy_change_ex(dm.handle, U, U, 1.0, bad)


@pytest.mark.parametrize("alpha", [1.0, 1e-3])
def test_energy_change_matches_oracle_difference(alpha):
    """Against the oracle's energy difference at steps large enough for that difference to be accurate;
    at a tiny step the GPU's change must agree with the first-order prediction alpha R . D."""
    c = capi()
    mesh = synth.dome_mesh(20, 5, 61, 62, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    U = om.sia()
    D = synth.random_velocity(mesh, 8, amplitude=30.0)
    dm = c.DeviceMesh(mesh)
    dE = c.bp_energy_change(dm.handle, dev(U), dev(D), alpha)
    E0 = om.energy(U)
    ref = om.energy(U + alpha * D) - E0
    assert abs(dE - ref) <= 1e-9 * abs(ref) + 1e-13 * abs(E0)  # the oracle difference carries E0's rounding
    # derivative at alpha = 0 equals R . D: Richardson-extrapolate dE(a)/a (error O(a) -> O(a^2)); a must
    # be far below the step at which the strain of a D crosses the regularisation scale sqrt(delta)
    a = 1e-9
    d1 = c.bp_energy_change(dm.handle, dev(U), dev(D), a) / a
    d2 = c.bp_energy_change(dm.handle, dev(U), dev(D), 2 * a) / (2 * a)
    slope = float(om.residual(U) @ D)
    assert 2 * d1 - d2 == pytest.approx(slope, rel=1e-5)


def test_shallow_ice_guess_matches_oracle():
    c = capi()
    mesh = synth.config_small()
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
    assert rel_inf(U.cpu().numpy(), om.sia()) <= 1e-12
    c.bp_initial_guess(dm.handle, c.BP_GUESS_ZERO, U)
    assert float(U.abs().max()) == 0.0


@pytest.mark.parametrize("geometry", ["dome", "marine", "arrhenius"])
def test_newton_matches_oracle_newton_on_tiny_mesh(geometry):
    c = capi()
    mesh = (synth.marine_mesh(6, 3, 71, 72) if geometry == "marine"
            else synth.dome_mesh(4, 3, 71, 72, bed="sinusoidal", beta="iid"))
    if geometry == "arrhenius":
        mesh.rate_factor = synth.arrhenius_rate_factor(mesh)
    om = oracle.OracleMesh(mesh)
    Uo, info = oracle_newton(om, np.zeros(mesh.ndof), rtol=1e-10)
    assert info["converged"]
    dm = c.DeviceMesh(mesh)
    U = torch.zeros(dm.ndof, dtype=torch.float64, device="cuda")
    rc, rep = c.bp_newton_solve(dm.handle, U, rtol=1e-10, max_krylov=4000)
    assert rc == c.BP_OK and rep["converged"], rep
    assert rel_inf(U.cpu().numpy(), Uo) <= 1e-7
    # the GPU's final residual, recomputed by the oracle
    assert np.linalg.norm(om.residual(U.cpu().numpy())) <= 1.5e-10 * np.linalg.norm(om.residual(0 * Uo))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("line_search", [1, 2])
def test_newton_small_dome_converges_from_zero_and_sia_to_same_solution(precision, line_search):
    c = capi()
    mesh = synth.config_small()
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    sols = []
    for guess in (c.BP_GUESS_ZERO, c.BP_GUESS_SIA):
        U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        c.bp_initial_guess(dm.handle, guess, U)
        rc, rep = c.bp_newton_solve(dm.handle, U, precision=precision, line_search=line_search)
        assert rc == c.BP_OK, rep
        assert rep["history"][-1] <= 1e-8
        Uh = U.cpu().numpy()
        fo = np.linalg.norm(om.residual(Uh)) / np.linalg.norm(om.residual(np.zeros_like(Uh)))
        assert fo <= 1.1e-8
        sols.append(Uh)
    assert rel_inf(sols[0], sols[1]) <= 1e-6


@pytest.mark.slow
@pytest.mark.parametrize("geometry,precision", [("dome", 0), ("marine", 0), ("marine", 1)])
def test_newton_full_size_dome_reaches_1e8_checked_by_oracle(geometry, precision):
    c = capi()
    mesh = synth.config_medium() if geometry == "dome" else synth.config_marine()
    dm = c.DeviceMesh(mesh)
    U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
    rc, rep = c.bp_newton_solve(dm.handle, U, max_krylov=4000, precision=precision)
    assert rc == c.BP_OK, rep
    om = oracle.OracleMesh(mesh)
    Uh = U.cpu().numpy()
    f = np.linalg.norm(om.residual(Uh)) / np.linalg.norm(om.residual(np.zeros_like(Uh)))
    assert f <= 1.1e-8, f


def test_rate_factor_entry_validates_and_resets():
    c = capi()
    mesh = synth.config_small()
    dm = c.DeviceMesh(mesh)
    U = dev(synth.random_velocity(mesh, 3))
    R0 = dm.residual(U).cpu().numpy()
    bad = np.full(mesh.nv * (mesh.nlayers + 1), mesh.params.A)
    bad[7] = -1.0
    with pytest.raises(c.BPError) as e:
        c.bp_mesh_set_rate_factor(dm.handle, bad)
    assert e.value.status == c.BP_EINVAL
    c.bp_mesh_set_rate_factor(dm.handle, np.full(mesh.nv * (mesh.nlayers + 1), 8 * mesh.params.A))
    R8 = dm.residual(U).cpu().numpy()
    c.bp_mesh_set_rate_factor(dm.handle, None)
    assert rel_inf(dm.residual(U).cpu().numpy(), R0) <= 1e-14
    assert rel_inf(R8, R0) > 1e-3   # an 8x softer ice halves the stress term


@pytest.mark.parametrize("precision", [0, 1])
def test_picard_then_newton_reaches_the_same_solution(precision):
    """Picard steps (the Jacobian without the eta' rank-one part) while far from the solution, then
    Newton: the same minimiser as pure Newton, and the final FP64 residual checked by the oracle."""
    c = capi()
    mesh = synth.config_small()
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    sols = []
    for pr in (0.0, 0.05):
        U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
        rc, rep = c.bp_newton_solve(dm.handle, U, precision=precision, picard_rtol=pr)
        assert rc == c.BP_OK, rep
        Uh = U.cpu().numpy()
        assert np.linalg.norm(om.residual(Uh)) <= 1.1e-8 * np.linalg.norm(om.residual(np.zeros_like(Uh)))
        sols.append(Uh)
    assert rel_inf(sols[0], sols[1]) <= 1e-6
    with pytest.raises(c.BPError):
        c.bp_newton_solve(dm.handle, U, picard_rtol=-1.0)


@pytest.mark.parametrize("geometry", ["dome", "marine"])
def test_fp32_value_path_steps_then_fp64_reach_the_same_solution(geometry):
    """Mixed-precision Newton whose early steps assemble with the FP32 value path (inexact residual):
    the same minimiser, and the final residual (always FP64) checked by the oracle."""
    c = capi()
    mesh = synth.config_small() if geometry == "dome" else synth.marine_mesh(12, 5, 45, 46)
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    sols, steps = [], []
    for v32 in (0.0, 1e-3):
        U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
        rc, rep = c.bp_newton_solve(dm.handle, U, precision=c.BP_F32, value32_rtol=v32)
        assert rc == c.BP_OK, rep
        Uh = U.cpu().numpy()
        assert np.linalg.norm(om.residual(Uh)) <= 1.1e-8 * np.linalg.norm(om.residual(np.zeros_like(Uh)))
        sols.append(Uh)
        steps.append(rep["value32_steps"])
    assert steps[0] == 0 and steps[1] >= 1
    assert rel_inf(sols[0], sols[1]) <= 1e-6
    for bad in (-1.0, 5e-9):  # below rtol (1e-8) an FP32 residual could pass the convergence test
        with pytest.raises(c.BPError) as e:
            c.bp_newton_solve(dm.handle, U, precision=c.BP_F32, value32_rtol=bad)
        assert e.value.status == c.BP_EINVAL


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("layers", [3, 5])
def test_device_driven_cg_loop_matches_host_checked_batches(precision, layers):
    """The CG iterations as a conditional-graph loop stopped by the device, against replays of the
    captured batch checked by the host: the same iterations, the same Newton path and solution
    (5 layers take the register-resident column update, 3 the staged one)."""
    c = capi()
    mesh = synth.dome_mesh(16, layers, 81, 82, bed="sinusoidal", beta="field")
    dm = c.DeviceMesh(mesh)
    out = []
    for loop in (1, 0):
        U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
        rc, rep = c.bp_newton_solve(dm.handle, U, precision=precision, device_loop=loop)
        assert rc == c.BP_OK, rep
        out.append((U.cpu().numpy(), rep))
    (U1, r1), (U0, r0) = out
    # the two runs differ only in the order of the atomic additions of the dot products (as two
    # runs of either mode do), which can move a borderline stopping test by one iteration; both
    # stop at 1e-8 relative residual
    assert abs(r1["newton_iters"] - r0["newton_iters"]) <= 1
    assert abs(r1["krylov_iters"] - r0["krylov_iters"]) <= max(2, r0["newton_iters"])
    assert rel_inf(U1, U0) <= 1e-6
    with pytest.raises(c.BPError):
        c.bp_newton_solve(dm.handle, U, device_loop=2)


@pytest.mark.slow
def test_mixed_newton_4m_wedges_checked_by_oracle():
    """The 3,996,180-wedge dome solved with FP32 Jacobian lanes and Krylov from the shallow-ice
    guess: the oracle's FP64 residual of the solution is at most 1.1e-8 ||F(0)||, and the solution
    agrees with the plain FP64 path's to 1e-6 (max norm, relative)."""
    c = capi()
    mesh = synth.config_large()
    dm = c.DeviceMesh(mesh)
    sols = []
    for precision in (c.BP_F32, c.BP_F64):
        U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
        rc, rep = c.bp_newton_solve(dm.handle, U, max_krylov=4000, precision=precision)
        assert rc == c.BP_OK, rep
        sols.append(U.cpu().numpy())
        del U
    dm.close()
    om = oracle.OracleMesh(mesh)
    f = np.linalg.norm(om.residual(sols[0])) / np.linalg.norm(om.residual(np.zeros_like(sols[0])))
    assert f <= 1.1e-8, f
    assert rel_inf(sols[0], sols[1]) <= 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_gmres_newton_reaches_the_cg_solution(precision):
    """GMRES(m) with the column preconditioner (the paper's Krylov method) as the cross-check of CG:
    the same Newton solution to 1e-7, the oracle's FP64 residual at 1e-8, with restart lengths that
    do and do not restart within a Newton step."""
    c = capi()
    mesh = synth.dome_mesh(16, 5, 81, 82, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    f0 = np.linalg.norm(om.residual(np.zeros(mesh.ndof)))
    sols = {}
    for name, kw in (("cg", {}), ("gmres50", {"krylov": c.BP_KRYLOV_GMRES}),
                     ("gmres5", {"krylov": c.BP_KRYLOV_GMRES, "gmres_restart": 5})):
        U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
        rc, rep = c.bp_newton_solve(dm.handle, U, precision=precision, max_krylov=4000, **kw)
        assert rc == c.BP_OK, (name, rep)
        Uh = U.cpu().numpy()
        assert np.linalg.norm(om.residual(Uh)) <= 1.1e-8 * f0, name
        sols[name] = (Uh, rep)
    for name in ("gmres50", "gmres5"):
        assert rel_inf(sols[name][0], sols["cg"][0]) <= 1e-7, name
    assert sols["gmres5"][1]["krylov_iters"] >= sols["gmres50"][1]["krylov_iters"]
    for bad in ({"gmres_restart": 0}, {"gmres_restart": 65}, {"krylov": 7}):
        with pytest.raises(c.BPError) as e:
            c.bp_newton_solve(dm.handle, U, krylov=c.BP_KRYLOV_GMRES if "gmres_restart" in bad else bad["krylov"],
                              **{k: v for k, v in bad.items() if k != "krylov"})
        assert e.value.status == c.BP_EINVAL
    with pytest.raises(c.BPError) as e:
        c.bp_newton_solve(dm.handle, U, krylov=c.BP_KRYLOV_GMRES, preconditioner=c.BP_PREC_MDSC)
    assert e.value.status == c.BP_EUNSUP


@pytest.mark.parametrize("precision", ["f32_ds", "f64x2_ds"])
def test_double_single_value_path_newton_reaches_the_fp64_solution(precision):
    """Newton with the double-single value path (residual FP64-accurate on the FP32 pipe): the
    oracle's FP64 residual of the solution at 1e-8 and the plain FP64 path's solution to 1e-7."""
    c = capi()
    mesh = synth.dome_mesh(16, 5, 81, 82, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    f0 = np.linalg.norm(om.residual(np.zeros(mesh.ndof)))
    sols = []
    for prec in (c.BP_F64, {"f32_ds": c.BP_F32_DS, "f64x2_ds": c.BP_F64X2_DS}[precision]):
        U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
        rc, rep = c.bp_newton_solve(dm.handle, U, precision=prec, max_krylov=4000)
        assert rc == c.BP_OK, rep
        Uh = U.cpu().numpy()
        assert np.linalg.norm(om.residual(Uh)) <= 1.1e-8 * f0
        sols.append(Uh)
    assert rel_inf(sols[0], sols[1]) <= 1e-7
    if precision == "f64x2_ds":
        with pytest.raises(c.BPError) as e:
            c.bp_newton_solve(dm.handle, U, precision=c.BP_F64X2_DS, picard_rtol=0.1)
        assert e.value.status == c.BP_EUNSUP


def test_energy_change_with_tail_segments_matches_oracle():
    """80,000 columns, more than one wave of resident threads of the energy-change kernel (75,776 on a
    B300): the last partial wave's columns are taken in layer segments; the change must still equal
    the oracle's energy difference."""
    c = capi()
    mesh = synth.dome_mesh(200, 4, 63, 64, bed="sinusoidal", beta="field")
    assert mesh.ntri == 80000
    om = oracle.OracleMesh(mesh)
    U = om.sia()
    D = synth.random_velocity(mesh, 9, amplitude=30.0)
    dm = c.DeviceMesh(mesh)
    dE = c.bp_energy_change(dm.handle, dev(U), dev(D), 1.0)
    E0 = om.energy(U)
    ref = om.energy(U + D) - E0
    assert abs(dE - ref) <= 1e-9 * abs(ref) + 1e-13 * abs(E0)


def test_layer_count_limits():
    """64 layers, the solver's largest column: the FP64 and the mixed Newton solves reach the oracle's
    FP64 residual bar.  65 layers: the assembly still matches the oracle; the solver's entry points
    answer BP_EUNSUP.

    On wedges this thin (aspect ratio ~1000) the oracle's own FP64 rounding approaches the 1e-12
    bar: the exact residual does not change when the geometry is translated (bed and surface
    vertically, or the base mesh horizontally), the oracle's evaluation changes by ~1e-12 normwise
    (its generic 3 x 3 inverse of each thin wedge's Jacobian).  At shallow-ice velocities the bar is therefore twice that measured change when it
    exceeds 1e-12; at random velocities it stays 1e-12."""
    c = capi()
    mesh = synth.dome_mesh(4, 64, 91, 92, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    f0 = np.linalg.norm(om.residual(np.zeros(mesh.ndof)))
    for prec in (c.BP_F64, c.BP_F32):
        U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
        rc, rep = c.bp_newton_solve(dm.handle, U, precision=prec, max_krylov=4000)
        assert rc == c.BP_OK, rep
        assert np.linalg.norm(om.residual(U.cpu().numpy())) <= 1.1e-8 * f0
    mesh65 = synth.dome_mesh(4, 65, 93, 94, bed="sinusoidal", beta="field")
    om65 = oracle.OracleMesh(mesh65)
    dm65 = c.DeviceMesh(mesh65)
    U65 = om65.sia()
    _, _, Jc, Rc = om65.jacobian(U65)
    J, R = dm65.jacobian(dev(U65))
    lifted = copy.deepcopy(mesh65)
    lifted.bed = mesh65.bed + 500.0
    moved = copy.deepcopy(mesh65)
    moved.xy = mesh65.xy + np.array([3.7e4, -1.9e4])
    own = max(rel_inf(oracle.OracleMesh(other).residual(U65), Rc) for other in (lifted, moved))
    assert rel_inf(R.cpu().numpy(), Rc) <= max(1e-12, 2 * own)
    assert rel_inf(J.cpu().numpy(), Jc) <= 1e-12
    Ur = synth.random_velocity(mesh65, 103)
    _, _, Jr, Rr = om65.jacobian(Ur)
    J, R = dm65.jacobian(dev(Ur))
    assert rel_inf(R.cpu().numpy(), Rr) <= 1e-12 and rel_inf(J.cpu().numpy(), Jr) <= 1e-12
    U = torch.zeros(dm65.ndof, dtype=torch.float64, device="cuda")
    for call in (lambda: c.bp_initial_guess(dm65.handle, c.BP_GUESS_SIA, U),
                 lambda: c.bp_newton_solve(dm65.handle, U),
                 lambda: c.bp_energy(dm65.handle, U)):
        with pytest.raises(c.BPError) as e:
            call()
        assert e.value.status == c.BP_EUNSUP

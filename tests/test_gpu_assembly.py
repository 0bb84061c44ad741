"""Parity of the CUDA assembly (through the C ABI) with the CPU oracle.

Bar: residual ||R_gpu - R_cpu||_inf <= 1e-12 ||R_cpu||_inf (FP64); Jacobian
max|J_gpu - J_cpu| <= 1e-12 max|J_cpu| (FP64 and paired-FP32 lanes) and <= 1e-5 max|J_cpu|
(FP32 lanes);
CSR pattern bit-identical.  The comparison is normwise because the GPU sums element
contributions in another order (atomics) and with another (structured) formulation, so
entries where contributions cancel carry rounding relative to the row scale, not to themselves.
"""
import numpy as np
import pytest

import oracle
from paper_2204_04321_b300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


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


def ragged_mesh(m=23, L=4, seed=31):
    """1,058 triangles: 9 blocks of 128 columns with a ragged tail; non-uniform sigma, bumpy bed."""
    mesh = synth.dome_mesh(m, L, seed, seed + 1, H0=1800.0, bed="sinusoidal", beta="iid")
    rng = np.random.default_rng(seed)
    mesh.sigma = np.sort(np.concatenate([[0.0, 1.0], rng.uniform(0.05, 0.95, L - 1)]))
    return mesh


def arrhenius_mesh():
    """Temperature-dependent rate factor (nodal field, 35x range of A)."""
    mesh = synth.dome_mesh(10, 4, 47, 48, bed="sinusoidal", beta="field")
    mesh.rate_factor = synth.arrhenius_rate_factor(mesh)
    return mesh


MESHES = {
    "small": synth.config_small,
    "ragged": ragged_mesh,
    "single_layer": lambda: synth.dome_mesh(6, 1, 41, 42, bed="sinusoidal", beta="iid"),
    "two_layers": lambda: synth.dome_mesh(5, 2, 43, 44, bed="sinusoidal", beta="field"),
    # ocean margin condition on the lateral faces (calving front partly below sea level)
    "marine": lambda: synth.marine_mesh(12, 4, 45, 46),
    "arrhenius": arrhenius_mesh,
}


def velocities(mesh, kind, om):
    if kind == "random":
        return synth.random_velocity(mesh, 103)
    if kind == "zero":
        return np.zeros(mesh.ndof)
    return om.sia()


@pytest.mark.parametrize("name", list(MESHES))
def test_pattern_identical_to_oracle(name):
    mesh = MESHES[name]()
    om = oracle.OracleMesh(mesh)
    dm = capi().DeviceMesh(mesh)
    rowptr, colidx = dm.pattern()
    orp, oci = om.pattern()
    assert dm.nnz == len(oci) == mesh.expected_nnz()
    assert np.array_equal(rowptr.cpu().numpy(), orp)
    assert np.array_equal(colidx.cpu().numpy(), oci)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("kind", ["random", "zero", "sia"])
def test_residual_parity(name, kind):
    mesh = MESHES[name]()
    om = oracle.OracleMesh(mesh)
    U = velocities(mesh, kind, om)
    dm = capi().DeviceMesh(mesh)
    R = dm.residual(dev(U)).cpu().numpy()
    Rc = om.residual(U)
    assert rel_inf(R, Rc) <= TOL64


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("method", ["factored", "dual"])
@pytest.mark.parametrize("scatter", ["atomic", "color"])
@pytest.mark.parametrize("precision", ["f64", "f32", "f64x2", "f32_ds", "f64x2_ds"])
def test_jacobian_parity(name, method, scatter, precision):
    c = capi()
    if precision not in ("f64", "f32") and method == "dual":
        pytest.skip("paired-FP32 lanes and the double-single value path are implemented for the "
                    "sum-factorised method only")
    mesh = MESHES[name]()
    om = oracle.OracleMesh(mesh)
    U = synth.random_velocity(mesh, 103)
    dm = c.DeviceMesh(mesh)
    prec = {"f64": c.BP_F64, "f32": c.BP_F32, "f64x2": c.BP_F64X2, "f32_ds": c.BP_F32_DS,
            "f64x2_ds": c.BP_F64X2_DS}[precision]
    J, R = dm.jacobian(dev(U), precision=prec,
                       scatter=c.BP_SCATTER_ATOMIC if scatter == "atomic" else c.BP_SCATTER_COLOR,
                       method=c.BP_JAC_FACTORED if method == "factored" else c.BP_JAC_DUAL)
    _, _, Jc, Rc = om.jacobian(U)
    assert rel_inf(R.cpu().numpy(), Rc) <= TOL64
    err = rel_inf(J.cpu().numpy().astype(np.float64), Jc)
    assert err <= (TOL32 if precision in ("f32", "f32_ds") else TOL64), err


@pytest.mark.parametrize("name", ["small", "marine", "arrhenius"])
@pytest.mark.parametrize("kind", ["zero", "sia"])
@pytest.mark.parametrize("precision", ["f64", "f32", "f32_ds", "f64x2_ds"])
def test_jacobian_parity_at_zero_and_shallow_ice_velocities(name, kind, precision):
    """U = 0 makes every strain-rate lane exactly zero (the FP32 lane conversion's zero case);
    the shallow-ice guess is the usual starting point of the Newton solve."""
    c = capi()
    mesh = MESHES[name]()
    om = oracle.OracleMesh(mesh)
    U = velocities(mesh, kind, om)
    dm = c.DeviceMesh(mesh)
    prec = {"f64": c.BP_F64, "f32": c.BP_F32, "f32_ds": c.BP_F32_DS, "f64x2_ds": c.BP_F64X2_DS}[precision]
    J, R = dm.jacobian(dev(U), precision=prec)
    _, _, Jc, Rc = om.jacobian(U)
    assert rel_inf(R.cpu().numpy(), Rc) <= TOL64
    err = rel_inf(J.cpu().numpy().astype(np.float64), Jc)
    assert err <= (TOL32 if precision in ("f32", "f32_ds") else TOL64), err


# FP32 value path: the element work at the quadrature points runs in FP32, so R carries FP32
# rounding of the element contributions (unit roundoff 6e-8) amplified by the cancellations of the
# velocity gradient (level-surface gradient minus shear times slope) and of the assembly; the bar
# is normwise, like the FP32-lane Jacobian's.
TOL32_VALUES = 1e-5


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("kind", ["random", "zero", "sia"])
@pytest.mark.parametrize("scatter", ["atomic", "color"])
def test_fp32_value_path_parity(name, kind, scatter):
    c = capi()
    mesh = MESHES[name]()
    om = oracle.OracleMesh(mesh)
    U = velocities(mesh, kind, om)
    dm = c.DeviceMesh(mesh)
    J, R = dm.jacobian(dev(U), precision=c.BP_F32_ALL,
                       scatter=c.BP_SCATTER_ATOMIC if scatter == "atomic" else c.BP_SCATTER_COLOR)
    assert J.dtype == torch.float32
    _, _, Jc, Rc = om.jacobian(U)
    errR = rel_inf(R.cpu().numpy(), Rc)
    errJ = rel_inf(J.cpu().numpy().astype(np.float64), Jc)
    assert errR <= TOL32_VALUES, errR
    assert errJ <= TOL32, errJ
    if kind != "zero":    # at U = 0 the stress terms vanish and R is the memoised load exactly
        assert errR > 1e-13   # the value path did run in FP32


def test_fp32_value_path_rejects_dual_numbers():
    c = capi()
    mesh = synth.config_small()
    dm = c.DeviceMesh(mesh)
    with pytest.raises(c.BPError) as e:
        dm.jacobian(dev(np.zeros(mesh.ndof)), precision=c.BP_F32_ALL, method=c.BP_JAC_DUAL)
    assert e.value.status == c.BP_EUNSUP


def test_jacobian_without_residual_and_repeat_calls_overwrite():
    c = capi()
    mesh = synth.config_small()
    om = oracle.OracleMesh(mesh)
    U = synth.random_velocity(mesh, 7)
    dm = c.DeviceMesh(mesh)
    Ud = dev(U)
    J1, _ = dm.jacobian(Ud, want_residual=False)
    J2, _ = dm.jacobian(Ud, J=J1, want_residual=False)  # same buffer: overwritten, not accumulated
    _, _, Jc, _ = om.jacobian(U)
    assert rel_inf(J2.cpu().numpy(), Jc) <= TOL64
    R = dm.residual(Ud)
    R = dm.residual(Ud, R=R)
    assert rel_inf(R.cpu().numpy(), om.residual(U)) <= TOL64


def test_colored_scatter_is_deterministic():
    c = capi()
    mesh = ragged_mesh()
    dm = c.DeviceMesh(mesh)
    Ud = dev(synth.random_velocity(mesh, 9))
    a, ra = dm.jacobian(Ud, scatter=c.BP_SCATTER_COLOR)
    b, rb = dm.jacobian(Ud, scatter=c.BP_SCATTER_COLOR)
    assert torch.equal(a, b) and torch.equal(ra, rb)


def _sampled_rows(mesh, nsample, seed):
    rng = np.random.default_rng(seed)
    verts = np.unique(rng.choice(mesh.nv, nsample, replace=False))
    mask = np.isin(mesh.tri, verts).any(axis=1)
    rows = np.concatenate([mesh.dof(verts, l, c) for l in range(mesh.nlayers + 1) for c in (0, 1)])
    return verts, mask, np.sort(rows)


@pytest.mark.slow
def test_full_size_dome_1m_wedges_sampled_parity():
    """Dome, 100,352 triangles x 10 layers: full-size launch, outputs checked on sampled rows.

    The oracle assembles only the columns touching 64 sampled base vertices, which is exactly
    what those vertices' rows receive."""
    c = capi()
    mesh = synth.config_medium()
    om = oracle.OracleMesh(mesh)
    U = om.sia() + synth.random_velocity(mesh, 205, amplitude=20.0)
    dm = c.DeviceMesh(mesh)
    assert dm.nnz == mesh.expected_nnz() == 43719548
    Ud = dev(U)
    verts, mask, rows = _sampled_rows(mesh, 64, 11)
    R = dm.residual(Ud).cpu().numpy()
    Rc = om.residual(U, tri_mask=mask)
    assert rel_inf(R[rows], Rc[rows]) <= TOL64
    rowptr, colidx = (t.cpu().numpy() for t in dm.pattern())
    for prec, tol in ((c.BP_F64, TOL64), (c.BP_F32, TOL32), (c.BP_F64X2, TOL64), (c.BP_F32_DS, TOL32),
                      (c.BP_F64X2_DS, TOL64)):
        J, Rj = dm.jacobian(Ud, precision=prec)
        J = J.cpu().numpy().astype(np.float64)
        assert rel_inf(Rj.cpu().numpy()[rows], Rc[rows]) <= TOL64
        # oracle element matrices of the masked columns, scattered into a dict of sampled rows
        want = {}
        rowset = set(rows.tolist())
        for t in np.nonzero(mask)[0]:
            for l in range(mesh.nlayers):
                _, Ke = om.element(U, int(t), l)
                d = [int(mesh.dof(mesh.tri[t, a], l + k, cc)) for k in (0, 1) for a in range(3) for cc in (0, 1)]
                for i in range(12):
                    if d[i] in rowset:
                        for j in range(12):
                            want[(d[i], d[j])] = want.get((d[i], d[j]), 0.0) + Ke[i, j]
        got = np.empty(len(want))
        ref = np.empty(len(want))
        for n, ((r, col), v) in enumerate(want.items()):
            lo, hi = rowptr[r], rowptr[r + 1]
            p = lo + np.searchsorted(colidx[lo:hi], col)
            assert colidx[p] == col
            got[n], ref[n] = J[p], v
        assert rel_inf(got, ref) <= tol
        # every entry of the sampled rows that no element touches stays zero
        assert len(want) == sum(rowptr[r + 1] - rowptr[r] for r in rows)


def test_status_codes_from_device_side_calls():
    c = capi()
    mesh = synth.config_small()
    dm = c.DeviceMesh(mesh)
    U = dev(np.zeros(mesh.ndof))
    J = torch.empty(dm.nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(c.BPError) as e:
        c.bp_assemble_jacobian(dm.handle, U, None, J, precision=7)
    assert e.value.status == c.BP_EINVAL
    with pytest.raises(c.BPError) as e:
        c.bp_assemble_jacobian(dm.handle, U, None, J, method=9)
    assert e.value.status == c.BP_EINVAL
    with pytest.raises(c.BPError) as e:
        c.bp_assemble_jacobian(dm.handle, U, None, J, precision=c.BP_F64X2, method=c.BP_JAC_DUAL)
    assert e.value.status == c.BP_EUNSUP


def test_paired_fp32_lanes_closer_to_oracle_than_fp32():
    """The paired-FP32 lanes carry ~46 significant bits: their Jacobian sits at FP64 rounding
    distance from the native-FP64 one, orders of magnitude closer than the FP32-lane Jacobian."""
    c = capi()
    mesh = ragged_mesh()
    dm = c.DeviceMesh(mesh)
    Ud = dev(synth.random_velocity(mesh, 17))
    J64, _ = dm.jacobian(Ud, precision=c.BP_F64, scatter=c.BP_SCATTER_COLOR)
    J2, _ = dm.jacobian(Ud, precision=c.BP_F64X2, scatter=c.BP_SCATTER_COLOR)
    J32, _ = dm.jacobian(Ud, precision=c.BP_F32, scatter=c.BP_SCATTER_COLOR)
    scale = float(J64.abs().max())
    e2 = float((J2 - J64).abs().max()) / scale
    e32 = float((J32.double() - J64).abs().max()) / scale
    assert e2 <= 1e-13 and e32 >= 1e-9 and e2 <= 1e-4 * e32, (e2, e32)



@pytest.mark.parametrize("precision", ["f64", "f32", "f64x2_ds", "f32_ds"])
def test_tail_split_columns_match_oracle(precision):
    """A mesh a little larger than one wave of resident threads (39,200 columns against 37,888 on a
    B300): the atomic launches take the last partial wave's columns in layer segments.  R and J
    over the whole mesh against the oracle, and against the coloured scatter (whole columns)."""
    c = capi()
    mesh = synth.dome_mesh(140, 5, 91, 92, bed="sinusoidal", beta="field")
    assert mesh.ntri == 39200
    om = oracle.OracleMesh(mesh)
    U = synth.random_velocity(mesh, 93)
    dm = c.DeviceMesh(mesh)
    prec = {"f64": c.BP_F64, "f32": c.BP_F32, "f64x2_ds": c.BP_F64X2_DS, "f32_ds": c.BP_F32_DS}[precision]
    J, R = dm.jacobian(dev(U), precision=prec, scatter=c.BP_SCATTER_ATOMIC)
    _, _, Jc, Rc = om.jacobian_colored(U, 8)
    assert rel_inf(R.cpu().numpy(), Rc) <= TOL64
    tol = TOL32 if precision in ("f32", "f32_ds") else TOL64
    assert rel_inf(J.cpu().numpy().astype(np.float64), Jc) <= tol
    Jk, Rk = dm.jacobian(dev(U), precision=prec, scatter=c.BP_SCATTER_COLOR)
    assert rel_inf(R.cpu().numpy(), Rk.cpu().numpy()) <= TOL64
    if precision == "f64":
        Rr = dm.residual(dev(U))
        assert rel_inf(Rr.cpu().numpy(), Rc) <= TOL64

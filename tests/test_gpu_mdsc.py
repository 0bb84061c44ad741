"""MDSC two-level preconditioner on the GPU (through the C ABI) against the oracle's cycle.

Bar: bp_mdsc_apply equals the oracle's symmetric cycle (the same Jacobian values, omega, Chebyshev
steps and Gershgorin interval) to 1e-9 normwise in FP64 -- rounding amplified by the two column
solves (block condition numbers up to ~1e5) and the plane iteration -- and, with FP32 factors and
arithmetic, to 20 unit roundoffs of FP32 times the largest column-block condition number (the
block elimination is backward stable; the cycle applies it twice); Newton with the MDSC cycle reaches
the same solution as with the column solve, in fewer CG iterations."""
import numpy as np
import pytest

import oracle
from oracle import mdsc
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


@pytest.mark.parametrize("m,L", [(10, 4), (14, 1), (16, 10)])
@pytest.mark.parametrize("precision", [0, 1])
def test_mdsc_cycle_matches_oracle(m, L, precision):
    c = capi()
    mesh = synth.dome_mesh(m, L, 61, 62, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    U = om.sia()
    dm = c.DeviceMesh(mesh)
    J, _ = dm.jacobian(dev(U), precision=precision)
    c.bp_mdsc_setup(dm.handle, J, precision=precision)
    Jh = J.cpu().numpy().astype(np.float64)
    Js = om.jacobian_scipy(U)[0].tocsr()  # the same pattern, in the same order
    Js.data[:] = Jh                      # the cycle of the same (for FP32: rounded) matrix
    tl = mdsc.TwoLevel(Js, mesh.nv, L)
    r = np.random.default_rng(9).normal(size=dm.ndof)
    z = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    c.bp_mdsc_apply(dm.handle, J, dev(r), z)
    err = rel_inf(z.cpu().numpy(), tl.apply(r))
    if precision == 0:
        tol = 1e-9
    else:
        tol = max(1e-4, 20 * 2.0**-24 * max(np.linalg.cond(T) for T in tl.T))
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("precision", [0, 1])
def test_newton_with_mdsc_reaches_the_same_solution_in_fewer_cg_iterations(precision):
    c = capi()
    mesh = synth.dome_mesh(24, 5, 71, 72, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    out = {}
    for prec_kind in (c.BP_PREC_COLUMN, c.BP_PREC_MDSC):
        U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
        rc, rep = c.bp_newton_solve(dm.handle, U, precision=precision, preconditioner=prec_kind)
        assert rc == c.BP_OK, rep
        Uh = U.cpu().numpy()
        assert np.linalg.norm(om.residual(Uh)) <= 1.1e-8 * np.linalg.norm(om.residual(np.zeros_like(Uh)))
        out[prec_kind] = (Uh, rep)
    (Uc, rc_), (Um, rm) = out[c.BP_PREC_COLUMN], out[c.BP_PREC_MDSC]
    assert rel_inf(Um, Uc) <= 1e-6
    assert rm["krylov_iters"] < rc_["krylov_iters"]
    with pytest.raises(c.BPError):
        c.bp_newton_solve(dm.handle, U, preconditioner=7)


def test_mdsc_apply_needs_setup_and_aligned_vectors():
    c = capi()
    mesh = synth.config_small()
    dm = c.DeviceMesh(mesh)
    J, _ = dm.jacobian(dev(np.zeros(mesh.ndof)))
    r = torch.zeros(dm.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(c.BPError) as e:
        c.bp_mdsc_apply(dm.handle, J, r, torch.empty_like(r))
    assert e.value.status == c.BP_EINVAL


@pytest.mark.parametrize("m,L", [(10, 4), (16, 10), (30, 3)])
@pytest.mark.parametrize("precision", [0, 1])
def test_mdsc_amg_hierarchy_and_cycle_match_oracle(m, L, precision):
    """The SA-AMG plane hierarchy: level sizes and every aggregate equal the oracle's (integer work,
    bit-exact); the cycle equals the oracle's TwoLevelAMG cycle on the same Jacobian values."""
    c = capi()
    mesh = synth.dome_mesh(m, L, 61, 62, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    U = om.sia()
    dm = c.DeviceMesh(mesh)
    J, _ = dm.jacobian(dev(U), precision=precision)
    c.bp_mdsc_amg_setup(dm.handle, J, precision=precision)
    Jh = J.cpu().numpy().astype(np.float64)
    Js = om.jacobian_scipy(U)[0].tocsr()
    Js.data[:] = Jh
    tl = mdsc.TwoLevelAMG(Js, mesh.nv, L, mesh.tri)
    sizes = c.bp_mdsc_amg_levels(dm.handle)
    assert sizes == tl.amg.sizes()
    for k, agg in enumerate(tl.amg.agg):
        assert np.array_equal(c.bp_mdsc_amg_aggregates(dm.handle, k, sizes[k]), agg), k
    r = np.random.default_rng(9).normal(size=dm.ndof)
    z = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    c.bp_mdsc_amg_apply(dm.handle, J, dev(r), z)
    err = rel_inf(z.cpu().numpy(), tl.apply(r))
    if precision == 0:
        tol = 1e-9
    else:
        tol = max(1e-4, 20 * 2.0**-24 * max(np.linalg.cond(T) for T in tl.T))
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("precision", [0, 1])
def test_newton_with_mdsc_amg_reaches_the_same_solution(precision):
    c = capi()
    mesh = synth.dome_mesh(24, 5, 71, 72, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    out = {}
    for prec_kind in (c.BP_PREC_COLUMN, c.BP_PREC_MDSC_AMG):
        U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, U)
        rc, rep = c.bp_newton_solve(dm.handle, U, precision=precision, preconditioner=prec_kind)
        assert rc == c.BP_OK, rep
        Uh = U.cpu().numpy()
        assert np.linalg.norm(om.residual(Uh)) <= 1.1e-8 * np.linalg.norm(om.residual(np.zeros_like(Uh)))
        out[prec_kind] = (Uh, rep)
    (Uc, rc_), (Um, rm) = out[c.BP_PREC_COLUMN], out[c.BP_PREC_MDSC_AMG]
    assert rel_inf(Um, Uc) <= 1e-6
    assert rm["krylov_iters"] < rc_["krylov_iters"]
    with pytest.raises(c.BPError) as e:
        c.bp_mdsc_amg_aggregates(dm.handle, 99, 10)
    assert e.value.status == c.BP_EINVAL

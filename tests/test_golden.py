"""Stored oracle values (tests/golden/): the oracle against its own committed output, and the CUDA
path against the stored values.

The fixture holds the residual on 200 rows, 200 Jacobian entries, the residual norm and the
discrete energy on the 10,240-wedge dome at seeded velocities (header of the file: Sec. 2, Sec. 3.1
Eq. residual and Eq. linearsystem).  The oracle must reproduce it to rounding (it is deterministic;
the slack covers another compiler's contraction choices); the GPU must match it within the FP64
parity bar (1e-12 of the largest residual / Jacobian entry, normwise as in the other parity tests).
"""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402
import oracle  # noqa: E402

TOL_ORACLE = 1e-13
TOL_GPU = 1e-12


@pytest.fixture(scope="module")
def stored():
    return make_golden.load()


def test_oracle_reproduces_stored_values(stored):
    scal, rows, ents = stored
    mesh, U = make_golden.cases()
    om = oracle.OracleMesh(mesh)
    rowptr, colidx, vals, R = om.jacobian(U)
    assert om.ndof == int(scal["ndof"]) and colidx.shape[0] == int(scal["nnz"])
    assert float(np.linalg.norm(R)) == pytest.approx(scal["norm2_R"], rel=TOL_ORACLE)
    assert om.energy(U) == pytest.approx(scal["energy"], rel=TOL_ORACLE)
    rmax, jmax = scal["max_abs_R"], scal["max_abs_J"]
    assert max(abs(R[i] - v) for i, v in rows) <= TOL_ORACLE * rmax
    for i, j, v in ents:
        k = rowptr[i] + int(np.searchsorted(colidx[rowptr[i]:rowptr[i + 1]], j))
        assert colidx[k] == j
        assert abs(vals[k] - v) <= TOL_ORACLE * jmax


@pytest.mark.gpu
def test_gpu_matches_stored_values(stored):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2204_04321_b300 import capi
    scal, rows, ents = stored
    mesh, U = make_golden.cases()
    dm = capi.DeviceMesh(mesh)
    Ud = torch.as_tensor(np.ascontiguousarray(U), device="cuda")
    J, R = dm.jacobian(Ud)
    rowptr, colidx = (t.cpu().numpy() for t in dm.pattern())
    R, J = R.cpu().numpy(), J.cpu().numpy()
    assert float(np.linalg.norm(R)) == pytest.approx(scal["norm2_R"], rel=TOL_GPU)
    assert capi.bp_energy(dm.handle, Ud) == pytest.approx(scal["energy"], rel=TOL_GPU)
    assert max(abs(R[i] - v) for i, v in rows) <= TOL_GPU * scal["max_abs_R"]
    for i, j, v in ents:
        k = rowptr[i] + int(np.searchsorted(colidx[rowptr[i]:rowptr[i + 1]], j))
        assert colidx[k] == j
        assert abs(J[k] - v) <= TOL_GPU * scal["max_abs_J"]
    dm.close()

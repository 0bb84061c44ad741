"""Ensemble assembly (one persistent launch over uneven meshes) against the oracle, per member.

Every tuning candidate (columns per block x scatter mode) is checked, plus the autotuned choice
replayed from its CUDA graph twice (outputs are overwritten, not accumulated)."""
import numpy as np
import pytest

import oracle
from paper_2204_04321_b300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def rel_inf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def members():
    ms = synth.ensemble_members(count=6, scale=0.03)   # 150 .. 1,500 triangles, 5 .. 20 layers each
    refs = []
    for i, m in enumerate(ms):
        om = oracle.OracleMesh(m)
        U = synth.random_velocity(m, 500 + i)
        _, _, Jc, Rc = om.jacobian(U)
        refs.append((U, Rc, Jc))
    return ms, refs


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_every_candidate_matches_oracle_per_member(members, precision, tol):
    from paper_2204_04321_b300 import capi
    ms, refs = members
    ens = capi.Ensemble(ms, [torch.as_tensor(r[0], device="cuda") for r in refs], precision=precision)
    assert len({m.nlayers for m in ms}) > 1 and len({m.ntri for m in ms}) == len(ms)
    for cpb, sc in capi.Ensemble.CANDIDATES:
        ens.select(cpb, sc)
        ens.assemble()
        torch.cuda.synchronize()
        for i, (U, Rc, Jc) in enumerate(refs):
            assert rel_inf(ens.R[i].cpu().numpy(), Rc) <= 1e-12, (cpb, sc, i)
            assert rel_inf(ens.J[i].cpu().numpy().astype(np.float64), Jc) <= tol, (cpb, sc, i)
    times, chosen = ens.tune(reps=2)
    assert chosen in capi.Ensemble.CANDIDATES and all(t > 0 for t in times.values())
    for _ in range(2):
        ens.assemble()
    torch.cuda.synchronize()
    for i, (U, Rc, Jc) in enumerate(refs):
        assert rel_inf(ens.R[i].cpu().numpy(), Rc) <= 1e-12
        assert rel_inf(ens.J[i].cpu().numpy().astype(np.float64), Jc) <= tol
    ens.close()


def test_misaligned_velocity_is_rejected():
    from paper_2204_04321_b300 import capi
    m = synth.dome_mesh(4, 2, 1, 2)
    dm = capi.DeviceMesh(m)
    buf = torch.zeros(dm.ndof + 1, dtype=torch.float64, device="cuda")
    R = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.BPError) as e:
        capi.bp_assemble_residual(dm.handle, buf[1:], R)   # 8-byte, not 16-byte aligned
    assert e.value.status == capi.BP_EINVAL


def test_misaligned_fp32_jacobian_is_rejected():
    from paper_2204_04321_b300 import capi
    m = synth.dome_mesh(4, 2, 1, 2)
    dm = capi.DeviceMesh(m)
    U = torch.zeros(dm.ndof, dtype=torch.float64, device="cuda")
    Jbuf = torch.zeros(dm.nnz + 1, dtype=torch.float32, device="cuda")
    for prec in (capi.BP_F32, capi.BP_F32_ALL):
        with pytest.raises(capi.BPError) as e:
            capi.bp_assemble_jacobian(dm.handle, U, None, Jbuf[1:], prec)   # 4-byte, not 8-byte aligned
        assert e.value.status == capi.BP_EINVAL

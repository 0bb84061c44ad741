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


@pytest.mark.slow
def test_full_ensemble_64_members_sampled_rows_match_oracle():
    """The 64-member ensemble of the benchmark (5k-50k triangles, 5-20 layers each, 19.5 M wedges)
    in one autotuned persistent launch: on every member, the rows of 3 sampled base vertices (all
    levels, both components) against the oracle's element loop over the columns touching them."""
    from paper_2204_04321_b300 import capi
    ms = synth.ensemble_members()
    Us = [synth.random_velocity(m, 500 + i) for i, m in enumerate(ms)]
    ens = capi.Ensemble(ms, [torch.as_tensor(u, device="cuda") for u in Us], precision=capi.BP_F64)
    ens.tune(reps=1)
    ens.assemble()
    torch.cuda.synchronize()
    worst_r = worst_j = 0.0
    for i, (m, U) in enumerate(zip(ms, Us)):
        om = oracle.OracleMesh(m)
        rng = np.random.default_rng(7000 + i)
        verts = np.unique(rng.choice(m.nv, 3, replace=False))
        mask = np.isin(m.tri, verts).any(axis=1)
        rows = np.sort(np.concatenate([m.dof(verts, l, c) for l in range(m.nlayers + 1) for c in (0, 1)]))
        Rc = om.residual(U, tri_mask=mask)
        R = ens.R[i].cpu().numpy()
        worst_r = max(worst_r, rel_inf(R[rows], Rc[rows]))
        rowptr, colidx = (t.cpu().numpy() for t in ens.dms[i].pattern())
        J = ens.J[i].cpu().numpy()
        want = {}
        rowset = set(rows.tolist())
        for t in np.nonzero(mask)[0]:
            for l in range(m.nlayers):
                _, Ke = om.element(U, int(t), l)
                d = [int(m.dof(m.tri[t, a], l + k, cc)) for k in (0, 1) for a in range(3) for cc in (0, 1)]
                for a in range(12):
                    if d[a] in rowset:
                        for b in range(12):
                            want[(d[a], d[b])] = want.get((d[a], d[b]), 0.0) + Ke[a, b]
        got = np.array([J[rowptr[r] + np.searchsorted(colidx[rowptr[r]:rowptr[r + 1]], c)] for (r, c) in want])
        ref = np.array(list(want.values()))
        worst_j = max(worst_j, rel_inf(got, ref))
        assert len(want) == sum(rowptr[r + 1] - rowptr[r] for r in rows)   # no other entry is touched
    assert worst_r <= 1e-12 and worst_j <= 1e-12, (worst_r, worst_j)
    ens.close()

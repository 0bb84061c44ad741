"""What the trained warm-start network gains, measured on unseen beta fields (GPU).

The committed network (paper_2204_04321_b300/weights, trained by `learned.py train` on 2,000
solutions of the 1M-wedge dome geometry) is checked for what it does gain and for what each
fallback rule guarantees:
  * its predicted profile scales beat the "no correction" (shallow-ice) baseline on unseen fields;
  * its guess is much closer to the converged solution than the shallow-ice guess, and the FP64
    energy judge, which measures that distance (Pi(U) - Pi(U*) ~ 1/2 |U - U*|_J^2), keeps it;
  * the FP64 residual-norm judge never hands Newton a start with a larger residual than the
    shallow-ice one, so the residual-judged solve is never worse than the shallow-ice solve;
  * either start reaches the same solution.
Newton steps alone do not profit from the closer guess: from any of these starts the first
residual is ~0.8 of F(0) (rough, high-frequency error components that no per-column guess
removes) and Newton overshoots from a rough start.  Picard (fixed-viscosity) steps do not
overshoot: the energy-judged guess followed by Picard steps until ||F|| <= 0.1 ||F(0)|| takes
fewer nonlinear steps than the shallow-ice start, where the same Picard steps from the shallow-ice
guess do not help."""
import numpy as np
import pytest

import oracle
from oracle import learned as olearn
from oracle import mlp as omlp

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def capi():
    from paper_2204_04321_b300 import capi as c
    return c


def rel_inf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("layers", [10, 4])
def test_decoder_matches_oracle(layers):
    """bp_learned_decode against the oracle's decoder on the oracle's shallow-ice guess, element by
    element (the nodal surface gradient behind both guesses is summed in different orders)."""
    from paper_2204_04321_b300 import synth
    c = capi()
    mesh = synth.dome_mesh(23, layers, 61, 62, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    Y = (np.random.default_rng(5).normal(size=(mesh.nv, 32)) * 0.5).astype(np.float32)
    U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    c.bp_learned_decode(dm.handle, torch.as_tensor(Y, device="cuda"), U)
    want = olearn.decode(Y, om.sia(), mesh.nv, layers)
    assert rel_inf(U.cpu().numpy(), want) <= 1e-12
    dm.close()


def test_training_targets_match_oracle():
    """bp_learned_targets (the per-column regularised profile fit) against the oracle's statement."""
    from paper_2204_04321_b300 import learned, synth
    c = capi()
    mesh = synth.dome_mesh(30, 10, 63, 64, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    S = om.sia()
    rng = np.random.default_rng(6)
    # a solution-like field: the shallow-ice profile rescaled per column, plus noise of 5 % of the
    # column's speed
    col = np.abs(S.reshape(mesh.nv, 22)).max(axis=1)
    noise = (rng.normal(size=(mesh.nv, 22)) * 0.05 * col[:, None]).reshape(-1)
    Uh = olearn.decode(rng.normal(size=(mesh.nv, 32)) * 0.4, S, mesh.nv, 10) + noise
    dm = c.DeviceMesh(mesh)
    T = torch.full((mesh.nv, 32), 9.0, dtype=torch.float32, device="cuda")
    c.bp_learned_targets(dm.handle, torch.as_tensor(Uh, device="cuda"), learned.FIT_REG, T)
    T = T.double().cpu().numpy()
    fit = lambda S_: olearn.profile_scales(Uh.reshape(mesh.nv, 11, 2), S_.reshape(mesh.nv, 11, 2), reg=learned.FIT_REG)
    want = fit(S)
    # tolerance: how far the oracle's own targets move when its shallow-ice input moves by 1e-13 of
    # each column's speed (the two guesses differ by ~1e-15 of it: atomics in the nodal surface
    # gradient), which matters only on ill-conditioned columns, plus the FP32 rounding of the output
    spread = np.zeros_like(want)
    for k in range(4):
        dS = (np.random.default_rng(100 + k).uniform(-1, 1, size=(mesh.nv, 22)) * 1e-13 * col[:, None]).reshape(-1)
        spread = np.maximum(spread, np.abs(fit(S + dS) - want))
    tol = 2 * spread + 2.0 ** -22 * np.maximum(1.0, np.abs(want))
    assert np.all(T[:, 4:] == 0)
    assert np.all(np.abs(T[:, :4] - want) <= tol), float((np.abs(T[:, :4] - want) - tol).max())
    moving = col > 1e-6 * col.max()
    assert np.mean(spread[moving] < 1e-6) > 0.95   # the comparison is tight on almost every moving column
    assert np.abs(want).max() > 0.1
    with pytest.raises(c.BPError):
        c.bp_learned_targets(dm.handle, torch.as_tensor(Uh, device="cuda"), -1.0, torch.empty_like(torch.as_tensor(T)).cuda())
    dm.close()


def constant_network(scales):
    """A network whose weights and hidden biases are zero: its output is b4 for every column, so the
    decoded guess is the shallow-ice profile with these exact (dyadic) scales."""
    P = omlp.unflatten(np.zeros(omlp.NPARAM))
    P["b4"][:4] = scales
    return omlp.flatten(P)


@pytest.mark.parametrize("judge", [0, 1, 2])
def test_learned_guess_matches_oracle_under_every_judge(judge):
    """bp_initial_guess_learned (shallow-ice guess, features, network, decoder, judge) against the
    oracle's pipeline, element by element, for networks the judge keeps and networks it rejects."""
    from paper_2204_04321_b300 import synth
    c = capi()
    mesh = synth.dome_mesh(30, 10, 201, 202, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    net = c.Mlp(seed=1)
    U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    decisions = []
    # on this mesh the oracle keeps the guesses with 12.5 % and 6.25 % less deformation under both
    # judges and rejects the others
    for scales in ([0.0, -0.125, 0.0, -0.125], [0.25, -0.5, 0.25, -0.5], [2.0, 2.0, 2.0, 2.0],
                   [0.0, -0.0625, 0.0, -0.0625], [0.0, 0.125, 0.0, 0.125], [-0.5, -0.25, -0.5, -0.25]):
        p = constant_network(scales)
        net.set_params(p.astype(np.float32))
        used = c.bp_initial_guess_learned(dm.handle, net, U, judge=judge)
        Uo, used_o, _, (f_net, f_sia) = olearn.learned_guess(om, p, judge)
        if judge != olearn.JUDGE_NONE and abs(f_net - f_sia) <= 1e-9 * abs(f_sia):
            continue   # a tie within rounding: either decision is correct
        assert used == used_o, (scales, f_net, f_sia)
        assert rel_inf(U.cpu().numpy(), Uo) <= 1e-12
        decisions.append(used)
    if judge != olearn.JUDGE_NONE:
        assert True in decisions and False in decisions   # both branches of the judge were exercised
    dm.close()


@pytest.mark.parametrize("judge", [0, 1, 2])
def test_trained_network_guess_matches_oracle_on_certified_columns(judge):
    """The committed trained network through the whole pipeline.  On columns whose features and
    hidden BF16 roundings the oracle certifies as fixed by the arithmetic, the guess must agree
    within the bound that FP32 accumulation of the last layer leaves on the outputs; the judge's
    decision must agree unless the two measures tie within rounding."""
    from paper_2204_04321_b300 import learned, synth
    c = capi()
    mesh = synth.dome_mesh(40, 10, 201, 202, bed="sinusoidal", beta="field")
    om = oracle.OracleMesh(mesh)
    dm = c.DeviceMesh(mesh)
    net = c.Mlp()
    net.load(learned.DEFAULT_WEIGHTS)
    p = net.get_params().astype(np.float64)
    U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    used = c.bp_initial_guess_learned(dm.handle, net, U, judge=judge)
    U = U.cpu().numpy()
    X = olearn.features(mesh)
    Uo, used_o, Y, (f_net, f_sia) = olearn.learned_guess(om, p, judge, X=X)
    S = om.sia()
    if judge != olearn.JUDGE_NONE and abs(f_net - f_sia) > 1e-6 * abs(f_sia):
        assert used == used_o, (f_net, f_sia)
    if not used:
        assert not used_o or abs(f_net - f_sia) <= 1e-6 * abs(f_sia)
        assert rel_inf(U, S) <= 1e-12
        return
    ok_f = np.all(olearn.feature_fp32_margin(mesh) > 1e-12, axis=1)
    ok_n, ybound = olearn.forward_certificate(p, X)
    ok = ok_f & ok_n
    assert ok.mean() >= 0.3, float(ok.mean())   # (small hidden activations leave the rest near a boundary)
    Sc = S.reshape(mesh.nv, 11, 2)
    b = Sc[:, :1, :]
    ub = np.stack([ybound[:, 0][:, None] * np.abs(b[:, :, 0]) + ybound[:, 1][:, None] * np.abs(Sc[:, :, 0] - b[:, :, 0]),
                   ybound[:, 2][:, None] * np.abs(b[:, :, 1]) + ybound[:, 3][:, None] * np.abs(Sc[:, :, 1] - b[:, :, 1])],
                  axis=2)
    err = np.abs(U - olearn.decode(Y, S, mesh.nv, 10)).reshape(mesh.nv, 11, 2)
    slack = 1e-12 * np.abs(U).max()
    assert np.all(err[ok] <= ub[ok] + slack), float((err[ok] - ub[ok]).max())
    assert err[~ok].max(initial=0.0) <= 5e-2 * np.abs(U).max()
    dm.close()


@pytest.mark.slow
def test_trained_network_gain_on_unseen_beta_fields():
    from paper_2204_04321_b300 import capi, learned, synth
    mesh = learned.geometry()
    net = capi.Mlp()
    net.load(learned.DEFAULT_WEIGHTS)
    X, T, _ = learned.generate(mesh, [learned.TEST_SEED0 + 100 + k for k in range(4)], 4096)
    loss_net, _ = net.gradient(X, T)
    loss_sia = float((T[:, :22].double() ** 2).sum(1).mean())   # prediction y = 0: the shallow-ice scales
    assert loss_net < 0.8 * loss_sia, (loss_net, loss_sia)
    rows = learned.evaluate(net, mesh, [learned.TEST_SEED0 + 200 + k for k in range(4)],
                            guesses=("sia", "learned", "learned_energy", "learned_picard"))
    # the energy-judged guess followed by Picard steps takes fewer nonlinear steps than the
    # shallow-ice start (40 unseen fields: 11.0 against 14.4 on average, time ratio 1.12)
    assert all(r["learned_picard"]["converged"] for r in rows)
    assert sum(r["learned_picard"]["newton_iters"] for r in rows) <= sum(r["sia"]["newton_iters"] for r in rows)
    for r in rows:
        sia, res, en = r["sia"], r["learned"], r["learned_energy"]
        assert sia["converged"] and res["converged"] and en["converged"]
        # residual judge: the start handed to Newton never has the larger FP64 residual
        assert res["initial_rel_residual"] <= sia["initial_rel_residual"] * (1 + 1e-12)
        assert res["newton_iters"] <= sia["newton_iters"] or res["learned_used"]
        # energy judge keeps the network guess, which is far closer to the solution
        assert en["learned_used"]
        assert en["guess_rel_err"] <= 0.6 * sia["guess_rel_err"], (en["guess_rel_err"], sia["guess_rel_err"])
        assert en["newton_iters"] <= sia["newton_iters"] + 2
    # same minimiser from either start
    dm = capi.DeviceMesh(mesh)
    capi.bp_mesh_set_beta(dm.handle, synth.lognormal_beta_field_torch(mesh.xy, learned.TEST_SEED0 + 200, "cuda"))
    Ua, _ = learned.solve(dm, capi.BP_F64, "sia")
    Ub, _ = learned.solve(dm, capi.BP_F64, "learned_energy", mlp=net)
    assert float((Ua - Ub).abs().max() / Ua.abs().max()) <= 1e-6

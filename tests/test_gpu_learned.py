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

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


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

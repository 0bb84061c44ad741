"""What the trained warm-start network gains, measured on unseen beta fields (GPU).

The committed network (paper_2204_04321_b300/weights, trained by `learned.py train` on 2,000
solutions of the 1M-wedge dome geometry) is checked for what it does gain -- its predicted
profile scales beat the "no correction" (shallow-ice) baseline on unseen fields -- and for what
the residual-judged fallback guarantees: a Newton solve from the learned guess never takes more
steps than from the shallow-ice guess and reaches the same solution."""
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
    rows = learned.evaluate(net, mesh, [learned.TEST_SEED0 + 200 + k for k in range(3)],
                            guesses=("sia", "learned"))
    for r in rows:
        assert r["sia"]["converged"] and r["learned"]["converged"]
        assert r["learned"]["newton_iters"] <= r["sia"]["newton_iters"]
        assert r["learned"]["initial_rel_residual"] <= r["sia"]["initial_rel_residual"] * (1 + 1e-12)
    # same minimiser from either start
    dm = capi.DeviceMesh(mesh)
    capi.bp_mesh_set_beta(dm.handle, synth.lognormal_beta_field_torch(mesh.xy, learned.TEST_SEED0 + 200, "cuda"))
    Ua, _ = learned.solve(dm, capi.BP_F64, "sia")
    Ub, _ = learned.solve(dm, capi.BP_F64, "learned", mlp=net)
    assert float((Ua - Ub).abs().max() / Ua.abs().max()) <= 1e-6

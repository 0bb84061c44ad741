"""Tensor-core MLP kernels (through the C ABI) against the CPU oracle of the same network.

The oracle rounds exactly the tensor-core operands to BF16 and accumulates in FP64; the kernels
accumulate in FP32 in an order of their own.  Two kinds of comparison follow from that:

* exact test networks (`synth.dyadic_mlp_case`): inputs, weights, biases and output errors are
  short dyadic fractions, so every sum the forward and backward passes form -- pre-activations,
  outputs, dW and bias gradients over the batch, dH over the outputs -- is exact in FP32 in any
  order (`oracle.learned.exact_case_certified` checks that for each input).  Outputs, loss and
  every gradient entry must then equal the oracle's bit for bit.
* random networks and inputs: per row the oracle tells whether any BF16 rounding of a hidden
  activation (or a ReLU sign) lies within an FP32 accumulation error of a rounding boundary
  (`oracle.learned.forward_certificate`, error model 2^-20 of the sum of term magnitudes, the
  bound for exact 16-term blocks accumulated 8 times); rows with none must agree within that
  model's bound on the last layer.  Every row stays within a couple of BF16 steps and nearly all
  within 1e-5 of the output scale.  Gradients of random batches (sums over all rows) are compared
  normwise.
"""
import os

import numpy as np
import pytest

from oracle import learned as olearn
from oracle import mlp as omlp
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


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def batch(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 16))
    X[:, 15] = 0.0
    Xb = torch.as_tensor(X, dtype=torch.float32).to(torch.bfloat16).cuda()
    T = torch.as_tensor(rng.normal(size=(n, 32)), dtype=torch.float32).cuda()
    return Xb, Xb.float().double().cpu().numpy(), T


def assert_certified_rows_match(params, X, Y):
    """Rows with no hidden rounding near a boundary agree within the last layer's accumulation bound;
    every row that a boundary flip can reach stays within a couple of BF16 steps, and nearly all rows
    agree to 1e-5 of the output scale.  (Small activations make most rows of a random network carry
    some rounding within the accumulation error of a boundary; whether it flips depends on the order.)"""
    Yo, _ = omlp.forward(np.asarray(params, dtype=np.float64), X, bf16=True)
    ok, ybound = olearn.forward_certificate(params, X)
    err = np.abs(Y - Yo)
    assert np.all(err[ok] <= ybound[ok]), float((err[ok] - ybound[ok]).max())
    row = err.max(axis=1) / np.abs(Yo).max()
    assert row.max() <= 5e-3 and np.mean(row > 1e-5) <= 0.03, (float(row.max()), float(np.mean(row > 1e-5)))
    return float(np.mean(ok))


def dyadic_net(seed, n):
    c = capi()
    params, X, E = synth.dyadic_mlp_case(seed, n)
    net = c.Mlp(seed=1)
    net.set_params(params)
    assert np.array_equal(net.get_params(), params)
    Xb = torch.as_tensor(X, dtype=torch.float32).to(torch.bfloat16).cuda()
    assert np.array_equal(Xb.double().cpu().numpy(), X)   # the inputs are BF16 numbers
    return net, params.astype(np.float64), X, E, Xb


@pytest.mark.parametrize("n", [128, 300, 1000, 5000])
def test_forward_bit_exact_on_exact_network(n):
    net, p, X, E, Xb = dyadic_net(20 + n, n)
    ok, details = olearn.exact_case_certified(p, X, np.zeros((n, 32)), 0.0)
    assert all(v for k, v in details.items() if k.startswith("z")), details
    Y = net.forward(Xb).double().cpu().numpy()
    Yo, _ = omlp.forward(p, X, bf16=True)
    assert np.array_equal(Y, Yo), (int((Y != Yo).sum()), float(np.abs(Y - Yo).max()))


@pytest.mark.parametrize("n", [256, 1024])
def test_loss_and_gradient_bit_exact_on_exact_network(n):
    net, p, X, E, Xb = dyadic_net(40 + n, n)
    ok, details = olearn.exact_case_certified(p, X, E, 2.0 / n)
    assert ok, details
    Yo, _ = omlp.forward(p, X, bf16=True)
    T = Yo - E   # targets with exactly known output errors (exact FP32 numbers)
    assert np.array_equal(T.astype(np.float32).astype(np.float64), T)
    loss, g = net.gradient(Xb, torch.as_tensor(T, dtype=torch.float32).cuda())
    lo, go = omlp.loss_and_gradient(p, X, T, bf16=True)
    assert loss == lo
    g = g.double().cpu().numpy()
    off = 0
    for name, shp in omlp.SHAPES:   # every entry of every parameter block
        k = int(np.prod(shp))
        assert np.array_equal(g[off:off + k], go[off:off + k]), (name, float(np.abs(g[off:off + k] - go[off:off + k]).max()))
        off += k
    assert np.abs(go).max() > 0


@pytest.mark.parametrize("n", [128, 1000, 5000])
def test_forward_matches_oracle_on_certified_rows(n):
    net = capi().Mlp(seed=3)
    Xb, X, _ = batch(n, n)
    Y = net.forward(Xb).double().cpu().numpy()
    frac = assert_certified_rows_match(net.get_params().astype(np.float64), X, Y)
    assert frac >= 0.08


@pytest.mark.parametrize("n", [256, 1000])
def test_gradient_matches_oracle_normwise(n):
    net = capi().Mlp(seed=4)
    Xb, X, T = batch(n, 10 + n)
    loss, g = net.gradient(Xb, T)
    lo, go = omlp.loss_and_gradient(net.get_params().astype(np.float64), X, T.double().cpu().numpy(), bf16=True)
    assert loss == pytest.approx(lo, rel=1e-5)
    g = g.double().cpu().numpy()
    # per parameter block (the bias and weight gradients differ in scale); a BF16 flip of one
    # uncertified activation moves the sums by ~1e-3 of a block (the exact network fixes every entry)
    off = 0
    for name, shp in omlp.SHAPES:
        k = int(np.prod(shp))
        assert rel(g[off:off + k], go[off:off + k]) <= 3e-3, name
        off += k


def test_adam_first_step_and_training_reduces_loss():
    net = capi().Mlp(seed=5)
    Xb, X, T = batch(2048, 77)
    p0 = net.get_params().astype(np.float64)
    _, g = net.gradient(Xb, T)
    g = g.double().cpu().numpy()
    lr = 1e-3
    net.train_step(Xb, T, lr)
    dp = net.get_params().astype(np.float64) - p0
    big = np.abs(g) > 1e-2 * np.abs(g).max()
    # first Adam step: m_hat = g, v_hat = g^2  =>  delta = -lr g / (|g| + eps)
    np.testing.assert_allclose(dp[big], -lr * np.sign(g[big]), rtol=0, atol=1e-6)
    l0 = net.gradient(Xb, T)[0]
    for _ in range(300):
        net.train_step(Xb, T, 2e-3)
    assert net.gradient(Xb, T)[0] < 0.5 * l0


def test_params_roundtrip_and_set_resets():
    net = capi().Mlp(seed=6)
    p = net.get_params()
    q = (np.random.default_rng(0).normal(size=p.shape) * 0.1).astype(np.float32)
    net.set_params(q)
    assert np.array_equal(net.get_params(), q)
    Xb, X, _ = batch(300, 1)
    assert_certified_rows_match(q.astype(np.float64), X, net.forward(Xb).double().cpu().numpy())


def test_save_and_load_through_the_c_abi(tmp_path):
    """bp_mlp_save / bp_mlp_load write and read .npy files that numpy reads and writes too."""
    c = capi()
    net = c.Mlp(seed=8)
    path = str(tmp_path / "w.npy")
    net.save(path)
    assert np.array_equal(np.load(path), net.get_params())
    q = np.random.default_rng(1).normal(size=net.nparam).astype(np.float32)
    np.save(path, q)
    other = c.Mlp(seed=9)
    other.load(path)
    assert np.array_equal(other.get_params(), q)
    np.save(path, q[:-1])   # another array: refused, parameters unchanged
    with pytest.raises(c.BPError) as e:
        other.load(path)
    assert e.value.status == c.BP_EIO
    np.save(path, q.astype(np.float64))
    with pytest.raises(c.BPError) as e:
        other.load(path)
    assert e.value.status == c.BP_EIO
    with pytest.raises(c.BPError) as e:
        other.load(str(tmp_path / "missing.npy"))
    assert e.value.status == c.BP_EIO
    assert np.array_equal(other.get_params(), q)


def test_features_match_oracle():
    """The 16 BF16 features equal the oracle's bit for bit, except where FP64 evaluation order could
    move a quantity across an FP32 rounding midpoint (none expected at this size)."""
    c = capi()
    mesh = synth.dome_mesh(30, 10, 201, 202, bed="sinusoidal", beta="field")
    dm = c.DeviceMesh(mesh)
    X = torch.empty(mesh.nv, 16, dtype=torch.bfloat16, device="cuda")
    c.bp_mlp_features(dm.handle, X)
    got = X.double().cpu().numpy()
    want = olearn.features(mesh)
    certain = olearn.feature_fp32_margin(mesh) > 1e-12
    assert certain.mean() > 0.97
    assert np.array_equal(got[certain], want[certain]), int((got[certain] != want[certain]).sum())
    bad = synth.dome_mesh(6, 5, 1, 2)
    dmb = c.DeviceMesh(bad)
    with pytest.raises(c.BPError) as e:
        c.bp_mlp_features(dmb.handle, X)
    assert e.value.status == c.BP_EUNSUP


def test_set_beta_matches_fresh_upload():
    c = capi()
    mesh = synth.dome_mesh(12, 10, 201, 202, bed="sinusoidal", beta="field")
    dm = c.DeviceMesh(mesh)
    beta2 = synth.lognormal_beta_field(mesh.xy, 999)
    c.bp_mesh_set_beta(dm.handle, beta2)
    mesh2 = synth.dome_mesh(12, 10, 201, 202, bed="sinusoidal", beta="field")
    mesh2.beta = beta2
    dm2 = c.DeviceMesh(mesh2)
    U = torch.as_tensor(synth.random_velocity(mesh, 3), device="cuda")
    J1, R1 = dm.jacobian(U, scatter=c.BP_SCATTER_COLOR)
    J2, R2 = dm2.jacobian(U, scatter=c.BP_SCATTER_COLOR)
    assert torch.equal(J1, J2)  # the coloured scatter is deterministic
    # R starts from the driving-stress load, summed with atomics at upload: equal up to summation order
    assert float((R1 - R2).abs().max() / R2.abs().max()) <= 1e-14
    bt = synth.lognormal_beta_field_torch(mesh.xy, 999, "cuda")
    assert np.abs(bt - beta2).max() <= 1e-12 * beta2.max()


def test_learned_guess_falls_back_to_shallow_ice_for_untrained_network():
    c = capi()
    mesh = synth.dome_mesh(40, 10, 201, 202, bed="sinusoidal", beta="field")
    dm = c.DeviceMesh(mesh)
    net = c.Mlp(seed=11)
    U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
    used = c.bp_initial_guess_learned(dm.handle, net, U)
    S = torch.empty_like(U)
    c.bp_initial_guess(dm.handle, c.BP_GUESS_SIA, S)
    assert not used  # the untrained network's residual is larger: the shallow-ice guess is returned
    assert float((U - S).abs().max() / S.abs().max()) <= 1e-13  # (its nodal gradient is summed with atomics)
    # the energy judge rejects it as well; with no judge the network's own guess is returned
    assert not c.bp_initial_guess_learned(dm.handle, net, U, judge=c.BP_JUDGE_ENERGY)
    assert float((U - S).abs().max() / S.abs().max()) <= 1e-13
    assert c.bp_initial_guess_learned(dm.handle, net, U, judge=c.BP_JUDGE_NONE)
    assert float((U - S).abs().max() / S.abs().max()) > 1e-3
    with pytest.raises(c.BPError) as e:
        c.bp_initial_guess_learned(dm.handle, net, U, judge=7)
    assert e.value.status == c.BP_EINVAL

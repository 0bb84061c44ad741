"""Pins of the learned warm start's oracle (oracle/learned.py) against what the definitions fix.

* decoder: zero outputs reproduce the shallow-ice guess; scales of -1 give zero velocity; keeping
  only the sliding or only the deformation part; the u outputs never touch v; a hand-set column
  in closed form;
* judge: the fallback rule on its cases (smaller, equal, larger, not finite);
* features: a per-vertex loop written independently (per-triangle 2 x 2 solves for the surface
  gradient, explicit neighbour averages) and the hi / lo reconstruction of the FP32 values;
* profile scales: exact recovery of the scales a target was built with (no regularisation), the
  stationarity of the regularised objective, and the singular-column rule;
* FP32 analysis: the exact-sum rule against exact rational sums of FP32 additions in random
  orders, the exact test networks evaluated in rational arithmetic, and a planted BF16 rounding
  tie that the forward certificate must flag.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import learned as ol
from oracle import mlp as omlp
from paper_2204_04321_b300 import synth


def test_decoder_special_cases():
    rng = np.random.default_rng(0)
    nv, L = 7, 10
    S = rng.normal(size=2 * nv * (L + 1)) * 50
    Sc = S.reshape(nv, L + 1, 2)
    U0 = ol.decode(np.zeros((nv, 32)), S, nv, L)
    assert np.abs(U0 - S).max() <= 1e-13 * np.abs(S).max()          # y = 0: the shallow-ice guess
    assert np.all(ol.decode(np.full((nv, 32), -1.0), S, nv, L) == 0)  # scales 0: no velocity
    Y = np.zeros((nv, 32))
    Y[:, 1] = Y[:, 3] = -1.0                                           # deformation parts removed
    Ub = ol.decode(Y, S, nv, L).reshape(nv, L + 1, 2)
    assert np.allclose(Ub, np.repeat(Sc[:, :1, :], L + 1, axis=1), rtol=0, atol=1e-12)
    Y = np.zeros((nv, 32))
    Y[:, 0] = Y[:, 2] = -1.0                                           # sliding parts removed
    Ud = ol.decode(Y, S, nv, L).reshape(nv, L + 1, 2)
    assert np.allclose(Ud, Sc - Sc[:, :1, :], rtol=0, atol=1e-12) and np.all(Ud[:, 0, :] == 0)
    Y = np.zeros((nv, 32))
    Y[:, 0], Y[:, 1] = 0.3, -0.7                                       # u outputs leave v alone
    Uu = ol.decode(Y, S, nv, L).reshape(nv, L + 1, 2)
    assert np.abs(Uu[:, :, 1] - Sc[:, :, 1]).max() <= 1e-13 * np.abs(S).max()
    Y[:, 4:] = 123.0                                                   # outputs 4.. are not read
    assert np.array_equal(ol.decode(Y, S, nv, L), Uu.reshape(-1))


def test_decoder_hand_column():
    # one column, 3 levels: u_sia = (10, 14, 20), v_sia = (-2, -2, 1); y = (0.5, -0.25, 1, 2)
    S = np.array([10.0, -2.0, 14.0, -2.0, 20.0, 1.0])
    Y = np.zeros((1, 32))
    Y[0, :4] = [0.5, -0.25, 1.0, 2.0]
    U = ol.decode(Y, S, 1, 2)
    # u: 1.5 * 10 + 0.75 * (u - 10) -> 15, 18, 22.5;  v: 2 * (-2) + 3 * (v + 2) -> -4, -4, 5
    assert np.array_equal(U, np.array([15.0, -4.0, 18.0, -4.0, 22.5, 5.0]))


def test_judge_rule():
    assert ol.judge_keep(1.0, 2.0) and ol.judge_keep(2.0, 2.0)
    assert not ol.judge_keep(2.0, 1.0)
    assert not ol.judge_keep(float("nan"), 1.0) and not ol.judge_keep(float("inf"), 1.0)


def test_features_against_a_direct_loop():
    mesh = synth.dome_mesh(5, 10, 31, 32, bed="sinusoidal", beta="iid")
    q, q8, q40 = ol.feature_quantities(mesh)
    s = mesh.bed + mesh.thick
    num = np.zeros((mesh.nv, 2))
    den = np.zeros(mesh.nv)
    for t in mesh.tri:
        P = mesh.xy[t]
        A = np.array([P[1] - P[0], P[2] - P[0]])               # rows: edge vectors
        g = np.linalg.solve(A, np.array([s[t[1]] - s[t[0]], s[t[2]] - s[t[0]]]))
        area = 0.5 * abs(np.linalg.det(A))
        for a in t:
            num[a] += area * g
            den[a] += area
    gx, gy = num[:, 0] / den, num[:, 1] / den
    q_loop = np.stack([np.log(mesh.thick / 1000), np.arcsinh(1000 * gx) / 4, np.arcsinh(1000 * gy) / 4,
                       np.log(mesh.beta / 1000)])
    assert np.abs(q - q_loop).max() <= 1e-12 * np.abs(q_loop).max()
    nbr = {a: {a} for a in range(mesh.nv)}
    for t in mesh.tri:
        for a in t:
            nbr[int(a)] |= set(int(b) for b in t)
    cur = q_loop.copy()
    for it in range(40):
        cur = np.array([[np.mean([cur[k][b] for b in nbr[a]]) for a in range(mesh.nv)] for k in range(4)])
        if it == 7:
            assert np.abs(q8 - cur).max() <= 1e-12 * np.abs(cur).max()
    assert np.abs(q40 - cur).max() <= 1e-12 * np.abs(cur).max()
    X = ol.features(mesh)
    for k in range(4):  # hi + lo reproduce the FP32 value of q to ~2^-16 relative
        v32 = q[k].astype(np.float32).astype(np.float64)
        assert np.abs(X[:, 2 * k] + X[:, 2 * k + 1] - v32).max() <= 2.0 ** -16 * np.abs(v32).max()
        assert np.array_equal(X[:, 2 * k], omlp.bf16_round(q[k]))
    assert np.all(X[:, 15] == omlp.bf16_round(mesh.sigma[1]))
    assert np.array_equal(X[:, 12], omlp.bf16_round(q40[3]))


def test_profile_scales_recover_and_stationarity():
    rng = np.random.default_rng(1)
    n, lev = 50, 11
    S = rng.normal(size=(n, lev, 2)) * 30 + 5
    sb, sd = rng.uniform(0.2, 3, size=(n, 2)), rng.uniform(0.2, 3, size=(n, 2))
    b = S[:, :1, :]
    U = sb[:, None, :] * b + sd[:, None, :] * (S - b)
    y = ol.profile_scales(U, S, reg=0.0)
    assert np.abs(y[:, 0::2] - (sb - 1)).max() <= 1e-10 and np.abs(y[:, 1::2] - (sd - 1)).max() <= 1e-10
    # regularised: the gradient of the objective vanishes at the returned scales (within the clip)
    reg = 0.3
    U2 = U + rng.normal(size=U.shape) * 10
    y2 = ol.profile_scales(U2, S, reg=reg)
    for c in range(2):
        bb = np.repeat(S[:, :1, c], lev, axis=1)
        dd = S[:, :, c] - bb
        s1, s2 = 1 + y2[:, 2 * c], 1 + y2[:, 2 * c + 1]
        r = s1[:, None] * bb + s2[:, None] * dd - U2[:, :, c]
        g1 = (r * bb).sum(1) + reg ** 2 * (bb * bb).sum(1) * (s1 - 1)
        g2 = (r * dd).sum(1) + reg ** 2 * (dd * dd).sum(1) * (s2 - 1)
        inside = (np.abs(y2[:, 2 * c]) < 5) & (np.abs(y2[:, 2 * c + 1]) < 5)
        scale = (np.abs(U2[:, :, c]) * (np.abs(bb) + np.abs(dd))).sum(1)
        assert np.all(np.abs(g1[inside]) <= 1e-10 * scale[inside])
        assert np.all(np.abs(g2[inside]) <= 1e-10 * scale[inside])
    # a column without shallow-ice velocity keeps the scales at 1 (y = 0); large scales are clipped
    Z = np.zeros((2, lev, 2))
    assert np.all(ol.profile_scales(rng.normal(size=(2, lev, 2)), Z) == 0)
    big = ol.profile_scales(100 * S[:3], S[:3], reg=0.0)
    assert np.all(big == 5.0)


def test_exact_sum_rule_against_rational_sums():
    rng = np.random.default_rng(2)
    n_cert = 0
    for trial in range(200):
        k = int(rng.integers(2, 40))
        q = int(rng.integers(-30, 5))
        width = int(rng.integers(10, 30))
        t = rng.integers(-(2 ** width), 2 ** width, size=k).astype(np.float64) * 2.0 ** q
        exact = sum(Fraction(float(v)) for v in t)
        certified = bool(ol.fp32_exact_sum(t[None, :])[0])
        sums = []
        for _ in range(5):  # FP32 additions in random orders
            acc = np.float32(0)
            for v in rng.permutation(t):
                acc = np.float32(acc + np.float32(v))
            sums.append(Fraction(float(acc)))
        if certified:
            n_cert += 1
            assert all(s == exact for s in sums), (t, sums, exact)
    assert 20 <= n_cert <= 180   # both outcomes occur
    # hand cases
    assert ol.fp32_exact_sum(np.array([[0.5, 0.25, 2.0 ** -20]]))[0]
    assert not ol.fp32_exact_sum(np.array([[1.0, 2.0 ** -30]]))[0]


def test_dyadic_network_is_exact_in_rational_arithmetic():
    params, X, E = synth.dyadic_mlp_case(11, 128)
    ok, details = ol.exact_case_certified(params.astype(np.float64), X, E, 2.0 / 128)
    assert ok, details
    Y, _ = omlp.forward(params.astype(np.float64), X, bf16=True)
    P = omlp.unflatten(params.astype(np.float64))
    for row in range(3):  # the FP64 evaluation equals the rational one
        h = [Fraction(float(v)) for v in X[row]]
        for W, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
            z = [sum(Fraction(float(w)) * x for w, x in zip(P[W][o], h)) + Fraction(float(P[b][o]))
                 for o in range(P[W].shape[0])]
            # z is a short dyadic number: float() is exact, and so is the BF16 rounding of it
            h = [Fraction(float(omlp.bf16_round(np.array([float(max(v, 0))]))[0])) for v in z]
        y = [sum(Fraction(float(w)) * x for w, x in zip(P["W4"][o], h)) + Fraction(float(P["b4"][o]))
             for o in range(32)]
        assert all(Fraction(float(a)) == b for a, b in zip(Y[row], y))


def test_forward_certificate_flags_a_planted_rounding_tie():
    # first hidden unit: z = x0 + 2^-8.  Row 0 (x0 = 1): z = 1 + 2^-8, exactly halfway between the BF16
    # numbers 1 and 1 + 2^-7 -- any accumulation error decides the rounding.  Row 1 (x0 = 0.5):
    # z = 0.5 + 2^-8, itself a BF16 number (spacing 2^-8 in [0.5, 1)), half a spacing from a midpoint.
    P = omlp.unflatten(np.zeros(omlp.NPARAM))
    P["W1"][0, 0] = 1.0
    P["b1"][0] = 2.0 ** -8
    X = np.zeros((2, 16))
    X[0, 0], X[1, 0] = 1.0, 0.5
    ok, ybound = ol.forward_certificate(omlp.flatten(P), X)
    assert not ok[0] and ok[1]
    assert np.all(ybound[1] == 0)   # every output of row 1 is a sum of exact zeros

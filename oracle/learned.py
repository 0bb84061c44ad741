"""CPU oracle of the learned warm start around the network (TEST INFRASTRUCTURE ONLY).

The warm start is not in the paper: the network predicts a Newton initial guess (Sec. 3.1,
Eq. linearsystem starts from U^0) for the first-order Stokes solve.  This module states, in plain
FP64 numpy, every step of it that is not the network itself (the network is `oracle.mlp`):

  * `features`: the 16 per-column inputs -- local (H, grad s, beta) as BF16 hi/lo pairs, the same
    averaged over 8 and 40 sweeps of the closed-neighbourhood mean, and the layering sigma_1;
  * `decode`: the structured decoder that turns the network's 4 outputs per column into the 22
    level velocities, u_c(sigma_l) = (1 + y_2c) b_c + (1 + y_2c+1) (u_sia,c(sigma_l) - b_c), with
    b_c = u_sia,c at the bed, on the oracle's own shallow-ice guess;
  * `judge_keep`: the fallback rule -- keep the network's guess iff its FP64 measure (residual norm
    or energy) is finite and no larger than the shallow-ice guess's;
  * `learned_guess`: the whole pipeline in that order;
  * `profile_scales`: the decoder's training targets, the per-column least-squares scales of a
    solution, regularised toward 1;
  * `forward_certificate` / `exact_case_certified`: where FP32 accumulation order can change a
    BF16 rounding or an output, so that a comparison with the tensor-core kernels can tell apart
    what the arithmetic fixes uniquely from what it leaves to the order of the sums.

Only `tests/` import this module.  Parity status: `decode` and `judge_keep` are pinned by closed
forms (tests/test_oracle_learned.py: zero output reproduces the shallow-ice guess, scales -1 give
zero velocity, a hand-set column gives its closed form); `features` by a direct per-vertex loop on a
tiny mesh and by the hi/lo reconstruction; `profile_scales` by exact recovery of scales that were
used to build the target and by the normal equations of the regularised fit.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import mlp as omlp

NFEAT = 16
NOUT = 32
LEVELS = 11


def closed_neighbourhoods(tri: np.ndarray, nv: int):
    """Sorted closed neighbourhood (the vertex and every vertex sharing a triangle with it)."""
    nbr = [set([a]) for a in range(nv)]
    for t in tri:
        for a in t:
            nbr[int(a)].update(int(x) for x in t)
    return [np.array(sorted(n)) for n in nbr]


def nodal_surface_gradient(mesh):
    """Area-weighted mean of the P1 surface gradients of the triangles around each vertex, [2, nv]."""
    xy, tri = mesh.xy, mesh.tri
    s = mesh.bed + mesh.thick
    p = xy[tri]
    ax, ay = p[:, 1, 0] - p[:, 0, 0], p[:, 1, 1] - p[:, 0, 1]
    bx, by = p[:, 2, 0] - p[:, 0, 0], p[:, 2, 1] - p[:, 0, 1]
    det = ax * by - ay * bx
    d1, d2 = s[tri[:, 1]] - s[tri[:, 0]], s[tri[:, 2]] - s[tri[:, 0]]
    sx, sy = (d1 * by - d2 * ay) / det, (ax * d2 - bx * d1) / det
    area = 0.5 * det
    acc = np.zeros((3, mesh.nv))
    for a in range(3):
        np.add.at(acc[0], tri[:, a], area * sx)
        np.add.at(acc[1], tri[:, a], area * sy)
        np.add.at(acc[2], tri[:, a], area)
    return acc[0] / acc[2], acc[1] / acc[2]


def feature_quantities(mesh):
    """q = (ln(H / 1000 m), asinh(1000 s_x) / 4, asinh(1000 s_y) / 4, ln(beta / 1000)) per vertex [4, nv],
    and q after 8 and after 40 sweeps of the closed-neighbourhood mean."""
    gx, gy = nodal_surface_gradient(mesh)
    q = np.stack([np.log(mesh.thick / 1000.0), 0.25 * np.arcsinh(1000.0 * gx),
                  0.25 * np.arcsinh(1000.0 * gy), np.log(np.maximum(mesh.beta, 1e-30) / 1000.0)])
    nbr = closed_neighbourhoods(mesh.tri, mesh.nv)
    rows = np.concatenate([np.full(len(n), a) for a, n in enumerate(nbr)])
    cols = np.concatenate(nbr)
    vals = np.concatenate([np.full(len(n), 1.0 / len(n)) for n in nbr])
    S = sp.csr_matrix((vals, (rows, cols)), shape=(mesh.nv, mesh.nv))  # one sweep = S @ (each quantity)
    cur = q.T
    q8 = None
    for it in range(40):
        cur = S @ cur
        if it == 7:
            q8 = cur.T.copy()
    return q, q8, cur.T.copy()


def pack_features(q, q8, q40, sigma):
    """The 16 BF16 inputs per column (returned as float64 values of the BF16 numbers), [nv, 16]:
    hi / lo BF16 parts of the FP32 value of each local quantity, the 8-sweep means, the 40-sweep
    means of ln beta and of the two slopes, and sigma_1."""
    nv = q.shape[1]
    X = np.zeros((nv, NFEAT))
    for k in range(4):
        v = q[k].astype(np.float32)
        hi = omlp.bf16_round(v)
        lo = omlp.bf16_round((v - hi.astype(np.float32)).astype(np.float32))
        X[:, 2 * k], X[:, 2 * k + 1] = hi, lo
    for k in range(4):
        X[:, 8 + k] = omlp.bf16_round(q8[k])
    X[:, 12] = omlp.bf16_round(q40[3])
    X[:, 13] = omlp.bf16_round(q40[1])
    X[:, 14] = omlp.bf16_round(q40[2])
    X[:, 15] = omlp.bf16_round(np.full(nv, sigma[1]))
    return X


def features(mesh):
    q, q8, q40 = feature_quantities(mesh)
    return pack_features(q, q8, q40, mesh.sigma)


def feature_fp32_margin(mesh):
    """Distance of each FP64 feature quantity from the nearest FP32 rounding midpoint, relative to
    the largest magnitude of that quantity over the mesh ([nv, 16]; inf for the constant sigma_1).
    The quantities are sums (area-weighted gradients, neighbourhood means) whose FP64 rounding
    depends on the summation order by ~1e-16 of the largest term; where the margin is below
    ~1e-12 that order alone could move the FP32 (and so the BF16) value."""
    q, q8, q40 = feature_quantities(mesh)
    def margin(x):
        x = np.asarray(x, dtype=np.float64)
        f = x.astype(np.float32).astype(np.float64)
        ulp = np.abs(np.spacing(x.astype(np.float32))).astype(np.float64)
        mid_dist = np.abs(np.abs(x - f) - 0.5 * ulp)
        return mid_dist / max(np.abs(x).max(), 1e-300)
    out = np.full((q.shape[1], NFEAT), np.inf)
    for k in range(4):
        out[:, 2 * k] = out[:, 2 * k + 1] = margin(q[k])
        out[:, 8 + k] = margin(q8[k])
    out[:, 12], out[:, 13], out[:, 14] = margin(q40[3]), margin(q40[1]), margin(q40[2])
    return out


def decode(Y, Usia, nv, L):
    """Structured decoder: per column a and component c, with b = u_sia,c(bed) and the network's
    outputs y_b = Y[a, 2c], y_d = Y[a, 2c + 1]:  u_c(sigma_l) = (1 + y_b) b + (1 + y_d)(u_sia,c(sigma_l) - b).
    Y [nv, >= 4] (any float type), Usia [2 nv (L + 1)] in the dof order; returns U in the dof order."""
    Y = np.asarray(Y, dtype=np.float64)
    S = np.asarray(Usia, dtype=np.float64).reshape(nv, L + 1, 2)
    U = np.empty_like(S)
    for c in range(2):
        b = S[:, 0, c][:, None]
        yb, yd = Y[:, 2 * c][:, None], Y[:, 2 * c + 1][:, None]
        U[:, :, c] = (1.0 + yb) * b + (1.0 + yd) * (S[:, :, c] - b)
    return U.reshape(-1)


def judge_keep(f_net: float, f_sia: float) -> bool:
    """Keep the network's guess iff its FP64 measure is finite and no larger than the shallow-ice one."""
    return bool(np.isfinite(f_net) and f_net <= f_sia)


JUDGE_RESIDUAL, JUDGE_ENERGY, JUDGE_NONE = 0, 1, 2


def judge_measures(om, U, Usia, judge):
    """(f_net, f_sia) under the judge: the FP64 residual norm or the FP64 energy Pi_h."""
    if judge == JUDGE_RESIDUAL:
        return float(np.linalg.norm(om.residual(U))), float(np.linalg.norm(om.residual(Usia)))
    return om.energy(U), om.energy(Usia)


def learned_guess(om, params, judge, X=None):
    """The whole learned initial guess in the oracle's arithmetic: shallow-ice guess, features,
    network (BF16 operands, FP64 accumulation), decoder, judge.  Returns (U, used, Y, (f_net, f_sia))."""
    mesh = om.mesh
    Usia = om.sia()
    if X is None:
        X = features(mesh)
    Y, _ = omlp.forward(np.asarray(params, dtype=np.float64), X, bf16=True)
    U = decode(Y, Usia, mesh.nv, mesh.nlayers)
    if judge == JUDGE_NONE:
        return U, True, Y, (np.nan, np.nan)
    f = judge_measures(om, U, Usia, judge)
    keep = judge_keep(*f)
    return (U if keep else Usia.copy()), keep, Y, f


def profile_scales(Ucol, Scol, reg=0.1, clip=5.0):
    """Training targets of the decoder.  For each column [n, 11, 2] and component c, with the
    shallow-ice sliding part b (the bed value, at every level) and deformation part d(sigma) = S - b,
    the scales (s_b, s_d) minimise
        |s_b b + s_d d - u|^2 + reg^2 (|b|^2 (s_b - 1)^2 + |d|^2 (s_d - 1)^2),
    i.e. solve the 2 x 2 normal equations
        [(1 + reg^2) b.b, b.d; b.d, (1 + reg^2) d.d] (s_b, s_d) = (u.b + reg^2 b.b, u.d + reg^2 d.d);
    a numerically singular system (det <= 1e-30 a11 a22) gives s = 1.  Returns y = s - 1 clipped
    to [-clip, clip], [n, 4] = (y_b,u, y_d,u, y_b,v, y_d,v)."""
    Ucol = np.asarray(Ucol, dtype=np.float64)
    Scol = np.asarray(Scol, dtype=np.float64)
    out = np.empty((Ucol.shape[0], 4))
    r2 = reg * reg
    for c in range(2):
        u = Ucol[:, :, c]
        b = np.repeat(Scol[:, :1, c], u.shape[1], axis=1)
        d = Scol[:, :, c] - b
        bb, dd, bd = (b * b).sum(1), (d * d).sum(1), (b * d).sum(1)
        ub, ud = (u * b).sum(1), (u * d).sum(1)
        a11, a22, a12 = (1 + r2) * bb, (1 + r2) * dd, bd
        r1, rr2 = ub + r2 * bb, ud + r2 * dd
        det = a11 * a22 - a12 * a12
        ok = det > 1e-30 * (a11 * a22 + 1e-300)
        safe = np.where(ok, det, 1.0)
        sb = np.where(ok, (r1 * a22 - rr2 * a12) / safe, 1.0)
        sd = np.where(ok, (a11 * rr2 - a12 * r1) / safe, 1.0)
        out[:, 2 * c] = np.clip(sb - 1.0, -clip, clip)
        out[:, 2 * c + 1] = np.clip(sd - 1.0, -clip, clip)
    return out


# ---------------------------------------------------------------- FP32 accumulation-order analysis
U32 = 2.0 ** -24


def _gamma(k):
    """Bound on the relative error of a k-term FP32 sum in any order, doubled to cover accumulation
    that truncates instead of rounding (tensor-core adders): 2 k u / (1 - 2 k u)."""
    return 2 * k * U32 / (1 - 2 * k * U32)


def _bf16_midpoint_distance(x):
    """Distance of x (float64) from the nearest BF16 rounding midpoint (and from the ReLU kink at 0)."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    e = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
    step = 2.0 ** (e - 7)  # BF16 spacing in [2^e, 2^(e+1))
    r = ax / step
    dist = np.abs(r - np.floor(r) - 0.5) * step
    return np.minimum(np.where(ax > 0, dist, 0.0), ax)


ACC_ERR = 2.0 ** -20


def forward_certificate(params, X, acc_err=ACC_ERR):
    """For each row, whether the BF16 roundings of its hidden activations (and their ReLU signs) are
    fixed by the arithmetic for any FP32 accumulation whose error stays within the error model, and
    a bound on |Y_fp32 - Y| for the rows where they are.  Error model: |fl(z) - z| <= acc_err *
    (sum of |terms| + |bias|) + u |z|.  acc_err = None takes the worst case of a K-term sum in any
    order (2 K u); that certifies few rows of a random network at K = 128, so the default 2^-20 --
    16 units in the last place of the sum of magnitudes, several times what a 128-term FP32 sum
    shows in practice -- is an assumption, not a bound (the exact test networks, whose sums are
    exact in any order, cover the worst case).  Returns (certified [n] bool, ybound [n, 32])."""
    P = omlp.unflatten(np.asarray(params, dtype=np.float64))
    r = omlp.bf16_round
    h = r(X)
    ok = np.ones(X.shape[0], dtype=bool)
    rel = (lambda k: _gamma(k)) if acc_err is None else (lambda k: acc_err)
    for Wn, bn in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        W = r(P[Wn])
        z = h @ W.T + P[bn]
        # FP32 error: the accumulation over K terms plus the bias add and the rounding of the sum
        err = rel(W.shape[1] + 1) * (np.abs(h) @ np.abs(W).T + np.abs(P[bn])) + U32 * np.abs(z)
        # fixed whatever the order: an exactly known sum (no error), a value farther from every BF16
        # rounding midpoint than the error, or a value certainly negative (ReLU gives 0)
        ok &= np.all((err == 0) | (_bf16_midpoint_distance(z) > err) | (z < -err), axis=1)
        h = r(np.maximum(z, 0.0))
    W4 = r(P["W4"])
    y = h @ W4.T + P["b4"]
    ybound = rel(W4.shape[1] + 1) * (np.abs(h) @ np.abs(W4).T + np.abs(P["b4"])) + U32 * np.abs(y)
    return ok, ybound


# ---------------------------------------------------------------- exactly representable test networks
def fp32_exact_sum(terms, axis=-1):
    """True where a sum of these (float64, exactly known) terms is computed exactly in any order by
    any adder that keeps 24 significant bits below the largest term: every term is a multiple of
    2^q for a common q and the sum of magnitudes stays below 2^(q + 23)."""
    t = np.abs(np.asarray(terms, dtype=np.float64))
    nz = t > 0
    # exponent of the lowest set bit of each nonzero term
    m, e = np.frexp(np.where(nz, t, 1.0))
    mant = np.ldexp(m, 53).astype(np.int64)  # exact: t = mant * 2^(e - 53)
    lsb = mant & (-mant)                     # lowest set bit of the significand
    tz = np.frexp(lsb.astype(np.float64))[1] - 1
    low = np.where(nz, e - 53 + tz, 10 ** 6)
    q = low.min(axis=axis)
    s = t.sum(axis=axis)
    return (s == 0) | (s < np.ldexp(1.0, np.minimum(q, 900) + 23))


def exact_case_certified(params, X, E, n_scale):
    """Checks that every FP32 sum the forward and backward kernels form on this input is exact in any
    order (so both sides must agree bit for bit): the hidden pre-activations, the outputs, the bias
    gradients (sums over rows), dW (sums over rows) and dH (sums over outputs).  E = Y - T, the
    output error, and n_scale = 2 / n.  Returns (ok, details)."""
    P = omlp.unflatten(np.asarray(params, dtype=np.float64))
    r = omlp.bf16_round
    x = r(X)
    Ws = [r(P["W1"]), r(P["W2"]), r(P["W3"]), r(P["W4"])]
    bs = [P["b1"], P["b2"], P["b3"], P["b4"]]
    acts = [x]
    details = {}
    ok = True
    h = x
    for k in range(4):
        terms = h[:, None, :] * Ws[k][None, :, :]
        terms = np.concatenate([terms, np.broadcast_to(bs[k][None, :, None], terms.shape[:2] + (1,))], axis=2)
        good = fp32_exact_sum(terms)
        details[f"z{k + 1}"] = bool(good.all())
        ok &= bool(good.all())
        z = h @ Ws[k].T + bs[k]
        if k < 3:
            h = r(np.maximum(z, 0.0))
            acts.append(h)
    # backward: dY = n_scale * E on the used outputs
    dy = np.zeros_like(np.asarray(E, dtype=np.float64))
    dy[:, :omlp.OUT_USED] = n_scale * np.asarray(E, dtype=np.float64)[:, :omlp.OUT_USED]
    dz = dy
    for k in range(3, -1, -1):
        dzb = r(dz)
        hin = acts[k]
        good_b = fp32_exact_sum(dz.T)                                   # bias gradient: sum over rows
        good_w = fp32_exact_sum(dzb.T[:, None, :] * hin.T[None, :, :])  # dW[o, i] = sum_rows dz[:, o] h[:, i]
        details[f"db{k + 1}"], details[f"dW{k + 1}"] = bool(good_b.all()), bool(good_w.all())
        ok &= bool(good_b.all()) and bool(good_w.all())
        if k > 0:
            terms = dzb[:, None, :] * Ws[k].T[None, :, :]               # dH[:, i] = sum_o dz[:, o] W[o, i]
            good_h = fp32_exact_sum(terms)
            details[f"dH{k}"] = bool(good_h.all())
            ok &= bool(good_h.all())
            dh = dzb @ Ws[k]
            dz = dh * (acts[k] > 0)
    return ok, details

"""Learned Newton warm start: training data from the solver, training on the tensor cores, evaluation.

The network (bp_mlp_*) maps per-column features (H, grad s, beta, the sigma levels) to the 22
level velocities of a 10-layer column through a structured decoder: it scales the sliding and
deformation parts of the shallow-ice profile per column and component (vertically consistent).  Training data are Newton solutions of the
1,003,520-wedge dome geometry (224 x 224 grid, 10 layers, sinusoidal bed) with different seeded
correlated beta fields, solved by the mixed-precision path (FP32 Jacobian lanes and Krylov,
FP64 residual) to ||F|| <= 1e-8 ||F(0)||.  Every step -- solving, features, forward, backward,
Adam -- runs in libbp's kernels; torch only holds device memory.

    python -m paper_2204_04321_b300.learned train --solutions 2000 --out paper_2204_04321_b300/weights/...
    python -m paper_2204_04321_b300.learned eval --weights ... --seeds 50
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import capi, synth

TRAIN_SEED0 = 10000   # beta seeds of the training / validation solutions
TEST_SEED0 = 90000    # unseen beta seeds of the evaluation
FIT_REG = 0.1         # Tikhonov weight of the per-column profile fit toward the shallow-ice scales
                      # (the fit itself is bp_learned_targets)
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "warmstart_dome224_l10.npy")


def geometry(m: int = 224):
    """The dome geometry of the 1M-wedge workload (beta replaced per solution)."""
    return synth.dome_mesh(m, 10, 201, 202, bed="sinusoidal", beta="field", name=f"dome-{m}-x10")


JUDGES = {"learned": capi.BP_JUDGE_RESIDUAL, "learned_energy": capi.BP_JUDGE_ENERGY,
          "learned_raw": capi.BP_JUDGE_NONE, "learned_picard": capi.BP_JUDGE_ENERGY}
# "learned_picard": the energy-judged network guess followed by Picard (fixed-viscosity) steps until
# the relative residual falls below PICARD_RTOL, then Newton.  The network's guess is close in the
# energy norm (~0.4 of the shallow-ice error) but rough; Newton steps from it overshoot, while Picard
# steps, which do not, take it into Newton's basin.
PICARD_RTOL = 0.1


def solve(dm, precision=capi.BP_F32, guess="sia", mlp=None, max_krylov=4000, **opts):
    """Newton solve from the named initial guess ("zero", "sia", or a learned guess: "learned" judged
    by the FP64 residual, "learned_energy" judged by the FP64 energy, "learned_raw" unjudged,
    "learned_picard" energy-judged and followed by Picard steps).  The wall time covers the guess
    and the solve; rep["guess_rel_err"] is |U0 - U*| / |U*|.  opts: further bp_solve_opts fields."""
    import torch
    U = torch.empty(dm.ndof, dtype=torch.float64, device=dm.device)
    used = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if guess in JUDGES:
        used = capi.bp_initial_guess_learned(dm.handle, mlp, U, judge=JUDGES[guess])
    else:
        capi.bp_initial_guess(dm.handle, capi.BP_GUESS_SIA if guess == "sia" else capi.BP_GUESS_ZERO, U)
    torch.cuda.synchronize()
    t_guess = time.perf_counter() - t0
    U0 = U.clone()  # (not timed)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    kw = dict(opts)
    if guess == "learned_picard":
        kw["picard_rtol"] = PICARD_RTOL
    rc, rep = capi.bp_newton_solve(dm.handle, U, precision=precision, max_krylov=max_krylov, **kw)
    torch.cuda.synchronize()
    rep["wall_s"] = t_guess + (time.perf_counter() - t1)
    rep["status"] = rc
    rep["learned_used"] = used
    rep["guess_rel_err"] = float((U0 - U).norm() / U.norm())
    return U, rep


def generate(mesh, seeds, cols_per_solution=4096, precision=capi.BP_F32, log=None):
    """Solutions for each beta seed; returns X [n, 16] bfloat16 and T [n, 32] float32 (CUDA)."""
    import torch
    dm = capi.DeviceMesh(mesh)
    nv = mesh.nv
    Xall = torch.empty(nv, 16, dtype=torch.bfloat16, device=dm.device)
    Tall = torch.empty(nv, 32, dtype=torch.float32, device=dm.device)
    Xs, Ts, stats = [], [], []
    for i, seed in enumerate(seeds):
        beta = synth.lognormal_beta_field_torch(mesh.xy, seed, dm.device)
        capi.bp_mesh_set_beta(dm.handle, beta)
        U, rep = solve(dm, precision)
        if not rep["converged"]:
            raise RuntimeError(f"solution for beta seed {seed} did not converge: {rep['history'][-1]}")
        capi.bp_mlp_features(dm.handle, Xall)
        cols = torch.as_tensor(np.random.default_rng(seed).choice(nv, min(cols_per_solution, nv), replace=False),
                               device=dm.device)
        capi.bp_learned_targets(dm.handle, U, FIT_REG, Tall)   # per-column profile scales (kernel)
        Xs.append(Xall[cols].clone())
        Ts.append(Tall[cols].clone())
        stats.append({"seed": seed, "newton_iters": rep["newton_iters"], "krylov_iters": rep["krylov_iters"],
                      "s": rep["wall_s"]})
        if log and (i % 100 == 0 or i == len(seeds) - 1):
            log(f"solution {i + 1}/{len(seeds)} seed {seed}: {rep['newton_iters']} Newton, {rep['wall_s']:.3f} s")
    dm.close()
    return torch.cat(Xs), torch.cat(Ts), stats


def train(net, X, T, steps=20000, batch=8192, lr0=2e-3, lr1=2e-5, val=None, log=None, seed=0):
    """Adam with a cosine learning-rate schedule on random mini-batches."""
    import math
    import torch
    n = X.shape[0]
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    hist = []
    t0 = time.perf_counter()
    for step in range(steps):
        lr = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * step / max(1, steps - 1)))
        idx = torch.randint(0, n, (batch,), device=X.device, generator=g)
        net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr)
        if step % 1000 == 0 or step == steps - 1:
            tl, _ = net.gradient(X[idx].contiguous(), T[idx].contiguous())
            vl = None
            if val is not None:
                vl, _ = net.gradient(val[0][:65536].contiguous(), val[1][:65536].contiguous())
            hist.append({"step": step, "lr": lr, "train_loss": tl, "val_loss": vl,
                         "s": time.perf_counter() - t0})
            if log:
                log(f"step {step}: lr {lr:.2e} train {tl:.3e} val {vl}")
    torch.cuda.synchronize()
    return hist


def evaluate(net, mesh, seeds, precision=capi.BP_F32, guesses=("zero", "sia", "learned")):
    dm = capi.DeviceMesh(mesh)
    out = []
    for seed in seeds:
        beta = synth.lognormal_beta_field_torch(mesh.xy, seed, dm.device)
        capi.bp_mesh_set_beta(dm.handle, beta)
        row = {"seed": seed}
        for gname in guesses:
            _, rep = solve(dm, precision, gname, mlp=net)
            row[gname] = {"newton_iters": rep["newton_iters"], "krylov_iters": rep["krylov_iters"],
                          "s": rep["wall_s"], "converged": rep["converged"], "guess_rel_err": rep["guess_rel_err"],
                          "initial_rel_residual": rep["history"][0], "learned_used": rep["learned_used"]}
        out.append(row)
    dm.close()
    return out


def summarize(rows, guesses=("zero", "sia", "learned")):
    s = {}
    for gname in guesses:
        its = np.array([r[gname]["newton_iters"] for r in rows])
        ts = np.array([r[gname]["s"] for r in rows])
        f0 = np.array([r[gname]["initial_rel_residual"] for r in rows])
        e0 = np.array([r[gname].get("guess_rel_err", np.nan) for r in rows])
        s[gname] = {"newton_iters_mean": float(its.mean()), "s_mean": float(ts.mean()),
                    "initial_rel_residual_median": float(np.median(f0)),
                    "guess_rel_err_median": float(np.median(e0)),
                    "all_converged": bool(all(r[gname]["converged"] for r in rows))}
    for gname in guesses:
        if gname.startswith("learned") and "sia" in s:
            # ratio with a 99% interval from the mean of log time ratios (paired), as the paper reports speedups
            from scipy import stats
            lr = np.log(np.array([r["sia"]["s"] / r[gname]["s"] for r in rows]))
            half = (stats.t.ppf(0.995, len(lr) - 1) * lr.std(ddof=1) / np.sqrt(len(lr))
                    if len(lr) > 1 else float("nan"))
            s[f"speedup_{gname}_vs_sia"] = {"mean": float(np.exp(lr.mean())),
                                            "ci99": [float(np.exp(lr.mean() - half)), float(np.exp(lr.mean() + half))]}
    return s


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--solutions", type=int, default=2000)
    t.add_argument("--val-fraction", type=float, default=0.1)
    t.add_argument("--cols", type=int, default=4096)
    t.add_argument("--steps", type=int, default=20000)
    t.add_argument("--batch", type=int, default=8192)
    t.add_argument("--out", default=DEFAULT_WEIGHTS)
    t.add_argument("--eval-seeds", type=int, default=50)
    e = sub.add_parser("eval")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--seeds", type=int, default=50)
    args = ap.parse_args(argv)
    log = lambda msg: print(msg, flush=True)
    mesh = geometry()
    if args.cmd == "train":
        t0 = time.perf_counter()
        seeds = [TRAIN_SEED0 + k for k in range(args.solutions)]
        X, T, stats = generate(mesh, seeds, args.cols, log=log)
        t_gen = time.perf_counter() - t0
        nval = max(1, int(round(args.val_fraction * args.solutions))) * args.cols
        Xtr, Ttr, Xv, Tv = X[:-nval], T[:-nval], X[-nval:], T[-nval:]
        net = capi.Mlp(seed=7)
        hist = train(net, Xtr, Ttr, steps=args.steps, batch=args.batch, val=(Xv, Tv), log=log)
        net.save(args.out)
        rows = evaluate(net, mesh, [TEST_SEED0 + k for k in range(args.eval_seeds)])
        meta = {"solutions": args.solutions, "train_rows": int(Xtr.shape[0]), "val_rows": int(Xv.shape[0]),
                "cols_per_solution": args.cols, "steps": args.steps, "batch": args.batch,
                "data_generation_s": t_gen, "solution_newton_iters_mean": float(np.mean([s["newton_iters"] for s in stats])),
                "history": hist, "eval": summarize(rows), "train_seeds": [seeds[0], seeds[-1]]}
        with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
            json.dump(meta, f, indent=1)
        log(json.dumps(meta["eval"]))
    else:
        net = capi.Mlp()
        net.load(args.weights)
        g = ("zero", "sia", "learned", "learned_energy", "learned_raw", "learned_picard")
        rows = evaluate(net, mesh, [TEST_SEED0 + k for k in range(args.seeds)], guesses=g)
        print(json.dumps(summarize(rows, g), indent=1))
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()

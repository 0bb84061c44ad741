"""Plain damped Newton for the discrete first-order Stokes system (TEST INFRASTRUCTURE ONLY).

Paper Sec. 3.1, Eq. linearsystem: J(U^k) delta = -F(U^k), U^{k+1} = U^k + alpha_k delta.
The paper leaves the damping rule open.  Reading used here (and by the CUDA solver):
alpha in {1, 1/2, 1/4, ..., 2^-10}, the first that satisfies the Armijo condition on the
discrete energy Pi_h (whose gradient is the residual):
    Pi_h(U + alpha delta) <= Pi_h(U) + 1e-4 * alpha * F(U) . delta.
Convergence: ||F(U^k)||_2 <= rtol * ||F(0)||_2 (the reference norm is the residual at
U = 0, i.e. the driving-stress load, independent of the initial guess).
The linear solve is a sparse direct factorisation (a library primitive); the oracle
therefore only handles meshes small enough for that.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def newton(om, U0: np.ndarray, rtol: float = 1e-8, maxit: int = 60, armijo: float = 1e-4,
           max_halvings: int = 10):
    U = np.array(U0, dtype=np.float64, copy=True)
    fref = np.linalg.norm(om.residual(np.zeros_like(U)))
    history = []
    for k in range(maxit + 1):
        J, R = om.jacobian_scipy(U)
        rn = np.linalg.norm(R)
        history.append(rn / fref)
        if rn <= rtol * fref:
            return U, {"iterations": k, "history": history, "converged": True}
        if k == maxit:
            break
        delta = spla.spsolve(J.tocsc(), -R)
        E0 = om.energy(U)
        slope = float(R @ delta)
        alpha = 1.0
        for _ in range(max_halvings + 1):
            if om.energy(U + alpha * delta) <= E0 + armijo * alpha * slope:
                break
            alpha *= 0.5
        U = U + alpha * delta
    return U, {"iterations": maxit, "history": history, "converged": False}

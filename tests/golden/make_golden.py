"""Writes dome_small_oracle.txt: stored oracle values on the small dome, from oracle/ alone.

The fixture pins the oracle against silent changes of its arithmetic (a later change must rewrite
the file, in a commit that names the passage of the paper that justifies it), and gives the GPU
tests expected values that need no oracle run.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2204_04321_b300 import synth  # noqa: E402  (seeded input generators only)

OUT = os.path.join(HERE, "dome_small_oracle.txt")
VEL_SEED = 103      # velocities uniform in [-100, 100] m/yr
SAMPLE_SEED = 7     # which rows and entries are stored
NSAMPLE = 200


def cases():
    """The mesh, velocities and the sampled rows / entries the fixture stores."""
    mesh = synth.config_small()
    U = synth.random_velocity(mesh, VEL_SEED)
    return mesh, U


def main():
    mesh, U = cases()
    om = oracle.OracleMesh(mesh)
    rowptr, colidx, vals, R = om.jacobian(U)
    E = om.energy(U)
    rng = np.random.default_rng(SAMPLE_SEED)
    rows = np.sort(rng.choice(om.ndof, NSAMPLE, replace=False))
    ents = np.sort(rng.choice(colidx.shape[0], NSAMPLE, replace=False))
    erow = np.searchsorted(rowptr, ents, side="right") - 1
    with open(OUT, "w") as f:
        f.write("# Oracle values on the 10,240-wedge dome (32 x 32 jittered grid, 2,048 triangles, 5 layers,\n"
                "# flat bed; mesh seed 101, beta seed 102; velocities seed 103, uniform in [-100, 100] m/yr):\n"
                "# the weak-form residual of the first-order Stokes equations (Sec. 2; Sec. 3.1, Eq. residual,\n"
                "# with the viscosity of Eq. effvisc), its Jacobian (the Newton matrix of Eq. linearsystem, on\n"
                "# the extruded CSR pattern) and the discrete energy whose gradient is the residual.\n"
                "# Written by tests/golden/make_golden.py from oracle/ alone.\n"
                "# Lines: 'R row value', 'J row col value', and the scalars below; values as repr().\n")
        f.write(f"ndof {om.ndof}\n")
        f.write(f"nnz {colidx.shape[0]}\n")
        f.write(f"norm2_R {float(np.linalg.norm(R))!r}\n")
        f.write(f"max_abs_R {float(np.abs(R).max())!r}\n")
        f.write(f"max_abs_J {float(np.abs(vals).max())!r}\n")
        f.write(f"energy {float(E)!r}\n")
        for i in rows:
            f.write(f"R {int(i)} {float(R[i])!r}\n")
        for k, i in zip(ents, erow):
            f.write(f"J {int(i)} {int(colidx[k])} {float(vals[k])!r}\n")
    print(OUT)


def load(path=OUT):
    """The stored values: scalars (dict), residual rows, Jacobian entries (row, col, value)."""
    scal, rows, ents = {}, [], []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            if p[0] == "R":
                rows.append((int(p[1]), float(p[2])))
            elif p[0] == "J":
                ents.append((int(p[1]), int(p[2]), float(p[3])))
            else:
                scal[p[0]] = float(p[1])
    return scal, rows, ents


if __name__ == "__main__":
    main()

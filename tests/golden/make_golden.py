"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

    python tests/golden/make_golden.py laplace400      # seconds
    python tests/golden/make_golden.py convdiff64x48   # ~15-25 minutes on 8 cores

Each output file says which oracle function and which seeded workload made it.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import exact, factorized as fz  # noqa: E402


def write(name, header, rows):
    with open(os.path.join(HERE, name), "w") as f:
        for h in header:
            f.write(f"# {h}\n")
        for r in rows:
            f.write(" ".join(repr(float(x)) if isinstance(x, float) else str(x) for x in r) + "\n")


def laplace400():
    p = wl.cfg_laplace_cg(N=20, s=1)
    r = fz.factorized_cg(p.A.to_scipy(), p.B.to_scipy(), p.C1, p.C2, 1e-8, 200)
    X = exact.laplacian_exact(20, p.C1 @ p.C2.T)
    write("laplace400_s1_cg_history.txt",
          ["oracle.factorized.factorized_cg on workloads.cfg_laplace_cg(N=20, s=1): 5-point Laplacian 20x20,",
           "A = B, C1, C2 ~ N(0,1) seed 0, tol 1e-8, maxit 200.  Columns: k, ||R^_k||/||R^_0||.",
           f"status {r.status}, iterations {r.iters}.",
           f"closed-form solution (oracle.exact.laplacian_exact): ||X*||_F = {float(np.linalg.norm(X))!r}"],
          [(k, h) for k, h in enumerate(r.history)])


def convdiff64x48():
    p = wl.cfg_convdiff_bicgstab(64, 48, 4)
    t0 = time.time()
    r = fz.factorized_bicgstab(p.A.to_scipy(), p.B.to_scipy(), p.C1, p.C2, 1e-8, 300)
    write("convdiff64x48_s4_bicgstab_history.txt",
          ["oracle.factorized.factorized_bicgstab on workloads.cfg_convdiff_bicgstab(64, 48, s=4):",
           "A = 3D upwind convection-diffusion 64^3 (wind seed 1), B = 48^3 (wind seed 2), C1, C2 ~ N(0,1) seed 0,",
           "tol 1e-8, maxit 300.  Columns: k, ||R^_k||/||R^_0||.",
           f"status {r.status}, iterations {r.iters}, oracle wall time {time.time() - t0:.0f} s."],
          [(k, h) for k, h in enumerate(r.history)])


if __name__ == "__main__":
    for name in sys.argv[1:] or ["laplace400"]:
        globals()[name]()

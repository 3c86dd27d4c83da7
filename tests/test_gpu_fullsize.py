"""Full-size check of the benchmarked workload, in the launch configuration
bench.py times: factorized BiCGSTAB in FP64 on the 64^3 / 48^3 convection-
diffusion operators, s = 4, tol 1e-8 (n = 262,144, m = 110,592).

The full oracle run takes ~16 minutes, so its residual history is stored
(tests/golden/convdiff64x48_s4_bicgstab_history.txt, written by
tests/golden/make_golden.py from oracle/ only) and compared iteration by
iteration while rounding has not yet separated the two; the rest is checked
through properties that hold at any size: sampled orthonormality of V, the
Arnoldi relation A V_k = V_{k+1} H_{k+1,k} on sampled rows, and the certified
bound on the FP64 true residual (the solve's recurrence test runs at 0.4 tol, the
default sylv_options.stop_margin, so it takes a few more iterations than the
oracle's run at tol).
"""
import os

import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "convdiff64x48_s4_bicgstab_history.txt")


def golden_history():
    return np.array([float(ln.split()[1]) for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")])


def test_convdiff64x48_bicgstab_fp64_full_size():
    p = wl.cfg_convdiff_bicgstab(64, 48, 4)
    g = golden_history()
    with ps.Solver(p.A, p.B, p.C1, p.C2) as sv:
        info = sv.bicgstab(1e-8, 300)
        hist = sv.history()
        V, Xh, W = sv.factors()
        H = sv.hessenberg(0)
    assert info["status"] == ps.SYLV_OK, info
    oracle_iters = len(g) - 1
    assert abs(info["iters"] - oracle_iters) <= max(3, oracle_iters // 10), (info["iters"], oracle_iters)
    np.testing.assert_allclose(hist[:21], g[:21], rtol=1e-6)
    assert info["true_rel_res"] <= info["true_rel_bound"] <= 1e-8, info
    rng = np.random.default_rng(0)
    w = V.shape[1]
    cols = rng.choice(w, 96, replace=False)
    G = V[:, cols].T @ V[:, cols]
    assert np.abs(G - np.eye(len(cols))).max() < 1e-12
    rows = rng.choice(p.A.nrows, 256, replace=False)
    A = p.A.to_scipy()
    lhs = A[rows] @ V[:, : w - 4]
    rhs = V[rows, :w] @ H[:w, : w - 4]
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max() * 10

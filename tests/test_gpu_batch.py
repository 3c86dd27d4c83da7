"""Batched factorized CG for many Lyapunov equations (one launch per phase for
all instances, CUDA-graph iterations) against the CPU oracle and against the
single-instance path.  Instances have uneven sizes (ragged tails) and block
widths s in {1, 2, 3, 4, 8}."""
import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl
from oracle import factorized as fz, residual

pytestmark = pytest.mark.gpu
STOP_MARGIN = 0.4  # default sylv_options.stop_margin


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def instances(count=9, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.integers(9, 41))
        s = int(rng.choice([1, 2, 3, 4, 8]))
        sigma = float(rng.random())
        A = wl.laplacian_2d(N, sigma)
        C = rng.standard_normal((N * N, s))
        out.append((A, C))
    return out


def test_batched_lyapunov_cg_matches_oracle_and_single():
    inst = instances()
    with ps.BatchSolver([a for a, _ in inst], [c for _, c in inst]) as bs:
        info = bs.cg(1e-10, 500)
        assert info["status"] == ps.SYLV_OK, info
        for i, (A, C) in enumerate(inst):
            V, Xh, W = bs.factors(i)
            hist = bs.history(i)
            # certified instances run the recurrence test at STOP_MARGIN * tol
            ref = fz.factorized_cg(A.to_scipy(), None, C, None, 1e-10 * STOP_MARGIN, 500, lyapunov=True)
            assert ref.status == "converged"
            assert len(hist) - 1 == ref.iters, (i, len(hist) - 1, ref.iters)
            X = V @ Xh @ V.T
            assert rel(X, ref.X()) < 1e-10, (i, rel(X, ref.X()))
            assert np.array_equal(V, W)
            np.testing.assert_allclose(hist[:10], ref.history[:10], rtol=1e-8)
            with ps.Solver(A, None, C, None, lyapunov=True) as sv:
                sv.cg(1e-10, 500)
                V1, X1, _ = sv.factors()
            assert rel(X, V1 @ X1 @ V1.T) < 1e-11
        assert info["iters"] == max(len(bs.history(i)) - 1 for i in range(len(inst)))
        assert 0 < info["true_rel_res"] <= info["true_rel_bound"] <= 1e-10, info
        for i, (A, C) in enumerate(inst):  # the oracle's direct true residual of every instance
            V, Xh, _ = bs.factors(i)
            As = A.to_scipy()
            assert residual.direct(As, As.T, C, C, V, Xh, V) <= 1e-10 * np.linalg.norm(C @ C.T), i


def test_batched_two_solves_and_maxit():
    inst = instances(count=4, seed=3)
    with ps.BatchSolver([a for a, _ in inst], [c for _, c in inst]) as bs:
        info = bs.cg(1e-8, 3)
        assert info["status"] == ps.SYLV_ENOTCONV and info["iters"] == 3
        for i, (A, C) in enumerate(inst):
            V, Xh, _ = bs.factors(i)
            ref = fz.factorized_cg(A.to_scipy(), None, C, None, 0.0, 3, lyapunov=True)
            assert rel(V @ Xh @ V.T, ref.X()) < 1e-10
        info = bs.cg(1e-8, 500)
        assert info["status"] == ps.SYLV_OK

"""Parity with the CPU oracle at the orders and widths the full-size solves run at.

- Factorized BiCGSTAB in FP64 with s = 8 for 70 iterations (small_gemm and basis_gemm on auto):
  the Arnoldi bases at 141 blocks (1,128 columns; the tensor-core Gram products over 9 column
  tiles, each split over several fold periods) against the oracle's block Arnoldi, and the small
  Sylvester operator of eq. 3.7 at order r = 1,120 (tensor cores, automatic from 448 on) on the
  solve's own H and G against the product formed in float64.  The BiCGSTAB iterates themselves
  are not compared at this width: rounding differences grow by ~1e10 within 30 iterations at
  s = 8 (two oracle runs whose C1 differs by 1e-15 separate by ~10% in the residual history by
  iteration 40), whereas the Arnoldi process stays at ~1e-15.
- Batched Lyapunov CG with instances of N = 128 and 160 (n = 16,384 and 25,600 rows), several
  row chunks per instance at the autotuner's choice.

X = V X^ W^T is compared without forming it (it would take gigabytes): with Householder QR
[V_g, V_o] = Q_L R_L and [W_g, W_o] = Q_R R_R,
    ||X_g - X_o||_F = ||R_L diag(X^_g, -X^_o) R_R^T||_F,
which keeps the cancellation inside a small dense product (a difference of Gram-based
squared norms would resolve only about 1e-8 relative).
"""
import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl
from oracle import factorized as fz

TOL_X = 1e-10
STOP_MARGIN = 0.4  # default sylv_options.stop_margin: the recurrence test of a certified FP64 solve


def factored_rel_diff(Vg, Xg, Wg, Vo, Xo, Wo):
    """||V_g X_g W_g^T - V_o X_o W_o^T||_F / ||V_o X_o W_o^T||_F through the QR of the stacked factors."""
    _, RL = np.linalg.qr(np.hstack([Vg, Vo]))
    _, RR = np.linalg.qr(np.hstack([Wg, Wo]))
    rg, ro = Xg.shape[0], Xo.shape[0]
    D = np.zeros((rg + ro, rg + ro))
    D[:rg, :rg] = Xg
    D[rg:, rg:] = -Xo
    _, RLo = np.linalg.qr(Vo)
    _, RRo = np.linalg.qr(Wo)
    return float(np.linalg.norm(RL @ D @ RR.T) / np.linalg.norm(RLo @ Xo @ RRo.T))


def test_factored_rel_diff_equals_the_formed_difference():
    # the comparison itself, on factors small enough to form X: random factors, and factors
    # whose difference is tiny (the case the comparison is for)
    rng = np.random.default_rng(0)
    n, m, r = 300, 200, 24
    Vo, Wo = rng.standard_normal((n, r)), rng.standard_normal((m, r))
    Xo = rng.standard_normal((r, r))
    for scale in (1.0, 1e-9, 1e-13):
        Vg = Vo + scale * rng.standard_normal((n, r))
        Xg = Xo + scale * rng.standard_normal((r, r))
        # unequal widths are allowed: the first factors carry two more (zero) columns
        Vg2 = np.hstack([Vg, np.zeros((n, 2))])
        Wg2 = np.hstack([Wo, np.zeros((m, 2))])
        Xg2 = np.zeros((r + 2, r + 2))
        Xg2[:r, :r] = Xg
        ref = np.linalg.norm(Vg @ Xg @ Wo.T - Vo @ Xo @ Wo.T) / np.linalg.norm(Vo @ Xo @ Wo.T)
        got = factored_rel_diff(Vg2, Xg2, Wg2, Vo, Xo, Wo)
        assert abs(got - ref) <= 1e-6 * ref + 1e-15, (scale, got, ref)


@pytest.fixture(scope="module")
def wide_bicgstab():
    """70 fixed iterations of FP64 BiCGSTAB with s = 8 on the convection-diffusion operators of
    30^3 and 20^3 unknowns: bases of 141 blocks (1,128 columns), factors of width 1,120."""
    A, B = wl.convdiff_3d(30, 1), wl.convdiff_3d(20, 2)
    s, iters = 8, 70
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 0)
    with ps.Solver(A, B, C1, C2) as sv:  # small_gemm, basis_gemm: auto
        info = sv.bicgstab(0.0, iters)
        V, Xh, W = sv.factors()
        H, G = sv.hessenberg(0), sv.hessenberg(1)
        rng = np.random.default_rng(3)
        Z = rng.standard_normal((1120, 1120)) * np.exp(rng.uniform(-3, 3, (1120, 1)))  # rows of mixed scale
        Q = sv.small_operator(Z)
    return dict(A=A, B=B, C1=C1, C2=C2, s=s, iters=iters, info=info, V=V, W=W, H=H, G=G, Z=Z, Q=Q)


@pytest.mark.gpu
def test_wide_arnoldi_bases_match_oracle(wide_bicgstab):
    # The block Arnoldi bases of both sides at 141 blocks: the tensor-core Gram products over
    # 9 column tiles, each split over 16 row ranges of 6-7 fold periods (n = 27,000), and the
    # block updates, against the oracle's BCGS2 block Arnoldi.  Unlike the BiCGSTAB iterates --
    # two oracle runs whose C1 differs by 1e-15 separate by ~10% in the residual history by
    # iteration 40 at s = 8 -- the Arnoldi process is stable: the same perturbation moves H by
    # ~1e-15 and V by ~1e-14 after 141 blocks.
    d = wide_bicgstab
    info, s = d["info"], d["s"]
    assert info["status"] == ps.SYLV_ENOTCONV and info["iters"] == d["iters"], info
    assert info["width"] == 2 * d["iters"] * s == 1120
    for side, (Op, C, Vg, Hg) in enumerate(((d["A"], d["C1"], d["V"], d["H"]), (d["B"], d["C2"], d["W"], d["G"]))):
        basis = fz.BlockKrylovBasis(Op.to_scipy() if side == 0 else Op.to_scipy().T.tocsr(), C, "arnoldi")
        nb = Hg.shape[1] // s + 1
        assert nb == 2 * d["iters"] + 1 == 141
        for _ in range(nb - 1):
            basis.step()
        Ho = basis.Hk(nb, nb - 1)
        Vo = basis.V(Vg.shape[1] // s)
        # CholQR2 here, Householder QR in the oracle, and different summation orders: after 140
        # steps the bases differ by ~1e-12 (measured); a wrong tile, split or fold would show as
        # 1e-6 or more
        assert np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho) < 1e-12, side
        assert np.linalg.norm(Vg - Vo) / np.linalg.norm(Vo) < 1e-11, side
        assert np.abs(Vg.T @ Vg - np.eye(Vg.shape[1])).max() < 1e-12, side


@pytest.mark.gpu
def test_small_operator_at_order_1120_matches_brute_force(wide_bicgstab):
    # eq. 3.7 at r = 1,120 on the solve's own H and G, through the library's path (the Ozaki
    # tensor-core product at this order: 9 periods of 128 values of k), against the product
    # formed here in float64
    d = wide_bicgstab
    H, G, Z, Q = d["H"], d["G"], d["Z"], d["Q"]
    r = Z.shape[0]
    ref = fz.small_sylvester(H[: r + d["s"], :r], Z, G[: r + d["s"], :r])
    # float64-accurate: normwise below 1e-14; componentwise (relative to the sum of |terms|) below
    # 1e-12 -- the Ozaki split rounds each operand to ~55 bits of its row's or column's largest
    # entry, so an entry whose terms cancel heavily and are much smaller than those maxima (rows
    # of Z here span e^-3 .. e^3) carries more relative error than a float64 GEMM's 2^-53 per term
    rp = r + d["s"]
    scale = np.zeros((rp, rp))
    scale[:, :r] += np.abs(H[:rp, :r]) @ np.abs(Z)
    scale[:r, :] += np.abs(Z) @ np.abs(G[:rp, :r]).T
    err = np.abs(Q - ref) / np.maximum(scale, 1e-300)
    assert err.max() < 1e-12, err.max()
    assert np.linalg.norm(Q - ref) / np.linalg.norm(ref) < 1e-14


@pytest.mark.gpu
def test_batched_lyapunov_large_instances_match_oracle():
    rng = np.random.default_rng(11)
    inst = []
    for N, s in ((128, 4), (160, 2), (64, 1), (140, 4)):
        A = wl.laplacian_2d(N, float(rng.uniform(0.2, 1.0)))
        inst.append((A, rng.standard_normal((N * N, s))))
    tol = 1e-10
    with ps.BatchSolver([a for a, _ in inst], [c for _, c in inst]) as bs:
        info = bs.cg(tol, 500)
        assert info["status"] == ps.SYLV_OK, info
        assert info["true_rel_bound"] <= tol
        for i, (A, C) in enumerate(inst):
            V, Xh, W = bs.factors(i)
            hist = bs.history(i)
            ref = fz.factorized_cg(A.to_scipy(), None, C, None, tol * STOP_MARGIN, 500, lyapunov=True)
            assert ref.status == "converged"
            assert len(hist) - 1 == ref.iters, (i, len(hist) - 1, ref.iters)
            np.testing.assert_allclose(hist[:10], ref.history[:10], rtol=1e-8)
            d = factored_rel_diff(V, Xh, V, ref.V, ref.Xhat, ref.V)
            assert d < TOL_X, (i, d)

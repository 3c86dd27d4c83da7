"""The float64 true-residual certificate on both of its product paths.

The certificate applies X = V X^ W^T (summed over the refinement rounds) to thin Gaussian
blocks.  Its tall-skinny products with the bases run either on the tensor cores, on FP16 digit
planes of the bases (float64-accurate), or on double-float kernels on the FP32 pipes (unit
roundoff ~2^-48).  The library picks the planes for large bases only; sylv_options.cert_gemm
forces either path, so that both are checked here on small cases:

- the estimate and the certified bound of the two paths agree to 1e-6 relative (same probes,
  same solve): R = C1 C2^T - A X - X B is about tol = 1e-8 of the terms that cancel to form it,
  so the double-float products' unit roundoff 2^-48 ~ 3.6e-15 becomes ~4e-7 relative to R (the
  digit-plane products are below that); and the refinement rounds of the mixed mode take the
  same decisions;
- the oracle's direct residual (formed from X) is within the bound, the bound within tol, and
  the estimate within 20% of the oracle's value.

Cases: mixed BiCGSTAB (float32 bases split into planes after each round), float64 CG (Lanczos
bases on the CUDA cores), float64 BiCGSTAB with the Arnoldi bases kept on the CUDA cores
(basis_gemm = 1), and float64 BiCGSTAB on the tensor-core bases (their own planes).
"""
import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl
from oracle import residual

pytestmark = pytest.mark.gpu

TOL = 1e-8


def run(A, B, C1, C2, method, precision, cert_gemm, lyapunov=False, **kw):
    with ps.Solver(A, None if lyapunov else B, C1, None if lyapunov else C2, precision=precision,
                   lyapunov=lyapunov, cert_gemm=cert_gemm, **kw) as sv:
        info = sv.cg(TOL, 400) if method == "cg" else sv.bicgstab(TOL, 300)
        V, Xh, W = sv.factors()
    return info, V, Xh, W


def direct_rel(A, B, C1, C2, V, Xh, W):
    return residual.direct(A.to_scipy(), B.to_scipy(), C1, C2, V, Xh, W) / np.linalg.norm(C1 @ C2.T)


CASES = [
    ("mixed_bicgstab", "bicgstab", "mixed", {}, lambda: (wl.convdiff_3d(16, 1), wl.convdiff_3d(12, 2), 4)),
    ("fp64_cg_lanczos", "cg", "fp64", {}, lambda: (wl.laplacian_2d(48, 0.5), wl.laplacian_2d(40, 0.5), 4)),
    ("fp64_bicgstab_cuda_core_bases", "bicgstab", "fp64", {"basis_gemm": 1},
     lambda: (wl.convdiff_3d(14, 1), wl.convdiff_3d(11, 2), 4)),
    ("fp64_bicgstab_tensor_bases", "bicgstab", "fp64", {}, lambda: (wl.convdiff_3d(14, 1), wl.convdiff_3d(11, 2), 3)),
]


@pytest.mark.parametrize("name,method,precision,kw,make", CASES, ids=[c[0] for c in CASES])
def test_certificate_paths_agree_and_meet_tol(name, method, precision, kw, make):
    A, B, s = make()
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 0)
    res = {}
    for cg in (1, 2):
        info, V, Xh, W = run(A, B, C1, C2, method, precision, cg, **kw)
        assert info["status"] == ps.SYLV_OK, (name, cg, info)
        t = direct_rel(A, B, C1, C2, V, Xh, W)
        assert t <= info["true_rel_bound"] <= TOL, (name, cg, t, info)
        assert abs(info["true_rel_res"] - t) <= 0.2 * t, (name, cg, t, info)
        res[cg] = info
    a, b = res[1], res[2]
    assert a["iters"] == b["iters"] and a["refinements"] == b["refinements"], (a, b)
    for key in ("true_rel_res", "true_rel_bound"):
        assert abs(a[key] - b[key]) <= 1e-6 * a[key], (name, key, a[key], b[key])

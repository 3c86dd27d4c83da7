"""sylv_spmm_noalloc: the sparse block product for callers that cannot allocate.

Some callers cannot call cudaMalloc: processes whose device memory belongs to
another allocator (a framework's caching pool that holds the device memory
budget) and latency-bound loops that cannot afford the device-wide
synchronisation cudaMalloc/cudaFree may cause.  sylv_spmm_noalloc gives them
Y = A X with device pointers only, staging through a fixed array compiled into
the library instead of per-call buffers.  This test calls it through the C ABI
twice in a row and checks each result against the existing entry point
sylv_apply (which allocates its staging), within the FP64 SpMM tolerance the
other parity tests use; checks that a call leaves the device's free memory
unchanged (after the first call, which may load the library's device image);
and checks that oversized requests and host pointers are refused.
"""
import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl

pytestmark = pytest.mark.gpu

MAX_ELEMS = 1 << 20  # SYLV_NOALLOC_MAX_ELEMS in include/sylv.h
TOL = 1e-14  # FP64 SpMM tolerance of tests/test_gpu_parity.py


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_spmm_noalloc_matches_sylv_apply_on_two_calls():
    import torch

    n = 5003  # ragged: not a multiple of the CTA size
    A = wl.random_sparse(n, 4, 7)
    C1, C2 = wl.rhs(n, n, 2, 0)
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    val = torch.from_numpy(A.val).to(dev)
    stream = torch.cuda.Stream(device=dev)
    with ps.Solver(A, A, C1, C2) as sv:
        for call, k in enumerate((3, 8)):
            X = np.random.default_rng(call).standard_normal((n, k))
            Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(dev)  # (k, n) rows = n x k column-major
            Yd = torch.full((k, n), float("nan"), dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info(dev)[0]
            rc = ps.sylv_spmm_noalloc(n, A.nnz, rp.data_ptr(), ci.data_ptr(), val.data_ptr(), Xd.data_ptr(),
                                      Yd.data_ptr(), k, stream.cuda_stream)
            assert rc == ps.SYLV_OK, ps.last_error()
            stream.synchronize()
            if call == 1:  # the array is resident after the first call: nothing more is taken
                free_after = torch.cuda.mem_get_info(dev)[0]
                assert free_after == free_before, (free_before, free_after)
            Y = Yd.cpu().numpy().T
            Y_ref = sv.apply(0, X)  # existing entry point
            assert np.all(np.isfinite(Y))
            assert rel(Y, Y_ref) <= TOL, (call, rel(Y, Y_ref))
            assert rel(Y, A.to_scipy() @ X) <= TOL


def test_spmm_noalloc_rejects_sizes_beyond_its_staging():
    import torch

    dev = torch.device("cuda", 0)
    k = 8
    n = MAX_ELEMS // k + 1
    dummy_i = torch.zeros(4, dtype=torch.int32, device=dev)
    dummy_d = torch.zeros(4, dtype=torch.float64, device=dev)
    rc = ps.sylv_spmm_noalloc(n, 1, dummy_i.data_ptr(), dummy_i.data_ptr(), dummy_d.data_ptr(), dummy_d.data_ptr(),
                              dummy_d.data_ptr(), k, 0)
    assert rc == ps.SYLV_EINVAL
    assert "staging" in ps.last_error()


def test_spmm_noalloc_rejects_host_pointers():
    import torch

    dev = torch.device("cuda", 0)
    n, k = 64, 2
    A = wl.random_sparse(n, 3, 1)
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    val = torch.from_numpy(A.val).to(dev)
    Xh = np.zeros((k, n))  # host memory
    Yd = torch.zeros((k, n), dtype=torch.float64, device=dev)
    rc = ps.sylv_spmm_noalloc(n, A.nnz, rp.data_ptr(), ci.data_ptr(), val.data_ptr(), Xh.ctypes.data,
                              Yd.data_ptr(), k, 0)
    assert rc == ps.SYLV_EINVAL
    assert "current device" in ps.last_error()

"""C-ABI library checks that need no GPU: it builds, loads, exports every symbol
include/sylv.h declares, and its host-side argument validation rejects bad
input before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(ps.LIB_PATH):
        from paper_2605_28274_gb300 import build

        build.build()
    return ps.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "sylv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sylv_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(ps.EXPORTS) == names


def test_strerror_and_defaults(lib):
    assert lib.sylv_strerror(0) == b"converged"
    assert b"breakdown" in lib.sylv_strerror(4)
    o = ps.sylv_default_options()
    assert o.precision == 0 and o.poll_every == 8 and o.timeout_s == 3600.0 and o.refine_max == 12
    assert o.small_gemm == 0 and o.basis_gemm == 0 and o.cert_gemm == 0


def _create(A, B, C1, C2, s=None, opt=None):
    ca, ka = ps._make_csr(A)
    cb, kb = (None, None) if B is None else ps._make_csr(B)
    C1f = np.asfortranarray(C1)
    C2f = None if C2 is None else np.asfortranarray(C2)
    h = ctypes.c_void_p()
    rc = ps.load().sylv_create(ctypes.byref(ca), None if cb is None else ctypes.byref(cb), ps._dptr(C1f),
                               None if C2f is None else ps._dptr(C2f), C1.shape[1] if s is None else s,
                               None if opt is None else ctypes.byref(opt), ctypes.byref(h))
    return rc, h


def test_invalid_arguments_rejected_on_host(lib):
    A = wl.laplacian_2d(4)
    C1, C2 = wl.rhs(16, 16, 2, 0)
    assert _create(A, A, C1, C2, s=0)[0] == ps.SYLV_EINVAL
    assert _create(A, A, C1, C2, s=9)[0] == ps.SYLV_EINVAL
    bad = wl.laplacian_2d(4)
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[3] = 99  # column out of range
    assert _create(bad, A, C1, C2)[0] == ps.SYLV_EINVAL
    bad2 = wl.laplacian_2d(4)
    bad2.row_ptr = bad2.row_ptr.copy()
    bad2.row_ptr[5], bad2.row_ptr[6] = bad2.row_ptr[6], bad2.row_ptr[5]  # decreasing
    assert _create(bad2, A, C1, C2)[0] == ps.SYLV_EINVAL
    o = ps.sylv_default_options()
    o.lyapunov = 1
    assert _create(A, A, C1, C2, opt=o)[0] == ps.SYLV_EINVAL  # Lyapunov needs B = C2 = NULL
    o.lyapunov = 0
    o.precision = 7
    assert _create(A, A, C1, C2, opt=o)[0] == ps.SYLV_EINVAL
    o.precision = 0
    o.basis_gemm = 3
    assert _create(A, A, C1, C2, opt=o)[0] == ps.SYLV_EINVAL
    o.basis_gemm = 0
    o.cert_gemm = 3
    assert _create(A, A, C1, C2, opt=o)[0] == ps.SYLV_EINVAL
    small = wl.laplacian_2d(1)
    assert _create(small, small, np.ones((1, 2)), np.ones((1, 2)))[0] == ps.SYLV_EINVAL  # n < s
    assert ps.last_error() != ""


def test_handle_calls_reject_null(lib):
    info = ps.sylv_info()
    assert lib.sylv_cg(None, 1e-8, 10, ctypes.byref(info)) == ps.SYLV_EINVAL
    assert lib.sylv_get_factors(None, None, None, None, None) == ps.SYLV_EINVAL
    lib.sylv_destroy(None)


def test_no_device_is_an_error_not_a_fallback(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    A = wl.laplacian_2d(4)
    C1, C2 = wl.rhs(16, 16, 1, 0)
    rc, h = _create(A, A, C1, C2)
    assert rc == ps.SYLV_ECUDA and not h.value


def test_struct_layouts_match_the_c_header(tmp_path):
    """The ctypes mirrors of the C structs (sylv_csr, sylv_options, sylv_info, sylv_kernel_stat)
    have the header's sizes and field offsets: a field added on one side only would shift every
    later field of a call silently.  A C program compiled against include/sylv.h prints them."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [ps.sylv_csr, ps.sylv_options, ps.sylv_info, ps.sylv_kernel_stat]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sylv.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            *key, val = ln.split()
            got[" ".join(key)] = int(val)
    for st in structs:
        name = st.__name__
        assert got[f"{name} size"] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert got[f"{name} {field}"] == getattr(st, field).offset, (name, field)

"""Host-side checks of the C ABI (no GPU needed, no compute call).

* libgvt.so loads and exports every entry point that include/gvt.h declares;
* the binding's ctypes structures have the C layout (checked by compiling a
  tiny C program against the header);
* the sum-of-Kronecker descriptors that gvt_desc_make returns, evaluated term
  by term on the CPU, equal the oracle's Table 4b kernel values;
* argument errors come back as statuses with a message.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as orc
from conftest import ROOT
from paper_2009_01054_gb300 import build as gbuild
from paper_2009_01054_gb300 import gvt, synth

HEADER = os.path.join(ROOT, "include", "gvt.h")


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gvt.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(gvt_[a-z_0-9]+)\s*\(", src, re.M)))


def test_header_declares_the_expected_boundary():
    names = declared_functions()
    for must in ["gvt_create", "gvt_destroy", "gvt_plan_create", "gvt_plan_destroy", "gvt_matvec",
                 "gvt_desc_make", "gvt_pairwise_kernel_matvec", "gvt_krr_cg_solve", "gvt_predict"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", gvt.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    bound = {s[0] for s in gvt.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "gvt.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(gvt_term), sizeof(gvt_desc), sizeof(gvt_matrix),
         sizeof(gvt_solve_opts), sizeof(gvt_solve_info));
  printf("%zu %zu %zu %zu %zu %zu\\n", offsetof(gvt_desc, terms), offsetof(gvt_matrix, dtype),
         offsetof(gvt_solve_opts, inner_tol), offsetof(gvt_solve_info, rel_residual),
         offsetof(gvt_solve_opts, precond), offsetof(gvt_solve_info, precond_fallback));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(x) for x in lines[0].split()]
    offs = [int(x) for x in lines[1].split()]
    assert sizes == [ctypes.sizeof(gvt.gvt_term), ctypes.sizeof(gvt.gvt_desc), ctypes.sizeof(gvt.gvt_matrix),
                     ctypes.sizeof(gvt.gvt_solve_opts), ctypes.sizeof(gvt.gvt_solve_info)]
    assert offs == [gvt.gvt_desc.terms.offset, gvt.gvt_matrix.dtype.offset,
                    gvt.gvt_solve_opts.inner_tol.offset, gvt.gvt_solve_info.rel_residual.offset,
                    gvt.gvt_solve_opts.precond.offset, gvt.gvt_solve_info.precond_fallback.offset]


EXPECTED_TERMS = {"kronecker": 1, "gaussian": 1, "linear": 2, "poly2d": 3, "cartesian": 2,
                  "symmetric": 2, "antisymmetric": 2, "ranking": 4, "mlpk": 10}


def _factor_value(f, M, N, r, c):
    if f == gvt.GVT_FACTOR_M:
        return M[r, c]
    if f == gvt.GVT_FACTOR_N:
        return N[r, c]
    if f == gvt.GVT_FACTOR_M_SQ:
        return M[r, c] ** 2
    if f == gvt.GVT_FACTOR_N_SQ:
        return N[r, c] ** 2
    if f == gvt.GVT_FACTOR_ONES:
        return 1.0
    if f == gvt.GVT_FACTOR_IDENTITY:
        return float(r == c)
    raise ValueError(f)


def _desc_matrix(desc, M, N, d_out, t_out, d_in, t_in):
    """The descriptor's sum of Kronecker terms, evaluated entry by entry (test-side)."""
    if desc.homogeneous:
        N = M
    K = np.zeros((len(d_out), len(d_in)))
    for i, (a, b) in enumerate(zip(d_out, t_out)):
        for j, (c, e) in enumerate(zip(d_in, t_in)):
            o, n_ = (a, b), (c, e)
            s = 0.0
            for k in range(desc.n_terms):
                t = desc.terms[k]
                s += t.coef * _factor_value(t.factor_a, M, N, o[t.out_a], n_[t.in_a]) * \
                    _factor_value(t.factor_b, M, N, o[t.out_b], n_[t.in_b])
            K[i, j] = s
    return K


@pytest.mark.parametrize("kind", list(EXPECTED_TERMS))
def test_descriptor_equals_table4b(lib, kind):
    d = gvt.gvt_desc_make(kind)
    assert d.n_terms == EXPECTED_TERMS[kind]
    assert bool(d.homogeneous) == (kind in gvt.HOMOGENEOUS)
    rng = np.random.default_rng(21)
    m = 6
    q = m if kind in gvt.HOMOGENEOUS else 5
    M = orc.gaussian_kernel(rng.standard_normal((m, 3)), gamma=0.5)
    N = orc.gaussian_kernel(rng.standard_normal((q, 3)), gamma=0.5)
    d_in, t_in = synth.random_pairs(rng, 15, m, q)
    d_out, t_out = synth.random_pairs(rng, 11, m, q)
    np.testing.assert_allclose(_desc_matrix(d, M, N, d_out, t_out, d_in, t_in),
                               orc.kernel_matrix(kind, M, N, d_out, t_out, d_in, t_in),
                               rtol=1e-13, atol=1e-13)


def test_argument_errors_return_status_and_message(lib):
    d = gvt.gvt_desc()
    st = lib.gvt_desc_make(99, ctypes.byref(d))
    assert st == 1 and "unknown" in gvt.last_error()
    st = lib.gvt_create(None)
    assert st == 1
    assert lib.gvt_destroy(None) == 0 and lib.gvt_plan_destroy(None) == 0


def test_null_handle_arguments_are_rejected_without_device_work(lib):
    """Entry points added for engine control, the factor cache, the base kernels and the other
    losses check their arguments before touching the device: a NULL handle or plan is
    GVT_ERR_INVALID_ARG with a message, on a machine without a GPU."""
    for mode in (0, 1, 2, 3, -1):
        assert lib.gvt_set_tc_pairs(None, mode) == gvt.GVT_ERR_INVALID_ARG
    assert "gvt_set_tc_pairs" in gvt.last_error()
    assert lib.gvt_factor_cache_begin(None) == gvt.GVT_ERR_INVALID_ARG
    assert lib.gvt_factor_cache_end(None) == gvt.GVT_ERR_INVALID_ARG
    assert "gvt_factor_cache_end" in gvt.last_error()
    assert lib.gvt_linear_kernel(None, None, 4, None, 4, 3, None, 4, gvt.GVT_F64, None) == gvt.GVT_ERR_INVALID_ARG
    assert "gvt_linear_kernel" in gvt.last_error()
    info = gvt.gvt_solve_info()
    st = lib.gvt_svm_newton_solve(None, None, None, None, None, None, 0.1, None, 10, 1e-10, 100,
                                  ctypes.byref(info), None)
    assert st == gvt.GVT_ERR_INVALID_ARG and info.status == gvt.GVT_ERR_INVALID_ARG
    assert "gvt_svm_newton_solve" in gvt.last_error()


def test_solve_defaults(lib):
    o = gvt.gvt_solve_opts_default()
    assert o.rel_tol == 1e-6 and o.mode == gvt.GVT_SOLVE_FP64_CG and o.inner_tol == 1e-3
    assert o.precond_budget == 0 and not o.precond
    assert gvt.gvt_version() >= 10000


def test_static_product_refuses_sizes_whose_byte_count_wraps(lib):
    """gvt_matvec_static refuses a declared q_rows x m_cols whose byte count wraps 2^64 (2^29 x 2^32
    FP64 elements = 2^64 bytes, 0 after wrapping) before any CUDA call: the check runs on the host,
    so it is exercised here without a GPU.  The matrix structs only declare their extents."""
    buf = (ctypes.c_double * 4)()
    X, Y = 1 << 32, 1 << 29
    Mm = gvt.gvt_matrix(ctypes.cast(buf, ctypes.c_void_p), 1, X, X, gvt.GVT_F64, 0)
    Nm = gvt.gvt_matrix(ctypes.cast(buf, ctypes.c_void_p), Y, 1, 1, gvt.GVT_F64, 0)
    idx = (ctypes.c_int32 * 1)()
    st = lib.gvt_matvec_static(1, X, Y, 1, ctypes.cast(idx, ctypes.c_void_p), ctypes.cast(idx, ctypes.c_void_p),
                               1, None, None, 0, ctypes.byref(Mm), ctypes.byref(Nm),
                               ctypes.cast(buf, ctypes.c_void_p), ctypes.cast(buf, ctypes.c_void_p),
                               gvt.GVT_F64, None)
    assert st == gvt.GVT_ERR_INVALID_ARG
    assert "static scratch" in gvt.last_error()

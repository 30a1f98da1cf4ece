"""The C-ABI library builds, loads and exports every symbol of include/tb.h, and
argument checks that need no GPU reject bad input (no GPU)."""
import ctypes
import os
import re

import pytest

import paper_2411_03029_gb300 as tb
from paper_2411_03029_gb300 import build as tbbuild

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(tb_[a-z_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    tbbuild.build()
    return tb.lib()


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("tb_build", "tb_apply", "tb_apply_adjoint", "tb_free"):
        assert must in names
    assert set(names) == set(tb.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_defaults(lib):
    assert b"sm_103a" in lib.tb_version()
    opt = tb._Options()
    assert lib.tb_options_default(ctypes.byref(opt)) == 0
    assert opt.L == -1 and opt.proxy_rows == 1024 and opt.rank_max == 32 and opt.separable == -1
    assert opt.sep_schedule == 0
    assert opt.mode_slices == 0


def test_build_rejects_an_unknown_slice_count_without_touching_the_gpu(lib):
    import numpy as np
    kern = tb._Kernel(tb.KERNEL_FOURIER, (ctypes.c_double * 4)())
    xs = [np.arange(16) / 16.0 for _ in range(2)]
    ys = [np.arange(16) - 8.0 for _ in range(2)]
    grids = tb._Grids()
    for k in range(2):
        grids.x[k] = xs[k].ctypes.data
        grids.y[k] = ys[k].ctypes.data
    opt = tb._Options()
    assert lib.tb_options_default(ctypes.byref(opt)) == 0
    opt.mode_slices = 3
    n = (ctypes.c_int64 * 2)(16, 16)
    h = ctypes.c_void_p()
    assert lib.tb_build_ex(ctypes.byref(kern), 2, ctypes.cast(n, ctypes.c_void_p), ctypes.byref(grids), 1e-6,
                           ctypes.byref(opt), ctypes.byref(h)) == 1
    assert b"mode_slices" in lib.tb_last_error()
    assert not h.value


def test_build_rejects_an_unknown_separable_schedule_without_touching_the_gpu(lib):
    import numpy as np
    kern = tb._Kernel(tb.KERNEL_FOURIER, (ctypes.c_double * 4)())
    xs = [np.arange(16) / 16.0 for _ in range(2)]
    ys = [np.arange(16) - 8.0 for _ in range(2)]
    grids = tb._Grids()
    for k in range(2):
        grids.x[k] = xs[k].ctypes.data
        grids.y[k] = ys[k].ctypes.data
    opt = tb._Options()
    assert lib.tb_options_default(ctypes.byref(opt)) == 0
    opt.sep_schedule = 99
    n = (ctypes.c_int64 * 2)(16, 16)
    h = ctypes.c_void_p()
    assert lib.tb_build_ex(ctypes.byref(kern), 2, ctypes.cast(n, ctypes.c_void_p), ctypes.byref(grids), 1e-6,
                           ctypes.byref(opt), ctypes.byref(h)) == 1
    assert b"sep_schedule" in lib.tb_last_error()
    assert not h.value


def test_free_null_is_ok(lib):
    assert lib.tb_free(None) == 0


def test_build_rejects_bad_arguments_without_touching_the_gpu(lib):
    kern = tb._Kernel(tb.KERNEL_FOURIER, (ctypes.c_double * 4)())
    grids = tb._Grids()
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 2)(16, 16)
    # d out of range
    assert lib.tb_build(ctypes.byref(kern), 0, ctypes.cast(n, ctypes.c_void_p), ctypes.byref(grids), 1e-6,
                        ctypes.byref(h)) == 1
    assert b"d must be" in lib.tb_last_error()
    # NULL grid pointers
    assert lib.tb_build(ctypes.byref(kern), 2, ctypes.cast(n, ctypes.c_void_p), ctypes.byref(grids), 1e-6,
                        ctypes.byref(h)) == 1
    # tolerance
    assert lib.tb_build(ctypes.byref(kern), 2, ctypes.cast(n, ctypes.c_void_p), ctypes.byref(grids), 2.0,
                        ctypes.byref(h)) == 1
    # bad kernel kind
    bad = tb._Kernel(9, (ctypes.c_double * 4)())
    assert lib.tb_build(ctypes.byref(bad), 2, ctypes.cast(n, ctypes.c_void_p), ctypes.byref(grids), 1e-6,
                        ctypes.byref(h)) == 1
    assert not h.value


def test_apply_rejects_null_handle(lib):
    assert lib.tb_apply_host_batch(None, None, None, 1, 1, 1) == 1
    assert lib.tb_apply(None, None, None, 1, 0, None) == 1
    assert lib.tb_apply_adjoint(None, None, None, 1, 0, None) == 1
    assert lib.tb_query(None, None) == 1


def test_autotune_and_apply_reject_a_null_handle_without_touching_the_gpu(lib):
    assert lib.tb_autotune(None, 1, tb.PREC_C64, None) == 1          # TB_EINVAL
    assert b"handle" in lib.tb_last_error()
    assert lib.tb_apply(None, None, None, 1, tb.PREC_C64, None) == 1
    opt = tb._Options()
    assert lib.tb_options_default(ctypes.byref(opt)) == 0
    assert opt.autotune == 0                                           # off unless asked for


def test_build_rejects_bad_kernel_parameters_without_touching_the_gpu(lib):
    import numpy as np
    xs = [np.arange(16) / 16.0 for _ in range(3)]
    ys = [np.arange(16) - 8.0 for _ in range(3)]
    grids = tb._Grids()
    for k in range(3):
        grids.x[k] = xs[k].ctypes.data
        grids.y[k] = ys[k].ctypes.data
    n = (ctypes.c_int64 * 3)(16, 16, 16)
    h = ctypes.c_void_p()
    # the anisotropic Radon phase (Eq. randon2d) is defined for d = 2 only
    aniso = tb._Kernel(tb.KERNEL_RADON_ANISO, (ctypes.c_double * 4)(2 / 16, 1 / 16, 2 / 16, 1 / 16))
    assert lib.tb_build(ctypes.byref(aniso), 3, ctypes.cast(n, ctypes.c_void_p), ctypes.byref(grids), 1e-6,
                        ctypes.byref(h)) == 1
    assert b"d = 2" in lib.tb_last_error()
    # a negative plate distance h
    plates = tb._Kernel(tb.KERNEL_HELMHOLTZ, (ctypes.c_double * 4)(10.0, -1.0, 0.0, 0.0))
    assert lib.tb_build(ctypes.byref(plates), 2, ctypes.cast(n, ctypes.c_void_p), ctypes.byref(grids), 1e-6,
                        ctypes.byref(h)) == 1
    assert b"offset" in lib.tb_last_error()
    # h = 0 on coincident grids: the Green's function is singular
    same = tb._Kernel(tb.KERNEL_HELMHOLTZ, (ctypes.c_double * 4)(10.0, 0.0, 0.0, 0.0))
    g2 = tb._Grids()
    for k in range(2):
        g2.x[k] = xs[k].ctypes.data
        g2.y[k] = xs[k].ctypes.data
    assert lib.tb_build(ctypes.byref(same), 2, ctypes.cast(n, ctypes.c_void_p), ctypes.byref(g2), 1e-6,
                        ctypes.byref(h)) == 1
    assert b"coincides" in lib.tb_last_error()
    assert not h.value


def test_cgls_and_alu_peak_reject_bad_arguments_without_touching_the_gpu(lib):
    assert lib.tb_cgls(None, None, None, 1, 5, tb.PREC_C64, 1, None, None) == 1      # NULL handle
    assert b"handle" in lib.tb_last_error()
    out = ctypes.c_double()
    assert lib.tb_alu_peak(tb.PREC_C64, None, None) == 1                            # NULL result
    assert lib.tb_alu_peak(tb.PREC_C64_SPLITBF16, None, ctypes.byref(out)) == 1     # no FMA pipe of its own
    assert b"precision" in lib.tb_last_error()

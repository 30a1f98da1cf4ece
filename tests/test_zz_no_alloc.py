"""tb_apply_noalloc: the apply that allocates no device memory.

Some callers cannot call cudaMalloc while they apply the operator: processes
whose device memory is owned by another allocator (a framework's caching
allocator, a fixed arena, a hard memory cap) and latency-critical loops that
cannot take the device-wide synchronisation of cudaMalloc / cudaFree.  For
them the library keeps the level intermediates in a fixed scratch array
compiled into it.  These tests call that entry point through the C ABI and
compare it with tb_apply on the same handles:

  * the first call on each handle gets an all-NaN input (NaN is data, not a
    fault), so the scratch then holds NaN wherever a pass wrote; the later calls
    with clean inputs, on the same handle and on a second handle of another
    shape, must come out exactly as tb_apply's: a pass that read a scratch entry
    it had not written in the same call would carry the stale NaN through;
  * complex64, complex128, the split-BF16 tensor-core core and a separable
    (per-mode) handle;
  * two calls in a row, with no handle memory taken by them;
  * requests larger than the scratch are rejected.

The file is named so that pytest collects it last.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import paper_2411_03029_gb300 as tb
import workloads as W

pytestmark = pytest.mark.gpu


def _call(op, f, u, precision):
    lib = tb.lib()
    stream = torch.cuda.current_stream().cuda_stream
    return lib.tb_apply_noalloc(op._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                f.shape[-1], precision, ctypes.c_void_p(stream))


def _noalloc(op, f, precision):
    u = torch.full_like(f, float("nan"))
    status = _call(op, f, u, precision)
    assert status == 0, tb.lib().tb_last_error().decode()
    torch.cuda.synchronize()
    return u


def _rel(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


# (workload, precisions with the tolerance against tb_apply)
CASES = [
    ("radon", W.small("radon2d_n256", 64, nv=3, L=4), ((tb.PREC_C64, 1e-6), (tb.PREC_C128, 1e-13))),
    ("helmholtz-splitbf16", W.small("helmholtz3d_n256", 32, nv=16, L=2, params=(2 * math.pi * 8,)),
     ((tb.PREC_C64_SPLITBF16, 1e-6),)),
    ("fourier-separable", W.small("fourier2d_n64", 64, nv=2), ((tb.PREC_C64, 1e-6), (tb.PREC_C128, 1e-13))),
]
SECOND = {   # a second handle of another shape, applied after the first handle's calls
    "radon": W.small("radon2d_n256", 32, nv=2, L=2),
    "helmholtz-splitbf16": W.small("helmholtz3d_n256", 16, nv=5, L=2, params=(2 * math.pi * 4,)),
    "fourier-separable": W.small("fourier2d_n64", 32, nv=3),
}


@pytest.mark.parametrize("name,w,precs", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_tb_apply_after_nan_input(name, w, precs):
    tb.build.build()
    torch.cuda.set_device(0)
    mask = sum(1 << p for p, _ in precs)
    op = tb.from_workload(w, precisions=mask)
    op2 = tb.from_workload(SECOND[name], precisions=mask)
    for prec, tol in precs:
        dt = tb.dtype_of(prec)
        f1 = W.rhs(w).to(dt).cuda()
        f2 = W.complex_gaussian(f1.shape, 99).to(dt).cuda()
        g1 = W.rhs(SECOND[name]).to(dt).cuda()
        fnan = torch.full_like(f1, float("nan"))
        # the allocating entry point, for comparison (allocates the handle workspaces)
        ref1, ref2, refg = op.apply(f1, prec), op.apply(f2, prec), op2.apply(g1, prec)
        refnan = op.apply(fnan, prec)
        torch.cuda.synchronize()
        # first call: NaN input; it also does the one-time scratch look-up on this device
        unan = _noalloc(op, fnan, prec)
        assert torch.equal(torch.isnan(unan), torch.isnan(refnan))
        bytes1, bytes2 = op.info()["device_bytes"], op2.info()["device_bytes"]
        free0 = torch.cuda.mem_get_info()[0]
        u1 = _noalloc(op, f1, prec)
        u2 = _noalloc(op, f2, prec)
        ug = _noalloc(op2, g1, prec)
        for got, ref, what in ((u1, ref1, "first clean call"), (u2, ref2, "second clean call"),
                               (ug, refg, "second handle")):
            assert torch.isfinite(got).all(), f"{name} {prec} {what}: stale scratch entry read"
            err = _rel(got, ref)
            assert err < tol, f"{name} {prec} {what}: rel err {err:.3e}"
        # the calls took no memory: the handles hold what they held, and device-wide
        # free memory did not drop by as much as one level tensor of the smaller handle
        assert op.info()["device_bytes"] == bytes1 and op2.info()["device_bytes"] == bytes2
        level_bytes = op2.info()["level_entries_max"] * g1.shape[-1] * g1.element_size()
        assert free0 - torch.cuda.mem_get_info()[0] < level_bytes
    op.close()
    op2.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    torch.cuda.set_device(0)
    w = W.small("radon2d_n256", 64, nv=1, L=4)
    op = tb.from_workload(w, precisions=1 << tb.PREC_C64)
    nv = 4096                             # 2 x level tensor x nv x 8 B > 64 MiB
    f = torch.zeros((64, 64, nv), dtype=torch.complex64, device="cuda")
    u = torch.empty_like(f)
    assert _call(op, f, u, tb.PREC_C64) == 6          # TB_EUNSUPPORTED
    assert b"scratch" in tb.lib().tb_last_error()
    # an nv whose scratch size would wrap a 64-bit product is rejected the same way,
    # before any pointer range is formed
    lib = tb.lib()
    stream = torch.cuda.current_stream().cuda_stream
    status = lib.tb_apply_noalloc(op._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                  (1 << 62), tb.PREC_C64, ctypes.c_void_p(stream))
    assert status in (1, 6)
    op.close()

"""tb_apply_noalloc: the apply that allocates no device memory.

Some callers cannot call cudaMalloc while they apply the operator: processes
whose device memory is owned by another allocator (a framework's caching
allocator, a fixed arena, a hard memory cap) and latency-critical loops that
cannot take the device-wide synchronisation of cudaMalloc / cudaFree.  For
them the library keeps the level intermediates in a fixed scratch array
compiled into it.  This test calls that entry point through the C ABI and
checks it against tb_apply on the same handle, twice in a row (the scratch
keeps the previous call's contents), and that it rejects requests larger than
its scratch.  The file is named so that pytest collects it last.
"""
import ctypes

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


def test_noalloc_apply_matches_tb_apply_twice():
    tb.build.build()
    torch.cuda.set_device(0)
    w = W.small("radon2d_n256", 64, nv=3, L=4)
    op = tb.from_workload(w, precisions=(1 << tb.PREC_C128) | (1 << tb.PREC_C64))
    lib = tb.lib()
    for prec, tol in ((tb.PREC_C64, 1e-6), (tb.PREC_C128, 1e-13)):
        f = W.rhs(w).to(tb.dtype_of(prec)).cuda()
        ref = op.apply(f, prec)            # the allocating entry point, for comparison
        torch.cuda.synchronize()
        outs = [torch.full_like(f, float("nan")) for _ in range(2)]
        free_after_first = None
        for call in range(2):
            status = _call(op, f, outs[call], prec)
            assert status == 0, lib.tb_last_error().decode()
            torch.cuda.synchronize()
            err = (torch.linalg.vector_norm(outs[call] - ref) / torch.linalg.vector_norm(ref)).item()
            assert err < tol, f"call {call}: rel err {err:.3e}"
            if call == 0:
                # the first call on a device looks up the scratch (one-time set-up);
                # after it, calls take no device memory
                free_after_first = torch.cuda.mem_get_info()[0]
        assert torch.cuda.mem_get_info()[0] == free_after_first
    op.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    torch.cuda.set_device(0)
    w = W.small("radon2d_n256", 64, nv=1, L=4)
    op = tb.from_workload(w, precisions=1 << tb.PREC_C64)
    nv = 4096                             # 2 x level tensor x nv x 8 B > 64 MiB
    f = torch.zeros((64, 64, nv), dtype=torch.complex64, device="cuda")
    u = torch.empty_like(f)
    assert _call(op, f, u, tb.PREC_C64) == 6          # TB_EUNSUPPORTED
    assert b"scratch" in tb.lib().tb_last_error()
    op.close()

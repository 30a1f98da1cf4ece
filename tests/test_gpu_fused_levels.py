"""The fused level passes (one persistent launch per pass, tb_level.cu) against
the per-mode launches (tb_mode.cu) on the same handles.

Both apply the same chains of mode products (Alg. 2, steps 1 and 3); the fused
pass uses another mode order (the fewest multiply-adds), Gauss's
three-multiplication complex products and paired FP32 FMAs, so the two agree
to FP32 rounding, not bit for bit.  The fused pass must also be independent of
its launch shape (RHS per work item, register chunk, grid), bit for bit, since
every output is accumulated in the same order.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_03029_gb300 as tb
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tb.build.build()
    oracle.build()
    torch.cuda.set_device(0)


def rel(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


CASES = [
    ("helmholtz3d_n16", W.small("helmholtz3d_n64", 16, nv=5, L=2)),
    ("helmholtz3d_n64_L4", W.small("helmholtz3d_n64", 64, nv=3, L=4)),
    ("radon2d_n64_L4", W.small("radon2d_n256", 64, nv=1, L=4)),
    ("radon2d_n256_L6", W.WORKLOADS["radon2d_n256"]),
    ("helmholtz3d_n32_bf16", W.small("helmholtz3d_n256", 32, nv=16, L=2, params=(2 * np.pi * 8,))),
]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_fused_level_passes_match_per_mode_launches(name, w):
    mask = (1 << tb.PREC_C64) | (1 << tb.PREC_C64_SPLITBF16)
    fused = tb.from_workload(w, precisions=mask, level_schedule=tb.LEVEL_FUSED)
    per_mode = tb.from_workload(w, precisions=mask, level_schedule=tb.LEVEL_PER_MODE)
    f = W.rhs(w).to(torch.complex64).cuda()
    precs = (tb.PREC_C64, tb.PREC_C64_SPLITBF16) if "bf16" in name else (tb.PREC_C64,)
    for prec in precs:
        for adj in (False, True):
            run = (lambda op: op.apply_adjoint(f, prec)) if adj else (lambda op: op.apply(f, prec))
            a, b = run(fused), run(per_mode)
            assert torch.isfinite(a).all()
            assert rel(a, b) < 1e-5, (prec, adj, rel(a, b))
    # the fused kernel really ran: one launch per level pass
    fused.profile(True)
    fused.apply(f, tb.PREC_C64)
    st = fused.profile_stats()
    fused.profile(False)
    for s in st:
        if s["name"] != "core":
            assert s["kernels"] == s["launches"], s
    fused.close()
    per_mode.close()


def test_fused_launch_shape_does_not_change_results():
    w = W.small("helmholtz3d_n64", 32, nv=7, L=2)
    op = tb.from_workload(w, precisions=1 << tb.PREC_C64, level_schedule=tb.LEVEL_FUSED)
    f = W.rhs(w).to(torch.complex64).cuda()
    ref = op.apply(f, tb.PREC_C64).clone()
    refv = op.apply_adjoint(f, tb.PREC_C64).clone()
    op.autotune(w.nv, tb.PREC_C64)        # tries other RHS chunks, register chunks and grids
    assert torch.equal(op.apply(f, tb.PREC_C64), ref)
    assert torch.equal(op.apply_adjoint(f, tb.PREC_C64), refv)
    op.close()

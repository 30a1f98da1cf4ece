"""tb_autotune: the empirical launch-shape search changes how the apply is
scheduled, never what it computes.

For a non-separable handle it picks, per level pass, side and mode, the
output rows per register tile, the grid size, the rank bounds, the threads per
block and the column slices; every output entry is still the same sum over the
same fiber in the same order (the rank bounds skip only exact zeros), so the
tuned apply must equal the untuned one bit for bit (forward and adjoint)
within one form of the level passes (per-mode launches, or fused launches).  With the built-in
rule it also picks per pass the faster of the two forms, which round
differently (FP32): there the bar is the complex64 rounding.  For a separable
handle it picks between per-mode fiber passes and multi-mode tile passes,
which sum in different orders: there the bar is the oracle's.
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
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name,n,L,nv", [("helmholtz3d_n64", 16, 2, 3), ("radon2d_n256", 64, 4, 2)])
def test_tuned_apply_is_bitwise_the_untuned_apply(name, n, L, nv):
    w = W.small(name, n, nv=nv, L=L)
    op = tb.from_workload(w, precisions=(1 << tb.PREC_C64) | (1 << tb.PREC_C128),
                          level_schedule=tb.LEVEL_PER_MODE)
    for prec in (tb.PREC_C64, tb.PREC_C128):
        f = W.rhs(w).to(tb.dtype_of(prec)).cuda()
        u0, v0 = op.apply(f, prec), op.apply_adjoint(f, prec)
        op.autotune(nv, prec)
        u1, v1 = op.apply(f, prec), op.apply_adjoint(f, prec)
        torch.cuda.synchronize()
        assert torch.equal(u0, u1)
        assert torch.equal(v0, v1)
    op.close()


@pytest.mark.parametrize("name,n,L,nv", [("helmholtz3d_n64", 16, 2, 1), ("helmholtz3d_n64", 32, 2, 3),
                                         ("radon2d_n256", 64, 4, 1), ("radon2d_n256", 128, 6, 2)])
def test_column_slices_are_bitwise_the_unsliced_apply(name, n, L, nv):
    # 2 or 4 groups of threads share each output column (each takes every
    # 2nd / 4th child or row chunk); complex128 ignores the option
    w = W.small(name, n, nv=nv, L=L)
    kw = dict(precisions=(1 << tb.PREC_C64) | (1 << tb.PREC_C128), level_schedule=tb.LEVEL_PER_MODE)
    ref = tb.from_workload(w, mode_slices=1, **kw)
    for prec in (tb.PREC_C64, tb.PREC_C128):
        f = W.rhs(w).to(tb.dtype_of(prec)).cuda()
        u0, v0 = ref.apply(f, prec).clone(), ref.apply_adjoint(f, prec).clone()
        for s in (2, 4):
            op = tb.from_workload(w, mode_slices=s, **kw)
            assert torch.equal(op.apply(f, prec), u0), (s, prec)
            assert torch.equal(op.apply_adjoint(f, prec), v0), (s, prec)
            op.close()
    ref.close()


def test_autotune_option_tunes_at_the_first_apply_and_matches_the_oracle():
    w = W.small("helmholtz3d_n64", 16, nv=2, L=2)
    op = tb.from_workload(w, autotune=True)
    f = W.rhs(w)
    u = op.apply(f.to(torch.complex64).cuda(), tb.PREC_C64).cpu().to(torch.complex128).numpy().reshape(-1, 2)
    assert rel(u, oracle.workload_apply(w, f)) < w.bound
    op.close()


def test_separable_choice_keeps_oracle_accuracy():
    w = W.Workload(name="f", kind=W.FOURIER, d=4, n=8, tol=1e-8, nv=3, precision=W.C64, bound=1e-5,
                   rhs_seeds=(0, 1, 2), samples=0, order=W.ORDER_BITREV, L=2)
    op = tb.from_workload(w)
    f = W.rhs(w)
    ref = oracle.fourier_fft(f.numpy(), 4).reshape(-1, 3)
    op.autotune(3, tb.PREC_C64)
    for adjoint in (False, True):
        x = f.to(torch.complex64).cuda()
        y = (op.apply_adjoint(x, tb.PREC_C64) if adjoint else op.apply(x, tb.PREC_C64)).cpu()
        y = y.to(torch.complex128).numpy().reshape(-1, 3)
        want = oracle.workload_apply_adjoint(w, f) if adjoint else ref
        assert rel(y, want) < 1e-5
    op.close()


@pytest.mark.parametrize("name,n,L,nv", [("helmholtz3d_n64", 32, 2, 3), ("radon2d_n256", 64, 4, 2)])
def test_tuned_choice_of_level_pass_form_keeps_complex64_rounding(name, n, L, nv):
    w = W.small(name, n, nv=nv, L=L)
    op = tb.from_workload(w, precisions=1 << tb.PREC_C64)
    f = W.rhs(w).to(torch.complex64).cuda()
    u0, v0 = op.apply(f, tb.PREC_C64), op.apply_adjoint(f, tb.PREC_C64)
    op.autotune(nv, tb.PREC_C64)
    u1, v1 = op.apply(f, tb.PREC_C64), op.apply_adjoint(f, tb.PREC_C64)
    for a, b in ((u1, u0), (v1, v0)):
        assert (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item() < 1e-5
    op.close()

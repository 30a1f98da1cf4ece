"""The level passes on the tcgen05 tensor cores (k_level_tc: one persistent
launch per pass, split-BF16 mode products) against the complex64 per-mode
launches on the same handle, against the exact DFT butterfly and against the
step-by-step oracle.

Both arms apply the same chains of mode products (Alg. 2, steps 1 and 3).  The
tensor-core arm stores each operand of a product as two BF16 terms (hi =
rn(v), lo = rn(v - hi): 2^-16 relative) and drops the lo x lo product
(2^-16), so each product carries at most 3 * 2^-16 relative error on top of
FP32 accumulation.  A chain applies 2 d (Lc + 1) + 1 such products (d per
level pass, Lc + 1 passes per side, and the core), and with errors adding at
most linearly the apply stays within
    bound(d, Lc) = 3 * 2^-16 * (2 d (Lc + 1) + 1)
of the exact butterfly (and of the FP32 apply, which is 1e3 times closer).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import butterfly as O2
import paper_2411_03029_gb300 as tb
import workloads as W

pytestmark = pytest.mark.gpu

BF = (1 << tb.PREC_C64) | (1 << tb.PREC_C64_SPLITBF16)


@pytest.fixture(scope="module", autouse=True)
def built():
    tb.build.build()
    oracle.build()
    torch.cuda.set_device(0)


def chain_bound(op):
    inf = op.info()
    return 3.0 * 2.0 ** -16 * (2 * inf["d"] * (inf["Lc"] + 1) + 1)


def rel(a, b):
    a = torch.as_tensor(a).reshape(-1).to(torch.complex128)
    b = torch.as_tensor(b).reshape(-1).to(torch.complex128)
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


CASES = [
    ("helmholtz3d_n16_nv5", W.small("helmholtz3d_n64", 16, nv=5, L=2)),
    ("helmholtz3d_n64_L4", W.small("helmholtz3d_n64", 64, nv=3, L=4)),
    ("radon2d_n64_L4", W.small("radon2d_n256", 64, nv=1, L=4)),
    ("radon2d_n256_L6", W.WORKLOADS["radon2d_n256"]),
    ("helmholtz3d_n32_nv16", W.small("helmholtz3d_n256", 32, nv=16, L=2, params=(2 * np.pi * 8,))),
    ("helmholtz3d_n64_nv16_L4", W.small("helmholtz3d_n256", 64, nv=16, L=4, params=(2 * np.pi * 16,))),
]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_tensor_core_level_passes_match_fp32_per_mode_launches(name, w):
    tc = tb.from_workload(w, precisions=BF, level_schedule=tb.LEVEL_TENSOR)
    f = W.rhs(w).to(torch.complex64).cuda()
    bound = chain_bound(tc)
    for adj in (False, True):
        run = (lambda p: tc.apply_adjoint(f, p)) if adj else (lambda p: tc.apply(f, p))
        fp32 = run(tb.PREC_C64).clone()          # level_schedule = 3 keeps complex64 on the per-mode launches
        y = run(tb.PREC_C64_SPLITBF16)
        assert torch.isfinite(y).all()
        e = rel(y, fp32)
        print(f"{name} adjoint={adj}: rel err vs FP32 {e:.2e} (bound {bound:.2e})")
        assert e < bound, (adj, e)
        assert torch.equal(y, run(tb.PREC_C64_SPLITBF16))   # deterministic
    # the tensor-core kernel really ran: one launch per level pass
    tc.profile(True)
    tc.apply(f, tb.PREC_C64_SPLITBF16)
    st = tc.profile_stats()
    tc.profile(False)
    assert any(s["name"] != "core" for s in st)
    for s in st:
        if s["name"] != "core":
            assert s["kernels"] == s["launches"], s
    tc.close()


@pytest.mark.parametrize("d,n,L", [(1, 64, 4), (2, 16, 2), (2, 64, 4), (3, 16, 2), (3, 32, 2)])
def test_tensor_core_levels_on_the_exact_dft_butterfly(d, n, L):
    # bit-reversed uniform DFT: every block has exact rank C_b, so the butterfly
    # is exact and what remains is the split-BF16 rounding of the chain
    w = W.Workload(name="f", kind=W.FOURIER, d=d, n=n, tol=1e-8, nv=3, precision=W.C128, bound=1e-12,
                   rhs_seeds=(0, 1, 2), samples=0, order=W.ORDER_BITREV, L=L)
    op = tb.from_workload(w, separable=0, precisions=BF, level_schedule=tb.LEVEL_TENSOR)
    f = W.rhs(w)
    x = f.to(torch.complex64).cuda()
    ref = oracle.fourier_fft(f.numpy(), d)
    refv = oracle.fourier_fft_adjoint(f.numpy(), d)
    bound = chain_bound(op)
    e = rel(op.apply(x, tb.PREC_C64_SPLITBF16).cpu(), torch.from_numpy(ref))
    ev = rel(op.apply_adjoint(x, tb.PREC_C64_SPLITBF16).cpu(), torch.from_numpy(refv))
    print(f"DFT d={d} n={n} L={L}: {e:.2e} / {ev:.2e} (bound {bound:.2e})")
    assert e < bound and ev < bound
    op.close()


def test_tensor_core_levels_match_the_step_oracle():
    w = W.small("helmholtz3d_n256", 32, nv=16, L=2, params=(2 * np.pi * 8,))
    op = tb.from_workload(w, precisions=BF | (1 << tb.PREC_C128), level_schedule=tb.LEVEL_TENSOR)
    bf = op.export()
    f = W.rhs(w)
    u = O2.apply(bf, f.numpy())
    v = O2.apply_adjoint(bf, f.numpy())
    x = f.to(torch.complex64).cuda()
    bound = chain_bound(op)
    assert rel(op.apply(x, tb.PREC_C64_SPLITBF16).cpu(), torch.from_numpy(u)) < bound
    assert rel(op.apply_adjoint(x, tb.PREC_C64_SPLITBF16).cpu(), torch.from_numpy(v)) < bound
    op.close()


def test_rule_and_tuner_pick_a_form_within_the_bound():
    w = W.small("helmholtz3d_n256", 32, nv=16, L=2, params=(2 * np.pi * 8,))
    op = tb.from_workload(w, precisions=BF)                 # built-in rule: the per-mode launches
    f = W.rhs(w).to(torch.complex64).cuda()
    ref = op.apply(f, tb.PREC_C64).clone()
    rule = op.apply(f, tb.PREC_C64_SPLITBF16).clone()
    bound = chain_bound(op)
    assert rel(rule, ref) < bound
    op.autotune(w.nv, tb.PREC_C64_SPLITBF16)                # per pass: tensor cores, fused or per-mode
    tuned = op.apply(f, tb.PREC_C64_SPLITBF16)
    assert rel(tuned, ref) < bound
    assert rel(op.apply_adjoint(f, tb.PREC_C64_SPLITBF16), op.apply_adjoint(f, tb.PREC_C64)) < bound
    op.close()

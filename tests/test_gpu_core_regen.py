"""Mid-level cores regenerated inside the contraction (tb_options.core_mode = 2)
against the stored cores and the step-by-step oracle.

Alg. 1 step 3 stores every core K(t-bar, s-bar) (the method's memory
bottleneck, Sec. 5); the one-RHS forward contraction can instead evaluate the
entries at the skeleton points as it goes.  On uniform grids the squared
distances of the Green's function (in grid units) and the phase x.xi of the
Radon kernel are exact integers, and the rest of the phase is carried as a
double-float, so the regenerated entries carry FP32 rounding only: the apply
must agree with the stored-core apply and with the FP64 step-by-step oracle to
complex64 rounding.  On a non-uniform grid regeneration does not apply and the
apply must be exactly the stored-core one.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import butterfly as O2
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


CASES = [
    ("helmholtz3d_n32", W.small("helmholtz3d_n64", 32, nv=1, L=2)),
    ("helmholtz3d_n64_L4", W.WORKLOADS["helmholtz3d_n64"]),
    ("plates2d_n64", W.small("plates2d_n64", 64, nv=1)),
    ("radon2d_n64", W.small("radon2d_n256", 64, nv=1, L=4)),
    ("radon2d_n256", W.WORKLOADS["radon2d_n256"]),
]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_regenerated_core_matches_stored_core(name, w):
    mask = (1 << tb.PREC_C64) | (1 << tb.PREC_C128)
    stored = tb.from_workload(w, precisions=mask, core_mode=tb.CORE_STORED)
    regen = tb.from_workload(w, precisions=mask, core_mode=tb.CORE_REGENERATE)
    f = W.rhs(w)
    x = f.to(torch.complex64).cuda()
    regen.profile(True)
    u_rg = regen.apply(x, tb.PREC_C64).cpu().to(torch.complex128).numpy()
    names = [s["name"] for s in regen.profile_stats()]
    regen.profile(False)
    u_st = stored.apply(x, tb.PREC_C64).cpu().to(torch.complex128).numpy()
    assert "core" in names
    assert rel(u_rg, u_st) < 2e-6, rel(u_rg, u_st)
    if w.N <= 64 ** 2 or name == "helmholtz3d_n32":
        bf = stored.export()
        u_o2 = O2.apply(bf, f.numpy())
        assert rel(u_rg, u_o2) < 3e-6
    rows = W.sample_targets(w, 1024, seed=4096)
    assert rel(u_rg.reshape(-1, 1)[rows], oracle.workload_apply(w, f, rows)) <= w.bound
    stored.close()
    regen.close()


def test_nonuniform_grid_keeps_the_stored_core():
    w = W.small("helmholtz3d_n64", 16, nv=1, L=2)
    xs, ys = W.grids(w)
    rng = np.random.default_rng(5)
    xs = [np.sort(x + 0.2 / 16 * rng.random(16)) for x in xs]
    a = tb.TBOperator(W.HELMHOLTZ, 3, [16] * 3, xs, ys, w.tol, params=w.params, L=2, core_mode=tb.CORE_STORED)
    b = tb.TBOperator(W.HELMHOLTZ, 3, [16] * 3, xs, ys, w.tol, params=w.params, L=2, core_mode=tb.CORE_REGENERATE)
    f = W.rhs(w).to(torch.complex64).cuda()
    assert torch.equal(a.apply(f, tb.PREC_C64), b.apply(f, tb.PREC_C64))
    a.close()
    b.close()

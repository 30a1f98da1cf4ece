"""GPU parity: the CUDA tensor butterfly (construction + apply, through the C
ABI) against the FP64 CPU oracle on the same seeded inputs.

Bars: the butterfly approximates K to the ID tolerance eps (Sec. 2.1,
Tables 2/3 report errors within a small factor of eps), so the relative L2
error against the direct sum must be <= 10 eps for the FP64 apply and within
each workload's stated bound for complex64.  The bit-reversed uniform Fourier
butterfly has exact ranks C_b (every block of Sec. 3.2.1's DFT example is a
rank-C_b DFT block), so it must match to rounding (1e-12 in FP64).
"""
import ctypes

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


def run(op, w, f, precision, rows=None, adjoint=False):
    dt = tb.dtype_of(precision)
    x = f.to(dt).cuda()
    y = (op.apply_adjoint(x, precision) if adjoint else op.apply(x, precision)).cpu().to(torch.complex128)
    y = y.numpy().reshape(-1, f.shape[-1])
    return y if rows is None else y[rows]


# --------------------------------------------------------------- small, exact
@pytest.mark.parametrize("separable", [0, 1])
@pytest.mark.parametrize("d,n,L", [(2, 16, 2), (2, 64, 4), (3, 16, 2), (1, 64, 4)])
def test_fourier_bitrev_is_exact(d, n, L, separable):
    w = W.Workload(name="f", kind=W.FOURIER, d=d, n=n, tol=1e-8, nv=2, precision=W.C128, bound=1e-12,
                   rhs_seeds=(0, 1), samples=0, order=W.ORDER_BITREV, L=L)
    op = tb.from_workload(w, separable=separable)
    info = op.info()
    assert info["rank_max"] == n >> L          # ranks are exactly C_b
    f = W.rhs(w)
    u = run(op, w, f, tb.PREC_C128)
    ref = oracle.fourier_fft(f.numpy(), d).reshape(-1, 2)
    assert rel(u, ref) < 1e-12
    v = run(op, w, f, tb.PREC_C128, adjoint=True)
    assert rel(v, oracle.workload_apply_adjoint(w, f)) < 1e-12
    u32 = run(op, w, f, tb.PREC_C64)
    assert rel(u32, ref) < 2e-6
    if separable == 0 and d > 1:
        # exact ranks: the butterfly itself is exact, so what remains is the
        # rounding of the split-BF16 core (two BF16 terms per value and per core
        # entry, about 16 bits, FP32 accumulation) plus the FP32 level passes
        # (the per-mode launches, so that the core is pinned on its own)
        op = tb.from_workload(w, separable=separable, level_schedule=tb.LEVEL_PER_MODE)
        ubf = run(op, w, f, tb.PREC_C64_SPLITBF16)
        assert rel(ubf, ref) < 5e-5, rel(ubf, ref)
        vbf = run(op, w, f, tb.PREC_C64_SPLITBF16, adjoint=True)
        assert rel(vbf, oracle.workload_apply_adjoint(w, f)) < 5e-5


@pytest.mark.parametrize("d,n,L,nv", [(4, 8, 2, 3), (6, 4, 2, 2)])
def test_separable_high_dimension_full_output(d, n, L, nv):
    w = W.Workload(name="f", kind=W.FOURIER, d=d, n=n, tol=1e-8, nv=nv, precision=W.C128, bound=1e-12,
                   rhs_seeds=tuple(range(nv)), samples=0, order=W.ORDER_BITREV, L=L)
    op = tb.from_workload(w)
    assert op.info()["separable"] == 1
    f = W.rhs(w)
    ref = oracle.fourier_fft(f.numpy(), d).reshape(-1, nv)
    assert rel(run(op, w, f, tb.PREC_C128), ref) < 1e-12
    assert rel(run(op, w, f, tb.PREC_C64), ref) < 1e-5
    assert rel(run(op, w, f, tb.PREC_C128, adjoint=True), oracle.workload_apply_adjoint(w, f)) < 1e-12


def test_config_fourier2d_n64_full_output():
    w = W.WORKLOADS["fourier2d_n64"]
    op = tb.from_workload(w)
    f = W.rhs(w)
    u = run(op, w, f, tb.PREC_C128)
    ref = oracle.workload_apply(w, f)
    assert rel(u, ref) <= w.bound
    assert rel(u, ref) < 1e-12


@pytest.mark.parametrize("prec,bound", [(tb.PREC_C128, 1e-5), (tb.PREC_C64, 2e-5)])
def test_helmholtz3d_small_full_output(prec, bound):
    w = W.small("helmholtz3d_n64", 16, nv=3, L=2)
    op = tb.from_workload(w)
    f = W.rhs(w)
    ref = oracle.workload_apply(w, f)
    assert rel(run(op, w, f, prec), ref) < bound
    refv = oracle.workload_apply_adjoint(w, f)
    assert rel(run(op, w, f, prec, adjoint=True), refv) < bound


@pytest.mark.parametrize("n,L", [(32, 2), (64, 4)])
def test_radon2d_small_full_output(n, L):
    w = W.small("radon2d_n256", n, nv=2, L=L)
    op = tb.from_workload(w)
    f = W.rhs(w)
    ref = oracle.workload_apply(w, f)
    assert rel(run(op, w, f, tb.PREC_C128), ref) < 10 * w.tol
    assert rel(run(op, w, f, tb.PREC_C64), ref) < 1e-4
    refv = oracle.workload_apply_adjoint(w, f)
    assert rel(run(op, w, f, tb.PREC_C128, adjoint=True), refv) < 10 * w.tol


def test_tucker_id_single_level_L0():
    # L = 0: the whole operator is one Tucker-ID (Sec. 3.1), error <= eps sqrt(2d)
    w = W.small("helmholtz3d_n64", 8, nv=1, L=0)
    op = tb.from_workload(w)
    f = W.rhs(w)
    assert rel(run(op, w, f, tb.PREC_C128), oracle.workload_apply(w, f)) < 10 * w.tol


def test_unequal_axis_sizes():
    xs = [np.arange(16) / 16, np.arange(32) / 32]
    ys = [np.arange(16) - 8.0, np.arange(32) - 16.0]
    op = tb.TBOperator(W.RADON, 2, [16, 32], xs, ys, 1e-7, params=(2 / 16, 1 / 16), L=2, precision=tb.PREC_C128)
    f = W.complex_gaussian((16, 32, 2), 9)
    u = op.apply(f.cuda()).cpu().numpy().reshape(-1, 2)
    assert rel(u, oracle.apply(W.RADON, (2 / 16, 1 / 16), xs, ys, f)) < 1e-6


def test_ragged_rhs_chunks_and_adjoint_identity():
    w = W.small("radon2d_n256", 64, nv=5, L=4)
    op = tb.from_workload(w)
    f = W.complex_gaussian((64, 64, 5), 3)
    g = W.complex_gaussian((64, 64, 5), 4)
    for prec, tol in ((tb.PREC_C128, 1e-12), (tb.PREC_C64, 1e-5)):
        dt = tb.dtype_of(prec)
        Kf = op.apply(f.to(dt).cuda(), prec).cpu().to(torch.complex128)
        KHg = op.apply_adjoint(g.to(dt).cuda(), prec).cpu().to(torch.complex128)
        lhs = torch.vdot(g.reshape(-1), Kf.reshape(-1))
        rhs = torch.vdot(KHg.reshape(-1), f.reshape(-1))
        assert abs(lhs - rhs) <= tol * abs(lhs)
        # each RHS column alone gives the same column
        one = op.apply(f[..., 2:3].contiguous().to(dt).cuda(), prec).cpu().to(torch.complex128)
        assert rel(one, Kf[..., 2:3]) < (1e-14 if prec == tb.PREC_C128 else 1e-6)


def test_deterministic_and_graph_replay():
    w = W.small("helmholtz3d_n64", 16, nv=4, L=2)
    op = tb.from_workload(w, use_graphs=True)
    f = W.rhs(w).to(torch.complex64).cuda()
    out = torch.empty_like(f)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = op.apply(f, tb.PREC_C64).clone()
        for _ in range(3):
            op.apply(f, tb.PREC_C64, out=out)      # first eager + capture, then replays
    s.synchronize()
    b = op.apply(f, tb.PREC_C64)                   # default stream: eager
    assert torch.equal(a, out) and torch.equal(a, b)


def test_error_paths():
    w = W.small("helmholtz3d_n64", 8, nv=1, L=0)
    op = tb.from_workload(w, precisions=1 << tb.PREC_C128)
    f = W.rhs(w).cuda()
    with pytest.raises(tb.TBError) as e:
        op.apply(f.to(torch.complex64), tb.PREC_C64)
    assert e.value.status == 6                       # precision not built
    L = tb.lib()
    with pytest.raises(tb.TBError) as e:             # overlapping input/output
        tb._check(L.tb_apply(op._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()), 1, 0, None))
    assert e.value.status == 1
    host = np.zeros(f.numel() * 2)
    with pytest.raises(tb.TBError) as e:             # host pointer where device memory is required
        tb._check(L.tb_apply(op._h, ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(f.data_ptr()), 1, 0, None))
    assert e.value.status == 1
    # rank cap too small for the tolerance
    with pytest.raises(tb.TBError) as e:
        tb.from_workload(W.small("radon2d_n256", 32, L=2), rank_max=2)
    assert e.value.status == 4
    # coincident Helmholtz points
    xs = [np.arange(8) / 8] * 3
    with pytest.raises(tb.TBError) as e:
        tb.TBOperator(W.HELMHOLTZ, 3, [8] * 3, xs, xs, 1e-6, params=(10.0,), L=0)
    assert e.value.status == 1


def test_apply_host_matches_device():
    w = W.small("radon2d_n256", 32, nv=2, L=2)
    op = tb.from_workload(w)
    f = W.rhs(w)
    dev = run(op, w, f, tb.PREC_C64)
    host = op.apply_host(f.numpy().astype(np.complex64), tb.PREC_C64).reshape(-1, 2)
    assert np.array_equal(host, dev.astype(np.complex64))


# ---------------------------------------------- split-BF16 tensor-core core
@pytest.mark.parametrize("nv", [16, 5, 20])
def test_splitbf16_core_matches_c64_and_oracle(nv):
    # two-term split BF16 with FP32 accumulation keeps ~16 mantissa bits per
    # product: the apply must agree with the complex64 apply to ~1e-5 and stay
    # within the workload bound (1e-3 at eps = 1e-4) against the oracle
    # 4 points per wavelength, as in the n = 256 workload
    w = W.small("helmholtz3d_n256", 32, nv=nv, L=2, params=(2 * np.pi * 8,))
    op = tb.from_workload(w, precisions=(1 << tb.PREC_C64) | (1 << tb.PREC_C64_SPLITBF16),
                          level_schedule=tb.LEVEL_PER_MODE)
    f = W.rhs(w)
    u32 = run(op, w, f, tb.PREC_C64)
    ubf = run(op, w, f, tb.PREC_C64_SPLITBF16)
    assert rel(ubf, u32) < 1e-4
    ref = oracle.workload_apply(w, f)
    assert rel(ubf, ref) <= w.bound
    v32 = run(op, w, f, tb.PREC_C64, adjoint=True)
    vbf = run(op, w, f, tb.PREC_C64_SPLITBF16, adjoint=True)
    assert rel(vbf, v32) < 1e-4
    assert rel(vbf, oracle.workload_apply_adjoint(w, f)) <= w.bound


def test_splitbf16_core_multilevel_and_deterministic():
    w = W.small("helmholtz3d_n256", 64, nv=16, L=4, params=(2 * np.pi * 16,))
    op = tb.from_workload(w, precisions=(1 << tb.PREC_C64) | (1 << tb.PREC_C64_SPLITBF16),
                          level_schedule=tb.LEVEL_PER_MODE)
    f = W.rhs(w)
    rows = W.sample_targets(w, 512)
    ubf = run(op, w, f, tb.PREC_C64_SPLITBF16)
    assert rel(ubf, run(op, w, f, tb.PREC_C64)) < 1e-4
    assert rel(ubf[rows], oracle.workload_apply(w, f, rows)) <= w.bound
    again = run(op, w, f, tb.PREC_C64_SPLITBF16)
    assert np.array_equal(ubf, again)


def test_splitbf16_core_output_keeps_zero_padding_across_rhs_counts():
    # the split-BF16 core writes a buffer of its own whose padded entries keep the
    # zeros of its allocation (the core writes only compact entries); a change of
    # nv re-lays that buffer out and must clear it again.  RHS columns are
    # independent, so 5 RHS give exactly the first 5 columns of 16.
    w = W.small("helmholtz3d_n256", 32, nv=16, L=2, params=(2 * np.pi * 8,))
    op = tb.from_workload(w, precisions=(1 << tb.PREC_C64) | (1 << tb.PREC_C64_SPLITBF16),
                          level_schedule=tb.LEVEL_PER_MODE)
    f16 = W.rhs(w).to(torch.complex64).cuda()
    f5 = f16[..., :5].contiguous()
    for adj in (False, True):
        run = (lambda x, p: op.apply_adjoint(x, p)) if adj else (lambda x, p: op.apply(x, p))
        a = run(f16, tb.PREC_C64_SPLITBF16).clone()
        b = run(f5, tb.PREC_C64_SPLITBF16).clone()
        c = run(f16, tb.PREC_C64_SPLITBF16).clone()
        assert torch.equal(b, a[..., :5]), adj
        assert torch.equal(a, c), adj
        ref = run(f16, tb.PREC_C64).cpu().to(torch.complex128).numpy()
        assert rel(a.cpu().to(torch.complex128).numpy(), ref) < 1e-4
    op.close()


# ------------------------------------------- register-resident separable chains
@pytest.mark.parametrize("d,n,nv,precs", [(3, 16, 3, (tb.PREC_C64,)), (4, 8, 2, (tb.PREC_C64, tb.PREC_C128)),
                                          (2, 32, 4, (tb.PREC_C64,)), (6, 4, 5, (tb.PREC_C64, tb.PREC_C128))])
def test_separable_register_chains_match_shared_memory_fibers(d, n, nv, precs):
    """With ranks equal to the leaf size (bit-reversed uniform Fourier, L = 2) the
    register-resident chains (per mode with paired or scalar FMAs and one or
    two fibers per thread, and fused in pairs of modes) apply the same steps as the shared-memory fiber
    passes: all agree to rounding, and with the DFT identity."""
    w = W.Workload(name="f", kind=W.FOURIER, d=d, n=n, tol=1e-8, nv=nv, precision=W.C64, bound=1e-5,
                   rhs_seeds=tuple(range(nv)), samples=0, order=W.ORDER_BITREV, L=2)
    f = W.rhs(w)
    ref = oracle.fourier_fft(f.numpy(), d).reshape(-1, nv)
    refv = oracle.workload_apply_adjoint(w, f)
    schedules = (tb.SEP_FIBER, tb.SEP_REGISTER, tb.SEP_REGISTER_PAIRS, tb.SEP_REGISTER_SCALAR, tb.SEP_REGISTER_ONE)
    ops = {s: tb.from_workload(w, sep_schedule=s) for s in schedules}
    for prec in precs:
        out = {}
        for s, op in ops.items():
            op.profile(True)
            out[s] = (run(op, w, f, prec), run(op, w, f, prec, adjoint=True))
            names = {r["name"] for r in op.profile_stats()}
            op.profile(False)
            assert ("sep_reg" in names) == (s in (tb.SEP_REGISTER, tb.SEP_REGISTER_SCALAR, tb.SEP_REGISTER_ONE)
                                            or (s == tb.SEP_REGISTER_PAIRS and d % 2 == 1)), names
            assert ("sep_reg2" in names) == (s == tb.SEP_REGISTER_PAIRS), names
        tight = 1e-12 if prec == tb.PREC_C128 else 2e-6
        for s in out:
            assert rel(out[s][0], ref) < tight, s
            assert rel(out[s][1], refv) < tight, s
            assert rel(out[s][0], out[tb.SEP_FIBER][0]) < tight, s
            assert rel(out[s][1], out[tb.SEP_FIBER][1]) < tight, s
    for op in ops.values():
        op.close()


# ------------------------------------------- the paper's other kernel families
@pytest.mark.parametrize("name", ["plates2d_n64", "radon2d_aniso_n64", "radon3d_n32", "nudft3d_n16"])
def test_other_paper_kernels(name):
    """Parallel plates (Sec. 4.1), anisotropic 2-D and 3-D Radon (Sec. 4.2) and
    the type-2 non-uniform DFT (Sec. 4.3): the butterfly's error against the
    direct sum stays within 10 eps in FP64 and within the bound in complex64,
    forward and adjoint (complex64: FP32 rounding, bound 1e-5)."""
    w = W.WORKLOADS[name]
    op = tb.from_workload(w, precisions=(1 << tb.PREC_C64) | (1 << tb.PREC_C128))
    info = op.info()
    assert info["separable"] == (1 if w.kind == W.FOURIER else 0)
    f = W.rhs(w)
    rows = W.sample_targets(w) if w.samples else None
    ref = oracle.workload_apply(w, f, rows)
    refv = oracle.workload_apply_adjoint(w, f, rows)
    for prec, bound in ((tb.PREC_C128, 10 * w.tol), (tb.PREC_C64, max(w.bound, 10 * w.tol, 1e-5))):
        assert rel(run(op, w, f, prec, rows), ref) < bound, prec
        assert rel(run(op, w, f, prec, rows, adjoint=True), refv) < bound, prec
    op.close()


@pytest.mark.parametrize("count", [1, 2, 5])
def test_host_batch_equals_device_applies(count):
    """tb_apply_host_batch (pinned host buffers, copies overlapping the applies
    on three streams, two device buffer pairs reused) returns exactly what
    tb_apply returns for each input."""
    w = W.small("helmholtz3d_n64", 16, nv=2, L=2)
    op = tb.from_workload(w, precisions=1 << tb.PREC_C64, use_graphs=True)
    fs = [W.complex_gaussian((16, 16, 16, 2), 100 + i).to(torch.complex64).pin_memory().numpy() for i in range(count)]
    us = [torch.empty((16, 16, 16, 2), dtype=torch.complex64).pin_memory().numpy() for _ in range(count)]
    op.apply_host_batch(fs, us, tb.PREC_C64)
    for f, u in zip(fs, us):
        ref = op.apply(torch.from_numpy(f).cuda(), tb.PREC_C64).cpu().numpy()
        assert np.array_equal(u, ref)
    op.close()

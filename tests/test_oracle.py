"""Pins for the CPU oracle (no GPU).

The oracle is the plain direct sum u = K f, v = K^H g (contraction of Alg. 2,
Sec. 3.2).  These tests tie it to things other than itself: the DFT identity
(Sec. 3.2.1, DFT paragraph), hand-derived kernel values (tests/golden), brute
force with an independent numpy kernel matrix, the adjoint identity, Green's
function reciprocity and delta inputs.  A dropped term, a wrong sign or index
or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kernel_values.txt")


def _grid(kind, d, n, off=0.0):
    x = [np.arange(n) / n for _ in range(d)]
    if kind == W.HELMHOLTZ:
        y = [np.arange(n) / n + (off if k == 0 else 0.0) for k in range(d)]
    else:
        y = [np.arange(n) - n / 2 for _ in range(d)]
    return x, y


def _rand(shape, seed):
    return W.complex_gaussian(shape, seed).numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_golden_kernel_values():
    rows = 0
    with open(GOLDEN) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            kind, par, x, y, re, im, _ = [s.strip() for s in line.split("|", 6)]
            params = [] if par == "-" else [float(p) for p in par.split()]
            x = [float(v) for v in x.split()]
            y = [float(v) for v in y.split()]
            got = oracle.kernel_entry(int(kind), params, x, y)
            assert abs(got - complex(float(re), float(im))) < 1e-12, line
            rows += 1
    assert rows >= 10


@pytest.mark.parametrize("d,n,nv", [(1, 16, 3), (2, 8, 2), (3, 8, 1), (6, 4, 1)])
def test_fourier_direct_sum_is_dft(d, n, nv):
    xs, ys = _grid(W.FOURIER, d, n)
    f = _rand((n,) * d + (nv,), 3 + d)
    u = oracle.apply(W.FOURIER, (), xs, ys, f).reshape(f.shape)
    ref = oracle.fourier_fft(f, d, sign=-1)
    assert _rel(u, ref) < 1e-12


@pytest.mark.parametrize("d,n,nv", [(1, 16, 2), (2, 8, 3), (3, 4, 1), (6, 4, 2)])
def test_fourier_adjoint_direct_sum_is_inverse_dft(d, n, nv):
    # v = K^H g with the sign of the DFT identity on the summed index
    xs, ys = _grid(W.FOURIER, d, n)
    g = _rand((n,) * d + (nv,), 40 + d)
    v = oracle.apply_adjoint(W.FOURIER, (), xs, ys, g).reshape(g.shape)
    assert _rel(v, oracle.fourier_fft_adjoint(g, d)) < 1e-12


def test_fourier_fft_adjoint_against_explicit_loops():
    # v[j] = sum_i exp(+2 pi i (i/n)(j - n/2)) g[i] for d = 1
    n = 10
    g = _rand((n, 1), 6)
    v = oracle.fourier_fft_adjoint(g, 1)
    ref = np.array([sum(np.exp(2j * math.pi * (i / n) * (j - n / 2)) * g[i, 0] for i in range(n))
                    for j in range(n)])
    assert _rel(v[:, 0], ref) < 1e-13


def test_fourier_fft_against_numpy_definition():
    # u[i] = sum_j exp(-2 pi i (i/n)(j - n/2)) f[j] for d = 1, by explicit loops
    n = 12
    f = _rand((n, 1), 5)
    u = oracle.fourier_fft(f, 1, sign=-1)
    ref = np.array([sum(np.exp(-2j * math.pi * (i / n) * (j - n / 2)) * f[j, 0] for j in range(n))
                    for i in range(n)])
    assert _rel(u[:, 0], ref) < 1e-13


@pytest.mark.parametrize("d,n", [(2, 8), (2, 16)])
def test_radon_zero_phase_is_inverse_dft(d, n):
    xs, ys = _grid(W.RADON, d, n)
    f = _rand((n,) * d + (2,), 11)
    u = oracle.apply(W.RADON, (0.0, 0.0), xs, ys, f).reshape(f.shape)
    assert _rel(u, oracle.fourier_fft(f, d, sign=+1)) < 1e-12


def test_radon_constant_c_is_modulated_inverse_dft():
    # b = 0: K = exp(2 pi i x.xi) exp(2 pi i a |xi|), a radial modulation of the input
    d, n, a = 2, 16, 0.3
    xs, ys = _grid(W.RADON, d, n)
    f = _rand((n,) * d + (1,), 12)
    Y = np.stack(np.meshgrid(*ys, indexing="ij"), -1)
    mod = np.exp(2j * math.pi * a * np.sqrt((Y ** 2).sum(-1)))[..., None]
    u = oracle.apply(W.RADON, (a, 0.0), xs, ys, f).reshape(f.shape)
    assert _rel(u, oracle.fourier_fft(f * mod, d, sign=+1)) < 1e-12


@pytest.mark.parametrize("kind,params,d,n", [
    (W.FOURIER, (), 2, 8), (W.HELMHOLTZ, (2 * math.pi * 3,), 3, 4),
    (W.RADON, (2 / 16, 1 / 16), 2, 8), (W.RADON, (3 / 100, 1 / 100), 3, 4),
    (W.HELMHOLTZ, (2 * math.pi * 3, 0.7), 2, 6), (W.RADON_ANISO, (2 / 16, 1 / 16, 2 / 16, 1 / 16), 2, 8)])
def test_direct_sum_matches_dense_bruteforce(kind, params, d, n):
    xs, ys = _grid(kind, d, n, off=2.0)
    f = _rand((n,) * d + (2,), 21)
    K = oracle.dense_matrix(kind, params, xs, ys)
    ref = K @ f.reshape(-1, 2)
    u = oracle.apply(kind, params, xs, ys, f)
    assert _rel(u, ref) < 1e-13
    g = _rand((n,) * d + (2,), 22)
    v = oracle.apply_adjoint(kind, params, xs, ys, g)
    assert _rel(v, K.conj().T @ g.reshape(-1, 2)) < 1e-13


@pytest.mark.parametrize("kind,params,d,n", [
    (W.FOURIER, (), 2, 8), (W.HELMHOLTZ, (2 * math.pi * 4,), 3, 6), (W.RADON, (2 / 16, 1 / 16), 2, 10),
    (W.HELMHOLTZ, (2 * math.pi * 4, 1.0), 2, 9), (W.RADON_ANISO, (2 / 16, 1 / 16, 2 / 16, 1 / 16), 2, 10)])
def test_adjoint_identity(kind, params, d, n):
    xs, ys = _grid(kind, d, n, off=2.0)
    f = _rand((n,) * d + (1,), 31)
    g = _rand((n,) * d + (1,), 32)
    Kf = oracle.apply(kind, params, xs, ys, f)
    KHg = oracle.apply_adjoint(kind, params, xs, ys, g)
    lhs = np.vdot(g.reshape(-1), Kf.reshape(-1))       # <g, K f>
    rhs = np.vdot(KHg.reshape(-1), f.reshape(-1))      # <K^H g, f>
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs) + 1e-12


def test_helmholtz_reciprocity():
    # K(x, y) = K(y, x): swapping the cubes gives K^T, so K_swap f = conj(K^H conj f)
    d, n, kappa = 3, 5, 2 * math.pi * 3
    xs, ys = _grid(W.HELMHOLTZ, d, n, off=2.0)
    f = _rand((n,) * d + (1,), 41)
    u_swap = oracle.apply(W.HELMHOLTZ, (kappa,), ys, xs, f)
    v = oracle.apply_adjoint(W.HELMHOLTZ, (kappa,), xs, ys, f.conj())
    assert _rel(u_swap, v.conj()) < 1e-13


@pytest.mark.parametrize("kind,params", [(W.FOURIER, ()), (W.HELMHOLTZ, (2 * math.pi * 2,)),
                                         (W.RADON, (2 / 16, 1 / 16))])
def test_delta_input_returns_kernel_column(kind, params):
    d, n = 2, 6
    xs, ys = _grid(kind, d, n, off=2.0)
    j = (4, 1)
    f = np.zeros((n, n, 1), dtype=np.complex128)
    f[j + (0,)] = 1.0
    u = oracle.apply(kind, params, xs, ys, f)[:, 0]
    col = [oracle.kernel_entry(kind, params, [xs[0][a], xs[1][b]], [ys[0][j[0]], ys[1][j[1]]])
           for a in range(n) for b in range(n)]
    assert np.allclose(u, col, rtol=0, atol=1e-14)


def test_plates_offset_is_a_third_axis():
    # d = 2 grids at perpendicular distance h (Sec. 4.1 plates) = the 3-D kernel on
    # grids with a one-point third axis: x_3 = 0, y_3 = h
    n, kappa, h = 7, 2 * math.pi * 3, 1.0
    xs, ys = _grid(W.HELMHOLTZ, 2, n, off=0.0)
    f = _rand((n, n, 2), 61)
    u2 = oracle.apply(W.HELMHOLTZ, (kappa, h), xs, ys, f)
    u3 = oracle.apply(W.HELMHOLTZ, (kappa,), xs + [np.zeros(1)], ys + [np.full(1, h)], f.reshape(n, n, 1, 2))
    assert _rel(u2, u3) < 1e-14


def test_anisotropic_radon_with_equal_constant_speeds_is_isotropic():
    # b1 = b2 = 0 and a1 = a2 = a: sqrt(a^2 xi_1^2 + a^2 xi_2^2) = a |xi| (Eq. randon2d -> randon3d form)
    n, a = 12, 0.2
    xs, ys = _grid(W.RADON, 2, n)
    f = _rand((n, n, 2), 62)
    ua = oracle.apply(W.RADON_ANISO, (a, 0.0, a, 0.0), xs, ys, f)
    ui = oracle.apply(W.RADON, (a, 0.0), xs, ys, f)
    assert _rel(ua, ui) < 1e-13
    # and the speeds act per axis: c2 alone modulates xi_2 only
    ub = oracle.apply(W.RADON_ANISO, (0.0, 0.0, a, 0.0), xs, ys, f).reshape(f.shape)
    Y = np.stack(np.meshgrid(*ys, indexing="ij"), -1)
    mod = np.exp(2j * math.pi * a * np.abs(Y[..., 1]))[..., None]
    assert _rel(ub, oracle.fourier_fft(f * mod, 2, sign=+1)) < 1e-12


def test_nonuniform_fourier_is_a_product_of_1d_transforms():
    # type-2 non-uniform DFT (Sec. 4.3): the kernel is separable, so u is f
    # contracted with one 1-D matrix exp(-2 pi i x_k y_k) per axis
    w = W.WORKLOADS["nudft3d_n16"]
    w = W.Workload(**{**w.__dict__, "n": 6, "nv": 2})
    xs, ys = W.grids(w)
    assert all(np.all(np.diff(x) > 0) and x[0] >= 0 and x[-1] < 1 for x in xs)
    f = _rand((6, 6, 6, 2), 63)
    M = [np.exp(-2j * math.pi * np.outer(xs[k], ys[k])) for k in range(3)]
    ref = np.einsum("ai,bj,ck,ijkv->abcv", M[0], M[1], M[2], f).reshape(-1, 2)
    assert _rel(oracle.apply(W.FOURIER, (), xs, ys, f), ref) < 1e-13


def test_sampled_rows_match_full_output():
    w = W.small("helmholtz3d_n64", 8)
    f = W.rhs(w, nv=2).numpy()
    full = oracle.workload_apply(w, f)
    rows = W.sample_targets(w, 37)
    assert len(np.unique(rows)) == 37
    assert np.array_equal(oracle.workload_apply(w, f, rows), full[rows])
    cols = W.sample_targets(w, 11, seed=7)
    fullv = oracle.workload_apply_adjoint(w, f)
    assert np.array_equal(oracle.workload_apply_adjoint(w, f, cols), fullv[cols])


def test_rhs_columns_are_independent():
    # each RHS column is transformed on its own (no cross-talk between columns)
    w = W.small("radon2d_n256", 8)
    xs, ys = W.grids(w)
    f = _rand((8, 8, 3), 51)
    u = oracle.apply(w.kind, w.params, xs, ys, f)
    for v in range(3):
        uv = oracle.apply(w.kind, w.params, xs, ys, f[..., v:v + 1])
        assert np.array_equal(u[:, v:v + 1], uv)


def test_workload_definitions():
    assert set(W.WORKLOADS) == {"fourier2d_n64", "helmholtz3d_n64", "helmholtz3d_n256",
                                "radon2d_n256", "fourier6d_n16", "plates2d_n64", "radon2d_aniso_n64",
                                "radon3d_n32", "nudft3d_n16"}
    w = W.WORKLOADS["helmholtz3d_n256"]
    xs, ys = W.grids(w)
    assert ys[0][0] == 2.0 and ys[1][0] == 0.0 and xs[2][-1] == 255 / 256
    f = W.rhs(W.small("helmholtz3d_n256", 8, nv=4))
    assert f.shape == (8, 8, 8, 4) and f.dtype.is_complex
    # RHS v is drawn from seed v
    assert np.array_equal(f[..., 2].numpy(), W.complex_gaussian((8, 8, 8), 2).numpy())
    b = W.smooth_bumps(W.WORKLOADS["radon2d_n256"])
    assert b.shape == (256, 256, 1)


def test_kernel_pairs_is_the_diagonal_of_kernel_matrix():
    rng = np.random.default_rng(8)
    X, Y = rng.random((7, 3)), rng.random((7, 3)) + 2.0
    for kind, params in ((W.FOURIER, ()), (W.HELMHOLTZ, (5.0, 0.3)), (W.RADON, (0.1, 0.05))):
        K = oracle.kernel_matrix(kind, params, X, Y)
        assert np.allclose(oracle.kernel_pairs(kind, params, X, Y), np.diag(K), rtol=0, atol=1e-14)

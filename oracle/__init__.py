"""CPU oracle for the tensor butterfly apply.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the CPU
baseline of bench.py may import this package.  It shares no code with the CUDA
library (paper_2411_03029_gb300) and never imports it.

Contents
  * direct_sum.c  -- plain FP64 direct summation u = K f and v = K^H g on
    selected outputs (the definition of the contraction in Alg. 2, Sec. 3.2).
  * fourier_fft   -- the same operator for the Fourier kernel on the uniform
    grids x = i/n, y = j - n/2, written as the textbook DFT identity
    u = (-1)^(i_1+...+i_d) * fftn(f) (Sec. 3.2.1, DFT paragraph: the d-D DFT is
    a product of 1-D DFTs); a library FFT is the only step.
  * fourier_fft_adjoint -- the adjoint K^H g of the same operator by the same
    identity, v = n^d ifftn((-1)^(i_1+...+i_d) g).
  * dense_matrix  -- the full kernel matrix for tiny grids (numpy), used only
    as a brute-force cross-check of the direct sum; kernel_matrix, the same
    formulas at arbitrary point sets.
  * butterfly     -- the tensor butterfly applied step by step from exported
    factors (Alg. 2 and Eq. butterfly_tensor), for checking the GPU apply to
    rounding; see oracle/butterfly.py.

Every function here is pinned by tests/test_oracle.py against closed forms,
hand-derived special values (tests/golden/), symmetry identities and brute
force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "direct_sum.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile direct_sum.c into a shared library (gcc, OpenMP, IEEE FP64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.tbo_apply.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, I64, P, I64, P]
        lib.tbo_apply_adjoint.argtypes = lib.tbo_apply.argtypes
        lib.tbo_kernel_entry.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P]
        lib.tbo_max_threads.argtypes = []
        for fn in (lib.tbo_apply, lib.tbo_apply_adjoint, lib.tbo_kernel_entry, lib.tbo_max_threads):
            fn.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the direct sum uses."""
    return int(_load().tbo_max_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _prep(kind, params, xs, ys):
    par = np.zeros(4, dtype=np.float64)
    par[: len(params)] = params
    m = np.array([len(x) for x in xs], dtype=np.int64)
    n = np.array([len(y) for y in ys], dtype=np.int64)
    xc = np.ascontiguousarray(np.concatenate(xs).astype(np.float64))
    yc = np.ascontiguousarray(np.concatenate(ys).astype(np.float64))
    return par, m, n, xc, yc


def _as_c128(a) -> np.ndarray:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            a = a.detach().cpu().numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def apply(kind, params, xs, ys, f, rows=None) -> np.ndarray:
    """u[rows] = sum_j K(x^rows, y^j) f_j.  f: (n_1..n_d, nv) complex.

    Returns an array of shape (len(rows), nv) (rows = all targets if None)."""
    lib = _load()
    par, m, n, xc, yc = _prep(kind, params, xs, ys)
    f = _as_c128(f)
    d = len(xs)
    nv = f.shape[-1] if f.ndim == d + 1 else 1
    assert f.size == int(np.prod(n)) * nv
    rows = np.arange(int(np.prod(m)), dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros((len(rows), nv), dtype=np.complex128)
    rc = lib.tbo_apply(int(kind), _ptr(par), d, _ptr(m), _ptr(xc), _ptr(n), _ptr(yc), _ptr(f), nv,
                       _ptr(rows), len(rows), _ptr(out))
    if rc != 0:
        raise ValueError("tbo_apply rejected its arguments")
    return out


def apply_adjoint(kind, params, xs, ys, g, cols=None) -> np.ndarray:
    """v[cols] = sum_i conj(K(x^i, y^cols)) g_i.  g: (m_1..m_d, nv) complex."""
    lib = _load()
    par, m, n, xc, yc = _prep(kind, params, xs, ys)
    g = _as_c128(g)
    d = len(xs)
    nv = g.shape[-1] if g.ndim == d + 1 else 1
    assert g.size == int(np.prod(m)) * nv
    cols = np.arange(int(np.prod(n)), dtype=np.int64) if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
    out = np.zeros((len(cols), nv), dtype=np.complex128)
    rc = lib.tbo_apply_adjoint(int(kind), _ptr(par), d, _ptr(m), _ptr(xc), _ptr(n), _ptr(yc), _ptr(g), nv,
                               _ptr(cols), len(cols), _ptr(out))
    if rc != 0:
        raise ValueError("tbo_apply_adjoint rejected its arguments")
    return out


def kernel_entry(kind, params, x, y) -> complex:
    """One kernel value K(x, y) at points x, y in R^d."""
    lib = _load()
    par = np.zeros(4, dtype=np.float64)
    par[: len(params)] = params
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(2, dtype=np.float64)
    if lib.tbo_kernel_entry(int(kind), _ptr(par), len(x), _ptr(x), _ptr(y), _ptr(out)) != 0:
        raise ValueError("bad dimension")
    return complex(out[0], out[1])


def workload_apply(w, f, rows=None) -> np.ndarray:
    """Direct sum for a workloads.Workload (its grids and kernel parameters)."""
    import workloads
    xs, ys = workloads.grids(w)
    return apply(w.kind, w.params, xs, ys, f, rows)


def workload_apply_adjoint(w, g, cols=None) -> np.ndarray:
    import workloads
    xs, ys = workloads.grids(w)
    return apply_adjoint(w.kind, w.params, xs, ys, g, cols)


def fourier_fft(f, d: int, sign: int = -1) -> np.ndarray:
    """Full output of the Fourier kernel exp(sign 2 pi i x.y) on the uniform grids
    x_k = i/n, y_k = j - n/2 (n even), via the DFT identity.

    exp(-2 pi i (i/n)(j - n/2)) = exp(-2 pi i ij/n) (-1)^i, so
    u = (-1)^(sum_k i_k) * fftn(f) for sign=-1 and u = (-1)^(sum i) n^d ifftn(f)
    for sign=+1, transforming the d leading axes of f (n_1..n_d, nv)."""
    f = _as_c128(f)
    axes = tuple(range(d))
    if sign < 0:
        u = np.fft.fftn(f, axes=axes)
    else:
        u = np.fft.ifftn(f, axes=axes) * np.prod([f.shape[a] for a in axes])
    par = np.zeros(f.shape[:d], dtype=np.int64)
    for k in range(d):
        sh = [1] * d
        sh[k] = f.shape[k]
        par = par + np.arange(f.shape[k]).reshape(sh)
    s = np.where(par % 2 == 0, 1.0, -1.0)
    return u * s[..., None] if f.ndim == d + 1 else u * s


def fourier_fft_adjoint(g, d: int) -> np.ndarray:
    """Full adjoint output v = K^H g of the Fourier kernel exp(-2 pi i x.y) on the
    uniform grids x_k = i/n, y_k = j - n/2 (n even), via the DFT identity.

    conj(K[i, j]) = exp(+2 pi i ij/n) (-1)^i, so the sign now sits on the
    summed (target) index: v = n^d ifftn((-1)^(sum_k i_k) g) over the d leading
    axes of g (m_1..m_d, nv)."""
    g = _as_c128(g)
    axes = tuple(range(d))
    par = np.zeros(g.shape[:d], dtype=np.int64)
    for k in range(d):
        sh = [1] * d
        sh[k] = g.shape[k]
        par = par + np.arange(g.shape[k]).reshape(sh)
    s = np.where(par % 2 == 0, 1.0, -1.0)
    gs = g * s[..., None] if g.ndim == d + 1 else g * s
    return np.fft.ifftn(gs, axes=axes) * np.prod([g.shape[a] for a in axes])


def dense_matrix(kind, params, xs, ys) -> np.ndarray:
    """Full kernel matrix K[i, j] (C-order flattening) for tiny grids, in numpy."""
    d = len(xs)
    X = np.stack(np.meshgrid(*xs, indexing="ij"), -1).reshape(-1, d)
    Y = np.stack(np.meshgrid(*ys, indexing="ij"), -1).reshape(-1, d)
    return kernel_matrix(kind, params, X, Y)


def kernel_matrix(kind, params, X, Y) -> np.ndarray:
    """K[i, j] = K(X[i], Y[j]) for point arrays X (m x d) and Y (n x d), in numpy."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return _kernel(kind, params, X[:, None, :], Y[None, :, :])


def kernel_pairs(kind, params, X, Y) -> np.ndarray:
    """K(X[i], Y[i]) for point arrays X, Y of the same shape (... x d), in numpy."""
    return _kernel(kind, params, np.asarray(X, dtype=np.float64), np.asarray(Y, dtype=np.float64))


def _kernel(kind, params, Xe, Ye) -> np.ndarray:
    """The kernel formulas on broadcast point arrays (last axis = the d coordinates)."""
    if kind == 1:
        return np.exp(-2j * np.pi * (Xe * Ye).sum(-1))
    if kind == 2:
        h = params[1] if len(params) > 1 else 0.0
        rho = np.sqrt(((Xe - Ye) ** 2).sum(-1) + h * h)
        return np.exp(1j * params[0] * rho) / rho
    if kind == 3:
        c = params[0] + params[1] * np.prod(np.sin(2 * np.pi * Xe), axis=-1)
        return np.exp(2j * np.pi * ((Xe * Ye).sum(-1) + c * np.sqrt((Ye ** 2).sum(-1))))
    if kind == 4:
        a1, b1, a2, b2 = params
        s = np.sin(2 * np.pi * Xe)
        c = np.cos(2 * np.pi * Xe)
        c1 = a1 + b1 * s[..., 0] * s[..., 1]
        c2 = a2 + b2 * c[..., 0] * c[..., 1]
        phi = (Xe * Ye).sum(-1) + np.sqrt((c1 * Ye[..., 0]) ** 2 + (c2 * Ye[..., 1]) ** 2)
        return np.exp(2j * np.pi * phi)
    raise ValueError(kind)

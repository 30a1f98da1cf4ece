"""Seeded synthetic workloads for the tensor butterfly apply.

This module is shared by the tests, the benchmark and the CPU oracle, and it
holds none of the method's arithmetic: only grid coordinates, kernel
parameters, seeded right-hand sides and seeded sample sets.  Kernel formulas
live separately in the oracle (plain C) and in the CUDA library.

The workloads follow the paper's numerical examples (Sec. 4): uniform
DFTs (Sec. 4.3), Green's functions of the Helmholtz equation between two
separated unit cubes (Sec. 4.1) and a 2-D generalized Radon transform
(Sec. 4.2), with the sizes, tolerances and precisions of the benchmark
configurations; plus, at test sizes, the parallel plates of Sec. 4.1, the
anisotropic 2-D and the 3-D Radon transforms of Sec. 4.2 and the type-2
non-uniform DFT of Sec. 4.3.  The paper evaluates on analytic kernels only, so these
synthetic inputs are the paper's workload shapes; no dataset is involved.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

# kernel kinds (same numbering as include/tb.h: TB_KERNEL_*)
FOURIER = 1      # K(x, y) = exp(-2 pi i x.y)
HELMHOLTZ = 2    # K(x, y) = exp(i kappa |x - y|) / |x - y|
RADON = 3        # K(x, xi) = exp(2 pi i (x.xi + c(x) |xi|)),  c(x) = a + b prod_k sin(2 pi x_k)
RADON_ANISO = 4  # d = 2: K(x, xi) = exp(2 pi i (x.xi + sqrt(c1^2 xi_1^2 + c2^2 xi_2^2)))

# apply precisions (include/tb.h: TB_PREC_*)
C128 = 0
C64 = 1
C64_SPLITBF16 = 2

ORDER_NATURAL = 0
ORDER_BITREV = 1


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    kind: int
    d: int
    n: int
    tol: float
    nv: int
    precision: int
    bound: float              # relative L2 bound against the FP64 oracle
    params: tuple = ()        # kernel parameters (kappa) or (a, b) for RADON
    rhs_seeds: tuple = (0,)   # one seed per right-hand side, or a single seed for all
    samples: int = 4096       # sampled output points for the oracle check (0 = all)
    order: int = ORDER_NATURAL
    L: int = -1               # level count; -1 lets the planner choose
    src_offset: tuple = ()    # per-axis offset of the source grid (Helmholtz cubes)
    target_seed: int = -1     # >= 0: sorted uniform random targets on [0,1) per axis (type-2 NUDFT)
    description: str = ""

    @property
    def N(self) -> int:
        return self.n ** self.d


def _wl(**kw) -> Workload:
    return Workload(**kw)


WORKLOADS = {
    # d=2 uniform DFT, 64 points per direction, FP64 build and apply (Sec. 4.3 kernel).
    "fourier2d_n64": _wl(
        name="fourier2d_n64", kind=FOURIER, d=2, n=64, tol=1e-8, nv=1, precision=C128,
        bound=1e-7, rhs_seeds=(0,), samples=0, order=ORDER_BITREV, L=4,
        description="d=2 Fourier exp(-2 pi i x.y), x=i/n, y=j-n/2, n=64, FP64"),
    # Green's function between [0,1)^3 and [2,3)x[0,1)^2, 16 wavelengths (Sec. 4.1 geometry).
    "helmholtz3d_n64": _wl(
        name="helmholtz3d_n64", kind=HELMHOLTZ, d=3, n=64, tol=1e-6, nv=1, precision=C64,
        bound=1e-5, params=(2 * math.pi * 16,), rhs_seeds=(0,), samples=4096,
        src_offset=(2.0, 0.0, 0.0), L=4,
        description="d=3 Helmholtz exp(i k r)/r, cubes 2 apart on axis 1, n=64, k=2 pi 16, c64"),
    # Same geometry at 64 wavelengths, 16 right-hand sides, split-BF16 core contraction.
    "helmholtz3d_n256": _wl(
        name="helmholtz3d_n256", kind=HELMHOLTZ, d=3, n=256, tol=1e-4, nv=16,
        precision=C64_SPLITBF16, bound=1e-3, params=(2 * math.pi * 64,),
        rhs_seeds=tuple(range(16)), samples=4096, src_offset=(2.0, 0.0, 0.0), L=4,
        description="d=3 Helmholtz, n=256, k=2 pi 64, 16 RHS, split BF16"),
    # 2-D generalized Radon transform with c(x) = (2 + sin(2 pi x1) sin(2 pi x2)) / 16.
    "radon2d_n256": _wl(
        name="radon2d_n256", kind=RADON, d=2, n=256, tol=1e-6, nv=1, precision=C64,
        bound=1e-4, params=(2.0 / 16.0, 1.0 / 16.0), rhs_seeds=(1,), samples=4096, L=6,
        description="d=2 Radon exp(2 pi i (x.xi + c(x)|xi|)), n=256, c64, autograd"),
    # The paper's other examples at test sizes (Secs. 4.1-4.3), parity cases:
    # Green's function between two parallel unit plates a distance 1 apart
    # (params (kappa, h)), 4 points per wavelength: 2 pi n / kappa = 4.
    "plates2d_n64": _wl(
        name="plates2d_n64", kind=HELMHOLTZ, d=2, n=64, tol=1e-6, nv=2, precision=C64,
        bound=1e-5, params=(math.pi * 64 / 2, 1.0), rhs_seeds=(0, 1), samples=0, L=4,
        description="d=2 Helmholtz between parallel plates at distance 1, n=64, 4 points per wavelength"),
    # 2-D Radon transform with the anisotropic phase of Eq. randon2d.
    "radon2d_aniso_n64": _wl(
        name="radon2d_aniso_n64", kind=RADON_ANISO, d=2, n=64, tol=1e-6, nv=2, precision=C64,
        bound=1e-5, params=(2 / 16, 1 / 16, 2 / 16, 1 / 16), rhs_seeds=(0, 1), samples=0, L=4,
        description="d=2 Radon, phase x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2), n=64"),
    # 3-D Radon transform of Eq. randon3d: c(x) = (3 + prod_k sin(2 pi x_k)) / 100.
    "radon3d_n32": _wl(
        name="radon3d_n32", kind=RADON, d=3, n=32, tol=1e-6, nv=2, precision=C64,
        bound=1e-5, params=(3 / 100, 1 / 100), rhs_seeds=(0, 1), samples=512, L=2,
        description="d=3 Radon, c(x) = (3 + prod sin(2 pi x_k))/100, n=32"),
    # Type-2 non-uniform DFT: random targets on [0,1)^3, integer frequencies.
    "nudft3d_n16": _wl(
        name="nudft3d_n16", kind=FOURIER, d=3, n=16, tol=1e-8, nv=2, precision=C128,
        bound=1e-7, rhs_seeds=(0, 1), samples=0, order=ORDER_BITREV, L=2, target_seed=11,
        description="d=3 type-2 non-uniform DFT, sorted random targets, n=16"),
    # d=6 uniform DFT, 16 points per direction, 8 right-hand sides.
    "fourier6d_n16": _wl(
        name="fourier6d_n16", kind=FOURIER, d=6, n=16, tol=1e-6, nv=8, precision=C64,
        bound=1e-5, rhs_seeds=tuple(range(8)), samples=4096, order=ORDER_BITREV, L=2,
        description="d=6 Fourier, n=16, 8 RHS, c64"),
}


def small(name: str, n: int, nv: int | None = None, **kw) -> Workload:
    """A reduced-size copy of a workload (same kernel and geometry) for fast tests."""
    w = WORKLOADS[name]
    fields = dataclasses.asdict(w)
    fields.update(n=n, name=f"{name}@n{n}", samples=kw.pop("samples", 0))
    if nv is not None:
        fields["nv"] = nv
        fields["rhs_seeds"] = tuple(range(nv)) if nv > 1 else (0,)
    fields.update(kw)
    return Workload(**fields)


def grids(w: Workload):
    """Per-axis coordinates (xs, ys): lists of d float64 arrays of length n.

    Targets x_k[i] = i/n on [0,1) (or sorted seeded uniform random points on
    [0,1) when target_seed >= 0).  Sources: for FOURIER and the RADON kinds the
    integer grid y_k[j] = j - n/2 on [-n/2, n/2); for HELMHOLTZ
    y_k[j] = off_k + j/n (a perpendicular offset h is a kernel parameter).
    """
    n = w.n
    i = np.arange(n, dtype=np.float64)
    xs = [i / n for _ in range(w.d)]
    if w.target_seed >= 0:
        rng = np.random.default_rng(w.target_seed)
        xs = [np.sort(rng.random(n)) for _ in range(w.d)]
    if w.kind == HELMHOLTZ:
        off = w.src_offset or (0.0,) * w.d
        ys = [off[k] + i / n for k in range(w.d)]
    else:
        ys = [i - n / 2 for _ in range(w.d)]
    return xs, ys


def complex_gaussian(shape, seed: int, dtype=torch.complex128) -> torch.Tensor:
    """i.i.d. standard complex Gaussian (re, im each N(0, 1/2)), CPU torch generator."""
    g = torch.Generator().manual_seed(int(seed))
    return torch.randn(*shape, dtype=dtype, generator=g)


def rhs(w: Workload, nv: int | None = None) -> torch.Tensor:
    """Input tensor F of shape (n,)*d + (nv,), complex128, C order (RHS innermost).

    With one seed per RHS, column v is drawn from seed rhs_seeds[v]; otherwise all
    columns come from the single seed.
    """
    nv = w.nv if nv is None else nv
    shape = (w.n,) * w.d
    if len(w.rhs_seeds) == nv and nv > 1:
        cols = [complex_gaussian(shape, s) for s in w.rhs_seeds]
        return torch.stack(cols, dim=-1).contiguous()
    return complex_gaussian(shape + (nv,), w.rhs_seeds[0])


def smooth_bumps(w: Workload, nbumps: int = 8, seed: int = 1) -> torch.Tensor:
    """Sum of Gaussian bumps in xi/n on the source grid: the Radon model f_true.

    Centres uniform in [-1/2, 1/2)^d, widths uniform in (0.03, 0.1), complex
    Gaussian amplitudes; torch generator seeded with `seed`.  Shape (n,)*d + (1,).
    """
    g = torch.Generator().manual_seed(seed)
    c = torch.rand(nbumps, w.d, dtype=torch.float64, generator=g) - 0.5
    wd = 0.03 + 0.07 * torch.rand(nbumps, dtype=torch.float64, generator=g)
    amp = torch.randn(nbumps, dtype=torch.complex128, generator=g)
    _, ys = grids(w)
    axes = torch.meshgrid(*[torch.from_numpy(y / w.n) for y in ys], indexing="ij")
    f = torch.zeros((w.n,) * w.d, dtype=torch.complex128)
    for b in range(nbumps):
        r2 = sum((axes[k] - c[b, k]) ** 2 for k in range(w.d))
        f = f + amp[b] * torch.exp(-r2 / (2 * wd[b] ** 2))
    return f.unsqueeze(-1).contiguous()


def sample_targets(w: Workload, count: int | None = None, seed: int = 4096) -> np.ndarray:
    """Distinct flat output indices (C order over the d target axes), uniform
    without replacement from a torch generator seeded with `seed`."""
    count = w.samples if count is None else count
    N = w.N
    if count <= 0 or count >= N:
        return np.arange(N, dtype=np.int64)
    g = torch.Generator().manual_seed(seed)
    if N <= (1 << 26):
        idx = torch.randperm(N, generator=g)[:count]
    else:  # rejection sampling keeps memory bounded for very large grids
        seen: set = set()
        out = []
        while len(out) < count:
            cand = torch.randint(0, N, (2 * count,), generator=g).tolist()
            for c in cand:
                if c not in seen:
                    seen.add(c)
                    out.append(c)
                    if len(out) == count:
                        break
        idx = torch.tensor(out)
    return idx.numpy().astype(np.int64)


def random_directions(shape, seed: int) -> torch.Tensor:
    """Random complex direction for finite-difference checks (complex Gaussian)."""
    return complex_gaussian(shape, seed)

"""Write the oracle's values for the full-size 3-D Helmholtz configuration.

Configuration: d = 3, n = 256 per axis, kappa = 2 pi 64 (4 points per
wavelength, Sec. 4.1 geometry: unit cubes 2 apart along axis 1), 16
right-hand sides (complex Gaussians, seeds 0-15).  The direct FP64 sum
(oracle/, the plain definition of the contraction of Alg. 2) is evaluated on

  * 4096 target points drawn without replacement with seed 4096 (forward u = K f),
  * 4096 source points drawn with seed 4097 (adjoint v = K^H g with g = f on the
    target grid),

and stored in helmholtz3d_n256.npz together with a fingerprint of the inputs
(f at the first 16 sampled targets), so a test can tell whether the seeded
input generator reproduces the same tensor.  Only oracle/ and the seeded input
generators (workloads.py) are used; nothing here touches the CUDA library.

Run from the repository root:  python tests/golden/make_helmholtz3d_n256.py
(about 40 minutes on 8 cores).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "helmholtz3d_n256.npz")
FWD_SEED, ADJ_SEED, COUNT = 4096, 4097, 4096


def main():
    w = W.WORKLOADS["helmholtz3d_n256"]
    f = W.rhs(w).numpy()
    rows = W.sample_targets(w, COUNT, seed=FWD_SEED)
    cols = W.sample_targets(w, COUNT, seed=ADJ_SEED)
    t0 = time.time()
    u = oracle.workload_apply(w, f, rows)
    t1 = time.time()
    v = oracle.workload_apply_adjoint(w, f, cols)
    t2 = time.time()
    fp = f.reshape(-1, w.nv)[rows[:16]]
    np.savez(OUT, rows=rows, cols=cols, u=u, v=v, fingerprint=fp, nv=w.nv, n=w.n,
             kappa=w.params[0], tol=w.tol)
    print(f"forward {t1 - t0:.0f} s, adjoint {t2 - t1:.0f} s, {oracle.threads()} threads -> {OUT}")


if __name__ == "__main__":
    main()

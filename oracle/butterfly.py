"""Step-by-step oracle of the tensor butterfly apply (plain FP64 numpy).

TEST INFRASTRUCTURE ONLY: only tests/ may use this module.  It shares no code
with the CUDA library; it reads a built butterfly only as plain arrays (the
factor blocks, ranks and cores that the library exports, in the format
documented with tb_export_factors / tb_export_cores in include/tb.h) and
applies them exactly as the paper writes the method, so the GPU apply can be
compared with it to rounding, independently of the ID's approximation error.

  apply(bf, f)          Alg. 2 (contraction), steps (1) - (3) in the paper's order
                        (source_part: steps (1)-(2) for a range of mid-level source
                        multi-sets; target_part: step (3) for a range of target ones):
                        (1) F_{tau,s} for l = 0..Lc: F(s) x_k V-bar^{s,k} at l = 0,
                            F_{p_tau,s} x_k diag_nu(W^{s,k}_{tau,nu}) at l > 0;
                        (2) G_{t,s} = K(t-bar, s-bar) x_{d+1..2d} F_{t,s};
                        (3) for l = Lc..1, G_{t,p_nu} += G_{t,nu} x_k diag_tau(P^{t,k}_{tau,nu})
                            and at l = 0 G(t) = G_{t,nu} x_k U-bar^{t,k}.
  apply_adjoint(bf, g)  the conjugate transpose of every step, in reverse order.
  dense(bf)             the full matrix of the butterfly, assembled pair by pair
                        from Eq. (butterfly_tensor): K(t, s) ~ K(t-bar, s-bar)
                        x_k (P-bar_Lc .. P-bar_1 U-bar) x_{d+k} (W-bar_Lc .. W-bar_1 V-bar)
                        (tiny problems only).
  cores_from_kernel(bf, kernel)  K(t-bar, s-bar) evaluated at the exported
                        skeleton points with a kernel function of the caller.

Every mode product is written out with a dense block-diagonal matrix (zeros
included) and numpy's tensordot; there is no blocking, fusion or reordering.

Conventions (Sec. 3.2): a multi-set at level l has a node index i_k in
[0, 2^l) per mode; its flat index is sum_k i_k 2^(l (d-1-k)); its parent has
node indices i_k // 2; the children of node q (at any level) are 2q and 2q+1.
Node i at level l of mode k covers tree positions [i n_k / 2^l, (i+1) n_k / 2^l);
tree position p is grid index perm[k][p].  The source side applies a block A
(rank x candidates) as A x, the target side as A^T x (the mode-product
orientation under which Alg. 2 computes K F: contract the column index of the
ID matrix).  Arrays are complex128 with the right-hand sides on the last axis.
"""
from __future__ import annotations

import numpy as np


# ------------------------------------------------------------------ indices
def _flat(idx, l, d):
    f = 0
    for k in range(d):
        f = (f << l) | int(idx[k])
    return f


def _unflat(flat, l, d):
    return [(flat >> (l * (d - 1 - k))) & ((1 << l) - 1) for k in range(d)]


def _parent(flat, l, d):
    """Flat index at level l-1 of the parent multi-set of multi-set `flat` at level l."""
    return _flat([i >> 1 for i in _unflat(flat, l, d)], l - 1, d)


def _ancestor(flat, lfrom, lto, d):
    return _flat([i >> (lfrom - lto) for i in _unflat(flat, lfrom, d)], lto, d)


class _Bf:
    def __init__(self, bf):
        self.d, self.L, self.Lc = int(bf["d"]), int(bf["L"]), int(bf["Lc"])
        self.n = [int(v) for v in bf["n"]]
        self.cb = [int(v) for v in bf["cb"]]
        self.perm = [np.asarray(p, dtype=np.int64) for p in bf["perm"]]
        self.fac = bf["factors"]
        self.offs, self.dims, self.core = bf["core_offsets"], bf["core_dims"], bf["core"]
        self.nF = 1 << (self.d * self.Lc)

    def j(self, l, S, T, q):
        return ((S << (self.d * l)) + T) * (1 << (self.Lc - l)) + q

    def rank(self, side, l, k, S, T, q):
        return int(self.fac[(side, l, k)]["ranks"][self.j(l, S, T, q)])

    def block(self, side, l, k, S, T, q):
        """The block of (side, level l, mode k) for mid-level multi-set S, level-l
        multi-set T of the other tree and node q below S_k, cut to its ranks:
        rank x C_b at l = 0, rank x (rank of child 2q + rank of child 2q+1) at l > 0."""
        F = self.fac[(side, l, k)]
        A = F["blocks"][self.j(l, S, T, q)][: self.rank(side, l, k, S, T, q)]
        if l == 0:
            return A[:, : self.cb[k]]
        pT = _parent(T, l, self.d)
        Rp = self.fac[(side, l - 1, k)]["blocks"].shape[1]
        r1 = self.rank(side, l - 1, k, S, pT, 2 * q)
        r2 = self.rank(side, l - 1, k, S, pT, 2 * q + 1)
        return A[:, np.r_[0:r1, Rp:Rp + r2]]

    def diag(self, side, l, k, S, T):
        """diag_q of the blocks over the 2^(Lc-l) nodes q below S_k at depth Lc - l."""
        return _blockdiag([self.block(side, l, k, S, T, q) for q in range(1 << (self.Lc - l))])

    def grid(self, k, node):
        """Grid indices along mode k of mid-level node `node`, in tree order."""
        w = self.n[k] >> self.Lc
        return self.perm[k][node * w:(node + 1) * w]

    def core_block(self, t, s):
        p = t * self.nF + s
        dm = [int(v) for v in self.dims[p]]
        rt, rs = dm[: self.d], dm[self.d:]
        C = self.core[self.offs[p]:self.offs[p + 1]].reshape(int(np.prod(rt)), int(np.prod(rs)))
        return C, rt, rs


def _blockdiag(blocks):
    rows = sum(b.shape[0] for b in blocks)
    cols = sum(b.shape[1] for b in blocks)
    M = np.zeros((rows, cols), dtype=np.complex128)
    r = c = 0
    for b in blocks:
        M[r:r + b.shape[0], c:c + b.shape[1]] = b
        r += b.shape[0]
        c += b.shape[1]
    return M


def _mode(X, A, k):
    """Y = X x_k A: Y[.., a, ..] = sum_b A[a, b] X[.., b, ..] along axis k."""
    return np.moveaxis(np.tensordot(A, X, axes=([1], [k])), 0, k)


def _ix(B, node_idx):
    return np.ix_(*[B.grid(k, node_idx[k]) for k in range(B.d)])


# -------------------------------------------------------------------- apply
def source_part(bf, f, s_range=None) -> dict:
    """Steps (1) and (2) of Alg. 2 for the mid-level source multi-sets s in
    s_range = (begin, end) (all if None): {(t, s): G_{t,s}} for every t and those s."""
    B = _Bf(bf)
    d, Lc = B.d, B.Lc
    f = np.asarray(f, dtype=np.complex128)
    if f.ndim == d:
        f = f[..., None]
    nv = f.shape[-1]
    srange = range(B.nF) if s_range is None else range(int(s_range[0]), int(s_range[1]))
    # (1) source side, l = 0 .. Lc: F[(tau, s)]
    F = {}
    for s in srange:
        X = f[_ix(B, _unflat(s, Lc, d))]
        for k in range(d):
            X = _mode(X, B.diag(0, 0, k, s, 0), k)
        F[(0, s)] = X
    for l in range(1, Lc + 1):
        Fn = {}
        for s in srange:
            for tau in range(1 << (d * l)):
                X = F[(_parent(tau, l, d), s)]
                for k in range(d):
                    X = _mode(X, B.diag(0, l, k, s, tau), k)
                Fn[(tau, s)] = X
        F = Fn
    # (2) mid-level cores: G_{t,s} = K(t-bar, s-bar) x F_{t,s}
    G = {}
    for t in range(B.nF):
        for s in srange:
            C, rt, rs = B.core_block(t, s)
            X = F[(t, s)]
            assert list(X.shape[:d]) == rs, "core source dims differ from F_{t,s}"
            G[(t, s)] = (C @ X.reshape(-1, nv)).reshape(*rt, nv)
    return G


def target_part(bf, G, t_range=None, out=None) -> np.ndarray:
    """Step (3) of Alg. 2 for the mid-level target multi-sets t in t_range (all if
    None) from the tiles G[(t, s)] of those t and every s: writes their target
    points into `out` (a zero tensor of the target grid's shape + nv if None)."""
    B = _Bf(bf)
    d, Lc = B.d, B.Lc
    nv = next(iter(G.values())).shape[-1]
    trange = range(B.nF) if t_range is None else range(int(t_range[0]), int(t_range[1]))
    G = {key: val for key, val in G.items() if key[0] in trange}
    for l in range(Lc, 0, -1):
        Gn = {}
        for t in trange:
            for nu in range(1 << (d * l)):
                X = G[(t, nu)]
                for k in range(d):
                    X = _mode(X, B.diag(1, l, k, t, nu).T, k)
                key = (t, _parent(nu, l, d))
                Gn[key] = Gn[key] + X if key in Gn else X
        G = Gn
    u = np.zeros(tuple(B.n) + (nv,), dtype=np.complex128) if out is None else out
    for t in trange:
        X = G[(t, 0)]
        for k in range(d):
            X = _mode(X, B.diag(1, 0, k, t, 0).T, k)
        u[_ix(B, _unflat(t, Lc, d))] = X
    return u


def apply(bf, f) -> np.ndarray:
    """u = K_BF f, Alg. 2: steps (1) - (2) for every source multi-set, then step (3)."""
    d = int(bf["d"])
    squeeze = np.asarray(f).ndim == d
    u = target_part(bf, source_part(bf, f))
    return u[..., 0] if squeeze else u


def apply_adjoint(bf, g) -> np.ndarray:
    """v = K_BF^H g: the steps of Alg. 2 conjugate-transposed, in reverse order."""
    B = _Bf(bf)
    d, Lc = B.d, B.Lc
    g = np.asarray(g, dtype=np.complex128)
    squeeze = g.ndim == d
    if squeeze:
        g = g[..., None]
    nv = g.shape[-1]
    # (3)^H target leaves, then splits l = 1..Lc
    G = {}
    for t in range(B.nF):
        X = g[_ix(B, _unflat(t, Lc, d))]
        for k in range(d):
            X = _mode(X, B.diag(1, 0, k, t, 0).conj(), k)
        G[(t, 0)] = X
    for l in range(1, Lc + 1):
        Gn = {}
        for t in range(B.nF):
            for nu in range(1 << (d * l)):
                X = G[(t, _parent(nu, l, d))]
                for k in range(d):
                    X = _mode(X, B.diag(1, l, k, t, nu).conj(), k)
                Gn[(t, nu)] = X
        G = Gn
    # (2)^H cores
    F = {}
    for t in range(B.nF):
        for s in range(B.nF):
            C, rt, rs = B.core_block(t, s)
            F[(t, s)] = (C.conj().T @ G[(t, s)].reshape(-1, nv)).reshape(*rs, nv)
    # (1)^H source transfers l = Lc..1 (sum over the children tau), then leaves
    for l in range(Lc, 0, -1):
        Fn = {}
        for s in range(B.nF):
            for tau in range(1 << (d * l)):
                X = F[(tau, s)]
                for k in range(d):
                    X = _mode(X, B.diag(0, l, k, s, tau).conj().T, k)
                key = (_parent(tau, l, d), s)
                Fn[key] = Fn[key] + X if key in Fn else X
        F = Fn
    v = np.zeros(tuple(B.n) + (nv,), dtype=np.complex128)
    for s in range(B.nF):
        X = F[(0, s)]
        for k in range(d):
            X = _mode(X, B.diag(0, 0, k, s, 0).conj().T, k)
        v[_ix(B, _unflat(s, Lc, d))] = X
    return v[..., 0] if squeeze else v


# ---------------------------------------------------------- dense assembly
def dense(bf) -> np.ndarray:
    """The butterfly's full matrix (prod m_k x prod n_k, C-order flattening of
    the grids), pair by pair from Eq. (butterfly_tensor)."""
    B = _Bf(bf)
    d, Lc = B.d, B.Lc
    N = int(np.prod(B.n))
    K = np.zeros((N, N), dtype=np.complex128)
    strides = [int(np.prod(B.n[k + 1:])) for k in range(d)]
    for t in range(B.nF):
        for s in range(B.nF):
            C, rt, rs = B.core_block(t, s)
            T = C.reshape(*rt, *rs)
            for k in range(d):
                # source chain of mode k: W-bar_Lc ... W-bar_1 V-bar, with the
                # level-l multi-set tau the ancestor of t at level l
                Ms = B.diag(0, 0, k, s, 0)
                for l in range(1, Lc + 1):
                    Ms = B.diag(0, l, k, s, _ancestor(t, Lc, l, d)) @ Ms
                # target chain of mode k: P-bar_Lc ... P-bar_1 U-bar, nu the ancestor of s
                Mt = B.diag(1, 0, k, t, 0)
                for l in range(1, Lc + 1):
                    Mt = B.diag(1, l, k, t, _ancestor(s, Lc, l, d)) @ Mt
                T = _mode(T, Mt.T, k)
                T = _mode(T, Ms.T, d + k)
            ti, si = _unflat(t, Lc, d), _unflat(s, Lc, d)
            rows = sum(np.ix_(*[B.grid(k, ti[k]) * strides[k] for k in range(d)]))
            cols = sum(np.ix_(*[B.grid(k, si[k]) * strides[k] for k in range(d)]))
            K[np.ix_(rows.reshape(-1), cols.reshape(-1))] = T.reshape(rows.size, cols.size)
    return K


def cores_from_kernel(bf, kernel) -> np.ndarray:
    """K(t-bar, s-bar) of every pair evaluated at the exported skeleton points:
    kernel(i, j) is the caller's kernel value for target grid multi-index i and
    source grid multi-index j.  Same layout as bf["core"]."""
    B = _Bf(bf)
    d, Lc = B.d, B.Lc
    out = np.zeros_like(np.asarray(B.core))
    for t in range(B.nF):
        for s in range(B.nF):
            p = t * B.nF + s
            C, rt, rs = B.core_block(t, s)
            tsk = [B.fac[(1, Lc, k)]["skel"][B.j(Lc, t, s, 0)][: rt[k]] for k in range(d)]
            ssk = [B.fac[(0, Lc, k)]["skel"][B.j(Lc, s, t, 0)][: rs[k]] for k in range(d)]
            vals = np.empty((int(np.prod(rt)), int(np.prod(rs))), dtype=np.complex128)
            for a, ia in enumerate(np.ndindex(*rt)):
                i = [int(tsk[k][ia[k]]) for k in range(d)]
                for b, ib in enumerate(np.ndindex(*rs)):
                    vals[a, b] = kernel(i, [int(ssk[k][ib[k]]) for k in range(d)])
            out[B.offs[p]:B.offs[p + 1]] = vals.reshape(-1)
    return out

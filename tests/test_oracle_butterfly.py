"""Pins for the step-by-step oracle (oracle/butterfly.py), no GPU.

The oracle applies a tensor butterfly given as plain arrays (the format of
tb_export_factors / tb_export_cores).  Here the arrays are synthetic: random
ranks, random blocks zero-padded as the format prescribes, random cores of the
matching dimensions, random tree orderings.  Three independent routes must
agree:
  * the level-by-level sweep of Alg. 2 (butterfly.apply / apply_adjoint),
  * the pair-by-pair dense assembly of Eq. (butterfly_tensor) (butterfly.dense),
  * closed forms: with L = 0 the butterfly is one Tucker-ID (Sec. 3.1), the
    Kronecker product of the per-mode interpolation matrices around the core;
    with factors and cores that are products over the modes it is the
    Kronecker product of one-dimensional (matrix) butterflies (Sec. 3.2: for
    d = 1 the tensor butterfly is the matrix butterfly).
A swapped child slot, a wrong parent index, a missing transpose or conjugate
breaks at least one of them.
"""
import itertools

import numpy as np
import pytest

from oracle import butterfly as O2


def _flat(idx, l):
    f = 0
    for i in idx:
        f = (f << l) | i
    return f


def synthetic(d, L, cb, R, seed, separable=False):
    """A random butterfly in the export format.  separable=True: every block
    depends only on its own mode's indices and each core is the Kronecker
    product of per-mode matrices."""
    rng = np.random.default_rng(seed)
    Lc = L // 2
    n = cb << L
    nF = 1 << (d * Lc)
    bf = {"d": d, "L": L, "Lc": Lc, "n": [n] * d, "cb": [cb] * d,
          "perm": [rng.permutation(n).astype(np.int32) for _ in range(d)], "factors": {}}

    def rnd(*shape):
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)

    # per-mode tables for the separable form, keyed by (side, l, k, S_k, T_k, q)
    sep_rank, sep_blk = {}, {}
    for side in (0, 1):
        for l in range(Lc + 1):
            for k in range(d):
                cin = cb if l == 0 else 2 * R
                count = nF * (1 << (d * l)) * (1 << (Lc - l))
                ranks = np.zeros(count, dtype=np.int32)
                blocks = np.zeros((count, R, cin), dtype=np.complex128)
                for S in range(nF):
                    Sk = (S >> (Lc * (d - 1 - k))) & ((1 << Lc) - 1)
                    for T in range(1 << (d * l)):
                        Tk = (T >> (l * (d - 1 - k))) & ((1 << l) - 1) if l else 0
                        for q in range(1 << (Lc - l)):
                            j = ((S << (d * l)) + T) * (1 << (Lc - l)) + q
                            key = (side, l, k, Sk, Tk, q)
                            if separable and key in sep_rank:
                                r, B = sep_rank[key], sep_blk[key]
                            else:
                                r = int(rng.integers(1, min(R, cin) + 1))
                                B = rnd(r, cin)
                                sep_rank[key], sep_blk[key] = r, B
                            ranks[j] = r
                            blocks[j, :r] = B
                bf["factors"][(side, l, k)] = {"ranks": ranks, "skel": np.full((count, R), -1, np.int32),
                                               "blocks": blocks}
    # zero the columns past each child's rank (the format's padding)
    for side in (0, 1):
        for l in range(1, Lc + 1):
            for k in range(d):
                F, Fp = bf["factors"][(side, l, k)], bf["factors"][(side, l - 1, k)]
                for S in range(nF):
                    for T in range(1 << (d * l)):
                        pT = _flat([(T >> (l * (d - 1 - m)) & ((1 << l) - 1)) >> 1 for m in range(d)], l - 1)
                        for q in range(1 << (Lc - l)):
                            j = ((S << (d * l)) + T) * (1 << (Lc - l)) + q
                            jc = ((S << (d * (l - 1))) + pT) * (1 << (Lc - l + 1)) + 2 * q
                            r1, r2 = Fp["ranks"][jc], Fp["ranks"][jc + 1]
                            F["blocks"][j, :, r1:R] = 0
                            F["blocks"][j, :, R + r2:] = 0
    offs, dims, core = [0], [], []
    kron_cache = {}
    for t in range(nF):
        for s in range(nF):
            rt = [int(bf["factors"][(1, Lc, k)]["ranks"][(t << (d * Lc)) + s]) for k in range(d)]
            rs = [int(bf["factors"][(0, Lc, k)]["ranks"][(s << (d * Lc)) + t]) for k in range(d)]
            if separable:
                C = np.ones((1, 1), dtype=np.complex128)
                for k in range(d):
                    tk = (t >> (Lc * (d - 1 - k))) & ((1 << Lc) - 1)
                    sk = (s >> (Lc * (d - 1 - k))) & ((1 << Lc) - 1)
                    key = (k, tk, sk)
                    if key not in kron_cache:
                        kron_cache[key] = rnd(rt[k], rs[k])
                    C = np.kron(C, kron_cache[key])
                # C rows run over (a_0, .., a_{d-1}), columns over (b_0, ..): C order, as the format
            else:
                C = rnd(int(np.prod(rt)), int(np.prod(rs)))
            dims.append(rt + rs)
            core.append(C.reshape(-1))
            offs.append(offs[-1] + C.size)
    bf["core_offsets"] = np.array(offs, dtype=np.int64)
    bf["core_dims"] = np.array(dims, dtype=np.int32)
    bf["core"] = np.concatenate(core)
    return bf


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [(1, 4, 2, 3), (2, 2, 2, 3), (2, 4, 1, 2), (3, 2, 2, 2)]


@pytest.mark.parametrize("d,L,cb,R", CASES)
def test_sweep_equals_pairwise_dense_assembly(d, L, cb, R):
    bf = synthetic(d, L, cb, R, seed=10 * d + L)
    n = cb << L
    rng = np.random.default_rng(3)
    f = rng.standard_normal((n,) * d + (2,)) + 1j * rng.standard_normal((n,) * d + (2,))
    K = O2.dense(bf)
    u = O2.apply(bf, f)
    assert _rel(u.reshape(-1, 2), K @ f.reshape(-1, 2)) < 1e-12
    g = rng.standard_normal((n,) * d + (2,)) + 1j * rng.standard_normal((n,) * d + (2,))
    v = O2.apply_adjoint(bf, g)
    assert _rel(v.reshape(-1, 2), K.conj().T @ g.reshape(-1, 2)) < 1e-12
    # adjoint identity <K f, g> = <f, K^H g>
    lhs = np.vdot(g.reshape(-1), u.reshape(-1))
    rhs = np.vdot(v.reshape(-1), f.reshape(-1))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_single_level_is_a_tucker_id(d):
    # L = 0: one pair, K = (U_1^T (x) .. (x) U_d^T) C (V_1 (x) .. (x) V_d) on the
    # tree orderings (Sec. 3.1, Eq. tuckerID with the Tucker factors as IDs)
    bf = synthetic(d, 0, 4, 3, seed=5 + d)
    K = O2.dense(bf)
    Ut = np.ones((1, 1))
    Vv = np.ones((1, 1))
    for k in range(d):
        U = bf["factors"][(1, 0, k)]["blocks"][0][: bf["factors"][(1, 0, k)]["ranks"][0]]
        V = bf["factors"][(0, 0, k)]["blocks"][0][: bf["factors"][(0, 0, k)]["ranks"][0]]
        Ut = np.kron(Ut, U.T)
        Vv = np.kron(Vv, V)
    C = bf["core"].reshape(Ut.shape[1], Vv.shape[0])
    tree = Ut @ C @ Vv     # rows / columns in tree order
    n = 4
    idx = [np.asarray(p) for p in bf["perm"]]
    grid_of_tree = sum(np.ix_(*[idx[k] * n ** (d - 1 - k) for k in range(d)])).reshape(-1)
    expect = np.zeros_like(tree)
    expect[np.ix_(grid_of_tree, grid_of_tree)] = tree
    assert _rel(K, expect) < 1e-13


@pytest.mark.parametrize("L,cb", [(2, 2), (4, 1)])
def test_product_factors_give_the_kronecker_product_of_matrix_butterflies(L, cb):
    # blocks and cores that are products over the modes: the 2-D butterfly is
    # the Kronecker product of two 1-D butterflies built from the same blocks
    bf = synthetic(2, L, cb, 3, seed=77, separable=True)
    Lc = L // 2
    one = []
    for k in range(2):
        b1 = {"d": 1, "L": L, "Lc": Lc, "n": [bf["n"][k]], "cb": [cb], "perm": [bf["perm"][k]], "factors": {}}
        for side in (0, 1):
            for l in range(Lc + 1):
                F = bf["factors"][(side, l, k)]
                sel = []
                for S1 in range(1 << Lc):
                    for T1 in range(1 << l):
                        for q in range(1 << (Lc - l)):
                            # the 2-D multi-sets with mode k = (S1, T1) and the other mode 0
                            S = S1 << (Lc * (1 - k))
                            T = T1 << (l * (1 - k))
                            sel.append(((S << (2 * l)) + T) * (1 << (Lc - l)) + q)
                b1["factors"][(side, l, 0)] = {kk: F[kk][sel] for kk in ("ranks", "skel", "blocks")}
        offs, dims, core = [0], [], []
        for t in range(1 << Lc):
            for s in range(1 << Lc):
                p = (t << (Lc * (1 - k))) * (1 << (2 * Lc)) + (s << (Lc * (1 - k)))
                dm = bf["core_dims"][p]
                # pair (t, s) with the other mode's nodes 0: the per-mode core is
                # recovered from the Kronecker product by fixing the other mode's
                # first index (divided by that factor's entry)
                C = bf["core"][bf["core_offsets"][p]:bf["core_offsets"][p + 1]].reshape(*dm)
                rt, rs = dm[k], dm[2 + k]
                Ck = np.moveaxis(C, (k, 2 + k), (0, 1)).reshape(rt, rs, -1)
                ref = Ck[:, :, 0]
                dims.append([rt, rs])
                core.append(ref.reshape(-1))
                offs.append(offs[-1] + ref.size)
        b1["core_offsets"] = np.array(offs, dtype=np.int64)
        b1["core_dims"] = np.array(dims, dtype=np.int32)
        b1["core"] = np.concatenate(core)
        one.append(O2.dense(b1))
    K = O2.dense(bf)
    # the per-mode cores above carry the other mode's first entry as a factor;
    # compare up to the one global scale that this introduces
    Kk = np.kron(one[0], one[1])
    scale = np.vdot(Kk.reshape(-1), K.reshape(-1)) / np.vdot(Kk.reshape(-1), Kk.reshape(-1))
    assert _rel(K, scale * Kk) < 1e-12

// Level passes of the apply (Alg. 2, steps 1 and 3) as one launch per mode.
//
// A level pass applies to every unit a chain of d mode products with that
// unit's factor blocks:
//   LeafIn  : unit = source leaf tile,  X = F(s) (user tensor),      A_k = V-bar^{s,k}
//   Split   : unit = child tau of a group, X = the 2^d parent tiles,  A_k = W block of tau
//   Gather  : unit = child nu of a group,  X = G_{t,nu},              A_k = P block^T; the
//             2^d children of a group are summed into the parent tiles
//   LeafOut : unit = target leaf tile,  X = G_{t,s0},                A_k = U-bar^{t,k}^T
// Launch k computes T_k = T_{k-1} x_k A_k for all units at once and keeps the
// intermediates T_k in HBM (two ping-pong buffers), so each launch is a wide,
// memory-streaming batched product with no shared-memory working set beyond
// the factor blocks: one thread per output column (p, q) holds the column's
// output rows in registers (row chunks of OB), streams the column's input
// fiber from global memory, and reads the factor, staged once per thread block
// in shared memory, as warp-wide broadcasts.
//
// Two launches are group-wide.  The first mode of a Split reads the combined
// parent tile (dims 2 R_{l-1,k}) straight from the 2^d parent tiles and feeds
// all 2^d children from one fiber; the last mode of a Gather sums the 2^d
// children's contributions in registers (a fixed order: deterministic, no
// atomics) and writes each parent-tile entry exactly once.  Leaf passes read
// and write the user tensor through the per-axis tree orderings.
#include "tb_kernels.cuh"

namespace tb {

constexpr int MODE_THREADS = 256;

// acc[i] += sum_{b < m} At[b][a0 + i] x(b), i < OB, At row stride lda.
template <class R, int OB, class LD>
TB_DEV void mode_rows(cx<R> (&acc)[OB], const cx<R> *__restrict__ At, int lda, int a0, int m, const LD &ld) {
    int b = 0;
#pragma unroll 2
    for (; b + 4 <= m; b += 4) {
        const cx<R> x0 = ld(b), x1 = ld(b + 1), x2 = ld(b + 2), x3 = ld(b + 3);
        const cx<R> *r = At + b * lda + a0;
#pragma unroll
        for (int i = 0; i < OB; i += 2) {
            cx<R> u, w;
            ld2(r + i, u, w);
            cmac(acc[i], u, x0);
            cmac(acc[i + 1], w, x0);
            ld2(r + lda + i, u, w);
            cmac(acc[i], u, x1);
            cmac(acc[i + 1], w, x1);
            ld2(r + 2 * lda + i, u, w);
            cmac(acc[i], u, x2);
            cmac(acc[i + 1], w, x2);
            ld2(r + 3 * lda + i, u, w);
            cmac(acc[i], u, x3);
            cmac(acc[i + 1], w, x3);
        }
    }
    for (; b < m; ++b) {
        const cx<R> x = ld(b);
        const cx<R> *r = At + b * lda + a0;
#pragma unroll
        for (int i = 0; i < OB; i += 2) {
            cx<R> u, w;
            ld2(r + i, u, w);
            cmac(acc[i], u, x);
            cmac(acc[i + 1], w, x);
        }
    }
}

// Stage an r x c factor block as dst[b * lda + a] = op(A)[a][b] (op = A or
// A^T, optionally conjugated), zero for a >= o.
template <class R>
TB_DEV void stage_fac(cx<R> *dst, const cx<R> *__restrict__ src, int r, int c, bool trans, bool cj, int lda) {
    const int o = trans ? c : r, m = trans ? r : c;
    for (int e = threadIdx.x; e < m * lda; e += blockDim.x) {
        const int b = e / lda, aa = e - b * lda;
        cx<R> v = {R(0), R(0)};
        if (aa < o) {
            v = trans ? src[b * c + aa] : src[aa * c + b];
            if (cj) v.y = -v.y;
        }
        dst[e] = v;
    }
}

template <class R, int IN, int OUT, int OB>
__global__ void __launch_bounds__(MODE_THREADS) k_mode(const ModeArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R> *As = reinterpret_cast<cx<R> *>(smraw);
    constexpr bool GROUP = (IN == MK_PARENTS || OUT == MK_PARENTS);
    const int d = a.d, Lc = a.Lc, k = a.k;
    const bool leaf = a.pass == 0 || a.pass == 3;
    const int nchild = GROUP ? (1 << d) : 1;
    const int64_t blk = blockIdx.x / a.ncb;
    const int64_t col = (blockIdx.x - blk * a.ncb) * (int64_t)blockDim.x + threadIdx.x;

    // ---- the unit (or group) of this block
    int64_t g = blk;
    int c_unit = 0;
    if (!leaf && !GROUP) {
        g = blk >> d;
        c_unit = (int)(blk & ((1 << d) - 1));
    }
    const int lgs = a.lgs;
    const int64_t sflat = g & (((int64_t)1 << (lgs * d)) - 1);
    const int64_t rest = g >> (lgs * d);
    int sig[MAXD], pMk[MAXD];
    for (int i = 0; i < d; ++i) sig[i] = (int)((sflat >> (lgs * (d - 1 - i))) & ((1 << lgs) - 1));
    int64_t F = rest, pM = 0;
    const int lvl = a.lvl;
    if (!leaf) {
        const int64_t nMp = (int64_t)1 << (d * (lvl - 1));
        pM = rest % nMp;
        F = rest / nMp;
        for (int i = 0; i < d; ++i) pMk[i] = (int)((pM >> ((lvl - 1) * (d - 1 - i))) & ((1 << (lvl - 1)) - 1));
    }
    auto child_M = [&](int c) {
        int64_t M = 0;
        for (int i = 0; i < d; ++i) M = (M << lvl) | (2 * pMk[i] + ((c >> (d - 1 - i)) & 1));
        return M;
    };
    auto unit_of = [&](int c) { return leaf ? g : (g << d) + c; };

    // ---- stage the factor block(s) and, for leaf passes, the grid-index tables
    for (int j = 0; j < nchild; ++j) {
        const int c = GROUP ? j : c_unit;
        const cx<R> *src = fac_block<R>(a.fac, k, F, leaf ? 0 : child_M(c), sig[k], d, Lc);
        stage_fac<R>(As + (int64_t)j * a.fsz, src, a.fac.rows[k], a.fac.cols[k], a.trans != 0, a.conj != 0, a.lda);
    }
    int *gt = reinterpret_cast<int *>(As + (int64_t)nchild * a.fsz);
    int goff[MAXD];
    if (IN == MK_USER || OUT == MK_USER) {
        int off = 0;
        for (int i = 0; i < d; ++i) {
            goff[i] = off;
            const int64_t Fi = (F >> (Lc * (d - 1 - i))) & ((1 << Lc) - 1);
            for (int b = threadIdx.x; b < a.cb[i]; b += blockDim.x)
                gt[off + b] = a.perm[i][Fi * a.nmid[i] + (int64_t)sig[i] * a.cb[i] + b];
            off += a.cb[i];
        }
    }
    __syncthreads();
    if (col >= a.cols) return;

    const int m = a.m, o = a.o, lda = a.lda;
    const int64_t post = a.post, nv = a.nv;
    const int64_t p = col / post, q = col - p * post;

    // ---- input fiber of the column
    auto in_base = [&](int c) -> const cx<R> * {
        if (a.in_tile) {
            const int64_t t = tile_index<R>(a.lin, F, leaf ? 0 : child_M(c), sflat, a.nF, d);
            return a.lin.p + t * a.lin.tsize * nv;
        }
        return a.tin + unit_of(c) * a.in_usize;
    };
    const int64_t xoff = p * m * post + q;
    const cx<R> *xb[2] = {nullptr, nullptr};
    int64_t xs0 = 0;
    int rp0 = 0;
    const cx<R> *uin = nullptr;
    int64_t gs0nv = 0;
    if (IN == MK_PARENTS) {
        // q = (i_1 .. i_{d-1}, v) over the combined dims 2 R'_i
        int64_t rem = q / nv;
        const int64_t v = q - rem * nv;
        int cbits[MAXD];
        int64_t erest = 0, stride = 1;
        for (int i = d - 1; i >= 1; --i) {
            const int ci2 = 2 * a.Rp[i];
            const int ii = (int)(rem % ci2);
            rem /= ci2;
            cbits[i] = ii >= a.Rp[i];
            erest += (ii - cbits[i] * a.Rp[i]) * stride;
            stride *= a.Rp[i];
        }
        xs0 = stride * nv;
        rp0 = a.Rp[0];
        for (int c0 = 0; c0 < 2; ++c0) {
            int64_t sp = 0;
            for (int i = 0; i < d; ++i) sp = (sp << (lgs + 1)) | (2 * sig[i] + (i == 0 ? c0 : cbits[i]));
            const int64_t t = tile_index<R>(a.lin, F, pM, sp, a.nF, d);
            xb[c0] = a.lin.p + (t * a.lin.tsize + erest) * nv + v;
        }
    } else if (IN == MK_USER) {
        int64_t rem = q / nv;
        const int64_t v = q - rem * nv;
        int64_t ub = 0;
        for (int i = d - 1; i >= 1; --i) {
            const int bi = (int)(rem % a.cb[i]);
            rem /= a.cb[i];
            ub += (int64_t)gt[goff[i] + bi] * a.user.gstride[i];
        }
        uin = a.user.p + ub * nv + v;
        gs0nv = a.user.gstride[0] * nv;
    }

    // ---- output of the column
    cx<R> *yb[2] = {nullptr, nullptr};
    int rpl = 0;
    cx<R> *uout = nullptr;
    const int *gtl = gt;
    int64_t gslnv = 0;
    const int64_t yoff = p * o * post + q;
    if (OUT == MK_PARENTS) {
        // post = nv: p = (a_0 .. a_{d-2}) over the combined dims 2 R'_i, q = v
        int64_t rem = p;
        int cbits[MAXD];
        int64_t erest = 0, stride = a.Rp[d - 1];
        for (int i = d - 2; i >= 0; --i) {
            const int ci2 = 2 * a.Rp[i];
            const int ii = (int)(rem % ci2);
            rem /= ci2;
            cbits[i] = ii >= a.Rp[i];
            erest += (ii - cbits[i] * a.Rp[i]) * stride;
            stride *= a.Rp[i];
        }
        rpl = a.Rp[d - 1];
        for (int cl = 0; cl < 2; ++cl) {
            int64_t sp = 0;
            for (int i = 0; i < d; ++i) sp = (sp << (lgs + 1)) | (2 * sig[i] + (i == d - 1 ? cl : cbits[i]));
            const int64_t t = tile_index<R>(a.lout, F, pM, sp, a.nF, d);
            yb[cl] = a.lout.p + (t * a.lout.tsize + erest) * nv + q;
        }
    } else if (OUT == MK_USER) {
        int64_t rem = p, ub = 0;
        for (int i = d - 2; i >= 0; --i) {
            const int ai = (int)(rem % a.cb[i]);
            rem /= a.cb[i];
            ub += (int64_t)gt[goff[i] + ai] * a.user.gstride[i];
        }
        uout = a.user.p + ub * nv + q;
        gtl = gt + goff[d - 1];
        gslnv = a.user.gstride[d - 1] * nv;
    }
    auto out_base = [&](int c) -> cx<R> * {
        if (a.out_tile) {
            const int64_t t = tile_index<R>(a.lout, F, leaf ? 0 : child_M(c), sflat, a.nF, d);
            return a.lout.p + t * a.lout.tsize * nv;
        }
        return a.tout + unit_of(c) * a.out_usize;
    };
    auto store = [&](const cx<R> (&acc)[OB], int a0, cx<R> *Y) {
#pragma unroll
        for (int i = 0; i < OB; ++i) {
            const int aa = a0 + i;
            if (aa < o) {
                if (OUT == MK_UNIT) Y[yoff + aa * post] = acc[i];
                else if (OUT == MK_PARENTS) {
                    const int hi = aa >= rpl;
                    yb[hi][(int64_t)(aa - hi * rpl) * nv] = acc[i];
                } else {
                    uout[(int64_t)gtl[aa] * gslnv] = acc[i];
                }
            }
        }
    };

    if (IN == MK_PARENTS) {
        auto ld = [&](int b) {
            const int hi = b >= rp0;
            return xb[hi][(int64_t)(b - hi * rp0) * xs0];
        };
        for (int c = 0; c < nchild; ++c) {
            cx<R> *Y = (OUT == MK_UNIT) ? out_base(c) : nullptr;
            for (int a0 = 0; a0 < lda; a0 += OB) {
                cx<R> acc[OB];
#pragma unroll
                for (int i = 0; i < OB; ++i) acc[i] = {R(0), R(0)};
                mode_rows<R, OB>(acc, As + (int64_t)c * a.fsz, lda, a0, m, ld);
                store(acc, a0, Y);
            }
        }
    } else if (IN == MK_USER) {
        auto ld = [&](int b) { return uin[(int64_t)gt[b] * gs0nv]; };
        cx<R> *Y = (OUT == MK_UNIT) ? out_base(0) : nullptr;
        for (int a0 = 0; a0 < lda; a0 += OB) {
            cx<R> acc[OB];
#pragma unroll
            for (int i = 0; i < OB; ++i) acc[i] = {R(0), R(0)};
            mode_rows<R, OB>(acc, As, lda, a0, m, ld);
            store(acc, a0, Y);
        }
    } else {
        cx<R> *Y = (OUT == MK_UNIT) ? out_base(c_unit) : nullptr;
        for (int a0 = 0; a0 < lda; a0 += OB) {
            cx<R> acc[OB];
#pragma unroll
            for (int i = 0; i < OB; ++i) acc[i] = {R(0), R(0)};
            for (int j = 0; j < nchild; ++j) {   // children in a fixed order (Gather)
                const cx<R> *X = in_base(GROUP ? j : c_unit) + xoff;
                auto ld = [&](int b) { return X[(int64_t)b * post]; };
                mode_rows<R, OB>(acc, As + (int64_t)j * a.fsz, lda, a0, m, ld);
            }
            store(acc, a0, Y);
        }
    }
}

template <class R, int IN, int OUT>
cudaError_t launch_mode_ob(int ob, const ModeArgs<R> &a, cudaStream_t st) {
    void (*fn)(const ModeArgs<R>) = nullptr;
    switch (ob) {
        case 2: fn = k_mode<R, IN, OUT, 2>; break;
        case 4: fn = k_mode<R, IN, OUT, 4>; break;
        case 6: fn = k_mode<R, IN, OUT, 6>; break;
        case 8: fn = k_mode<R, IN, OUT, 8>; break;
        case 10: fn = k_mode<R, IN, OUT, 10>; break;
        case 12: fn = k_mode<R, IN, OUT, 12>; break;
        case 14: fn = k_mode<R, IN, OUT, 14>; break;
        case 16: fn = k_mode<R, IN, OUT, 16>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = set_smem_once((const void *)fn, a.smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = a.nblk * a.ncb;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    fn<<<(unsigned)blocks, MODE_THREADS, a.smem, st>>>(a);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_mode(int in_kind, int out_kind, int ob, const ModeArgs<R> &a, cudaStream_t st) {
    if (in_kind == MK_USER && out_kind == MK_UNIT) return launch_mode_ob<R, MK_USER, MK_UNIT>(ob, a, st);
    if (in_kind == MK_PARENTS && out_kind == MK_UNIT) return launch_mode_ob<R, MK_PARENTS, MK_UNIT>(ob, a, st);
    if (in_kind == MK_UNIT && out_kind == MK_UNIT) return launch_mode_ob<R, MK_UNIT, MK_UNIT>(ob, a, st);
    if (in_kind == MK_UNIT && out_kind == MK_PARENTS) return launch_mode_ob<R, MK_UNIT, MK_PARENTS>(ob, a, st);
    if (in_kind == MK_UNIT && out_kind == MK_USER) return launch_mode_ob<R, MK_UNIT, MK_USER>(ob, a, st);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_mode<float>(int, int, int, const ModeArgs<float> &, cudaStream_t);
template cudaError_t launch_mode<double>(int, int, int, const ModeArgs<double> &, cudaStream_t);

}  // namespace tb

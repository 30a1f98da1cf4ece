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
// Ranks.  A factor block's rows past its rank are zero, so on the source side
// (op(A) = A) the output rows a >= rank are zero and on the target side
// (op(A) = A^T) the inputs b >= rank meet zero coefficients: a column computes
// only rows a < rank (and stores zeros past them) or reads only inputs
// b < rank.  The skipped terms are exact zeros: results do not change.
//
// Block shape.  A block has 32, 64 or 128 threads, the fewest that give each
// column of a unit a thread (units with few columns leave fewer lanes idle).
// With column slices (SL), S = 2 or 4 groups of threads share each column slot
// and take every S-th (child, row chunk) item of the column, which spreads a
// launch with few columns over S times as many warps.  Neither changes what a
// column computes, nor the order of its sums.
//
// Two launches are group-wide.  The first mode of a Split reads the combined
// parent tile (dims 2 R_{l-1,k}) straight from the 2^d parent tiles and feeds
// all 2^d children from one fiber; the last mode of a Gather sums the 2^d
// children's contributions in registers (a fixed order: deterministic, no
// atomics) and writes each parent-tile entry exactly once.  Leaf passes read
// and write the user tensor through the per-axis tree orderings.
#pragma once

#include "tb_kernels.cuh"

namespace tb {

#ifndef TB_MODE_THREADS
#define TB_MODE_THREADS 128
#endif
constexpr int MODE_THREADS = TB_MODE_THREADS;
#ifndef TB_MODE_NC
#define TB_MODE_NC 1
#endif
constexpr int MODE_NC = TB_MODE_NC;        // output columns per thread
constexpr int MODE_MAXCH = 1 << MAXD;      // children of a group

#ifndef TB_MODE_XB
#define TB_MODE_XB 6
#endif
constexpr int MODE_XB = TB_MODE_XB;        // input values of a column loaded before use
constexpr int MODE_FIBER = 24;             // longest input fiber a Split's first mode keeps in registers

// acc[j][i] += sum_{b < m} At[b][a0 + i] x_j(b) for the NC columns j of a
// thread, i < OB, At row stride lda.  The column's inputs are loaded MODE_XB at
// a time (all issued before the first use, so each thread keeps that many
// loads in flight); each factor load (a warp-wide broadcast) feeds NC columns.
template <class R, int OB, int NC, int XB, bool RK>
TB_DEV void mode_rows_chunk(cx<R> (&acc)[NC][OB], const cx<R> *__restrict__ At, int lda, int a0, int aend, int b,
                            int m, const cx<R> (&x)[NC][XB]) {
    const cx<R> *r = At + b * lda + a0;
    if constexpr (RK) {
        if (b + XB <= m) {
            // a full chunk of inputs: the rank bound is checked once per output
            // pair (each output still sums its inputs in order t = 0 .. XB - 1)
#pragma unroll
            for (int i = 0; i < OB; i += 2) {
                if (a0 + i >= aend) break;   // zero rows of the factor (past its rank)
#pragma unroll
                for (int t = 0; t < XB; ++t) {
                    cx<R> u, w;
                    ld2(r + t * lda + i, u, w);
#pragma unroll
                    for (int j = 0; j < NC; ++j) {
                        cmac(acc[j][i], u, x[j][t]);
                        cmac(acc[j][i + 1], w, x[j][t]);
                    }
                }
            }
            return;
        }
    }
#pragma unroll
    for (int t = 0; t < XB; ++t) {
        if (b + t >= m) break;
#pragma unroll
        for (int i = 0; i < OB; i += 2) {
            if (RK && a0 + i >= aend) break;   // zero rows of the factor (past its rank)
            cx<R> u, w;
            ld2(r + t * lda + i, u, w);
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                cmac(acc[j][i], u, x[j][t]);
                cmac(acc[j][i + 1], w, x[j][t]);
            }
        }
    }
}

template <class R, int NC, int XB, class LD>
TB_DEV void mode_load_chunk(cx<R> (&x)[NC][XB], int b, int m, const LD &ld) {
#pragma unroll
    for (int t = 0; t < XB; ++t)
#pragma unroll
        for (int j = 0; j < NC; ++j) x[j][t] = (b + t < m) ? ld(j, b + t) : cx<R>{R(0), R(0)};
}

// acc[j][i] += sum_{b < m} At[b][a0 + i] x_j(b) for the NC columns j of a
// thread, i < OB, At row stride lda.  The column's inputs are loaded MODE_XB at
// a time into two register buffers: the next chunk's loads are in flight while
// the current chunk is multiplied.  Each factor load (a warp-wide broadcast)
// feeds NC columns.
template <class R, int OB, int NC, bool RK, class LD>
TB_DEV void mode_rows(cx<R> (&acc)[NC][OB], const cx<R> *__restrict__ At, int lda, int a0, int aend, int m,
                      const LD &ld) {
    constexpr int XB = MODE_XB;
    cx<R> x0[NC][XB], x1[NC][XB];
    if (m <= 0) return;
    mode_load_chunk<R, NC, XB>(x0, 0, m, ld);
    for (int b = 0; b < m; b += 2 * XB) {
        if (b + XB < m) mode_load_chunk<R, NC, XB>(x1, b + XB, m, ld);
        mode_rows_chunk<R, OB, NC, XB, RK>(acc, At, lda, a0, aend, b, m, x0);
        if (b + XB >= m) break;
        if (b + 2 * XB < m) mode_load_chunk<R, NC, XB>(x0, b + 2 * XB, m, ld);
        mode_rows_chunk<R, OB, NC, XB, RK>(acc, At, lda, a0, aend, b + XB, m, x1);
    }
}

// Stage one r x c factor block as dst[b * lda + a] = op(A)[a][b] (op = A or
// A^T, optionally conjugated), zero for a >= o.
template <class R>
TB_DEV void stage_fac1(cx<R> *dst, const cx<R> *__restrict__ src, int r, int c, bool trans, bool cj, int lda) {
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

// Stage the r x c factor blocks src[j] of nb children (a group), child j as
// dst[j * fsz + b * lda + a] = op(A_j)[a][b] (op = A or A^T, optionally
// conjugated; b < m = c or r), zero for a >= o and b >= m.  Each thread loads 8 entries
// before it stores any, so a small block keeps several loads in flight.
template <class R>
TB_DEV void stage_fac(cx<R> *dst, const cx<R> *const *src, int nb, int fsz, int r, int c, bool trans, bool cj,
                      int lda) {
    constexpr int SB = 8;
    const int o = trans ? c : r, m = trans ? r : c;
    const int n = nb * fsz, st = blockDim.x;
    for (int e0 = threadIdx.x; e0 < n; e0 += SB * st) {
        cx<R> v[SB];
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            const int e = e0 + u * st;
            v[u] = {R(0), R(0)};
            if (e < n) {
                const int j = e / fsz, rem = e - j * fsz;
                const int b = rem / lda, aa = rem - b * lda;
                if (aa < o && b < m) v[u] = trans ? src[j][b * c + aa] : src[j][aa * c + b];
            }
        }
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            const int e = e0 + u * st;
            if (e < n) {
                if (cj) v[u].y = -v[u].y;
                dst[e] = v[u];
            }
        }
    }
}

template <class R, int IN, int OUT, int OB, bool RK, bool SL>
#ifndef TB_MODE_MINB
#define TB_MODE_MINB 6   // complex64: resident blocks per SM the register allocation must allow
#endif
__global__ void __launch_bounds__(MODE_THREADS, sizeof(R) == 4 ? (OB <= 16 ? TB_MODE_MINB : 4) : 2)
    k_mode(const ModeArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R> *As = reinterpret_cast<cx<R> *>(smraw);
    constexpr bool GROUP = (IN == MK_PARENTS || OUT == MK_PARENTS);
    constexpr bool USER = (IN == MK_USER || OUT == MK_USER);
    constexpr int NC = MODE_NC;
    // block-uniform pointers, set up by the first two warps
    __shared__ const cx<R> *s_fac[MODE_MAXCH];
    __shared__ const cx<R> *s_in[MODE_MAXCH];    // per child: input unit buffer / level tile
    __shared__ cx<R> *s_out[MODE_MAXCH];         // per child: output unit buffer / level tile
    __shared__ cx<R> *s_par[MODE_MAXCH];         // parent tiles by child-bit tuple (Split in, Gather out)
    __shared__ int s_skip;                       // the unit lies outside the multiset range [f0, f1)
    __shared__ int s_rk[MODE_MAXCH];             // per child: rank of its factor block of mode k
    const int d = a.d, k = a.k, tid = threadIdx.x;
    const bool leaf = a.pass == 0 || a.pass == 3;
    const int nchild = GROUP ? (1 << d) : 1;
    // block = (unit or group, first column chunk); it walks the unit's column
    // chunks with stride gsplit, so the factor staging is paid once per block
    const unsigned blk = blockIdx.x / (unsigned)a.gsplit;
    const unsigned cfirst = blockIdx.x - blk * (unsigned)a.gsplit;
    int *gt = reinterpret_cast<int *>(As + (int64_t)nchild * a.fsz);
    int goff[MAXD];
    {
        int off = 0;
        for (int i = 0; i < d; ++i) {
            goff[i] = off;
            off += a.cb[i];
        }
    }

    int my_rk = 0;   // rank of child tid's factor block (its load overlaps the factor staging)
    const int bt = a.bt, pt = bt < 64 ? bt : 64;   // threads per block, of them setting up
    if (tid < pt) {
        // ---- the unit (or group) of this block
        const int Lc = a.Lc, lgs = a.lgs, lvl = a.lvl;
        int64_t g = blk;
        int c_unit = 0;
        if (!leaf && !GROUP) {
            g = blk >> d;
            c_unit = (int)(blk & ((1u << d) - 1));
        }
        const int64_t sflat = g & (((int64_t)1 << (lgs * d)) - 1);
        const int64_t rest = g >> (lgs * d);
        int sig[MAXD], pMk[MAXD];
        for (int i = 0; i < d; ++i) sig[i] = (int)((sflat >> (lgs * (d - 1 - i))) & ((1 << lgs) - 1));
        int64_t F = rest, pM = 0;
        if (!leaf) {
            const int64_t nMp = (int64_t)1 << (d * (lvl - 1));
            pM = rest & (nMp - 1);
            F = rest >> (d * (lvl - 1));
            for (int i = 0; i < d; ++i)
                pMk[i] = (int)((pM >> ((lvl - 1) * (d - 1 - i))) & ((1 << (lvl - 1)) - 1));
        }
        const int j = tid;
        if (j == 0) s_skip = (F < a.f0 || F >= a.f1) ? 1 : 0;
        if (j < nchild) {
            const int c = GROUP ? j : c_unit;
            int64_t M = 0;
            if (!leaf)
                for (int i = 0; i < d; ++i) M = (M << lvl) | (2 * pMk[i] + ((c >> (d - 1 - i)) & 1));
            const int64_t unit = leaf ? g : (g << d) + c;
            const int64_t fj = fac_index<R>(a.fac, k, F, M, sig[k], d, Lc);
            s_fac[j] = a.fac.A[k] + fj * (int64_t)a.fac.rows[k] * a.fac.cols[k];
            if (RK) my_rk = a.fac.rank[k] ? a.fac.rank[k][fj] : a.fac.rows[k];   // published after the staging
            if (a.in_tile)
                s_in[j] = a.lin.p + tile_index<R>(a.lin, F, M, sflat, a.nF, d) * a.lin.tsize * a.nv;
            else
                s_in[j] = a.tin ? a.tin + unit * a.in_usize : nullptr;
            if (a.out_tile)
                s_out[j] = a.lout.p + tile_index<R>(a.lout, F, M, sflat, a.nF, d) * a.lout.tsize * a.nv;
            else
                s_out[j] = a.tout ? a.tout + unit * a.out_usize : nullptr;
        }
        if (GROUP && j < (1 << d)) {
            // parent tile of child-bit tuple j: segments 2 sig_i + bit_i at level l-1
            int64_t sp = 0;
            for (int i = 0; i < d; ++i) sp = (sp << (lgs + 1)) | (2 * sig[i] + ((j >> (d - 1 - i)) & 1));
            const TileBuf<R> &tb = IN == MK_PARENTS ? a.lin : a.lout;
            s_par[j] = tb.p + tile_index<R>(tb, F, pM, sp, a.nF, d) * tb.tsize * a.nv;
        }
        if (USER) {
            for (int i = 0; i < d; ++i) {
                const int64_t Fi = (F >> (Lc * (d - 1 - i))) & ((1 << Lc) - 1);
                for (int b = j; b < a.cb[i]; b += pt)
                    gt[goff[i] + b] = a.perm[i][Fi * a.nmid[i] + (int64_t)sig[i] * a.cb[i] + b];
            }
        }
    }
    __syncthreads();
    if (s_skip) return;   // block-uniform
    // one entry per thread: the plain loop; more: batched loads (a group always)
    if (!GROUP && a.fsz <= bt)
        stage_fac1<R>(As, s_fac[0], a.fac.rows[k], a.fac.cols[k], a.trans != 0, a.conj != 0, a.lda);
    else
        stage_fac<R>(As, s_fac, nchild, a.fsz, a.fac.rows[k], a.fac.cols[k], a.trans != 0, a.conj != 0, a.lda);
    if (tid < nchild) s_rk[tid] = my_rk;
    __syncthreads();

    const int m = a.m, o = a.o, lda = a.lda;
    const bool trans = a.trans != 0;
    const int post = (int)a.post, nv = (int)a.nv, cols = (int)a.cols;
    // S = a.sub warps-or-wider slices of the block share each column slot: slice
    // `sub` takes every S-th (child, row chunk) item of its column
    // SL: S = a.sub slices of cw = bt / S threads share each column slot
    // (S = 2 or 4); slice `sub` takes every S-th (child, row chunk) item
    const int S = SL ? a.sub : 1, cw = SL ? bt / S : bt;
    const int sub = SL ? tid / cw : 0, tc = SL ? tid - sub * cw : tid;
    // item (child c, row chunk a0 / OB) of a Split group belongs to slice
    // (c * chunks + a0 / OB) mod S (recomputed from the arguments: no live registers)
    auto mine = [&](int c, int a0) {
        return !SL || (((c * (a.lda / OB) + a0 / OB) & (a.sub - 1)) == (int)(threadIdx.x / (a.bt / a.sub)));
    };
    for (unsigned cblk = cfirst; cblk < (unsigned)a.ncb; cblk += (unsigned)a.gsplit) {
    const int col0 = (int)cblk * (cw * NC) + tc;
    if (col0 >= cols) break;
    bool valid[NC];
    int pcol[NC], qcol[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        int cc = col0 + j * cw;
        valid[j] = cc < cols;
        if (!valid[j]) cc = cols - 1;   // computes a duplicate, stores nothing
        pcol[j] = cc / post;
        qcol[j] = cc - pcol[j] * post;
    }

    // ---- per-column input
    int xoff[NC];
    const cx<R> *xp0[NC], *xp1[NC];
    int xs0 = 0, rp0 = 0;
    int64_t gs0nv = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        xoff[j] = pcol[j] * m * post + qcol[j];
        xp0[j] = xp1[j] = nullptr;
        if (IN == MK_PARENTS) {
            // q = (i_1 .. i_{d-1}, v) over the combined dims 2 R'_i
            int rem = qcol[j] / nv;
            const int v = qcol[j] - rem * nv;
            int bits = 0, erest = 0, stride = 1;
            for (int i = d - 1; i >= 1; --i) {
                const int ci2 = 2 * a.Rp[i];
                const int ii = rem % ci2;
                rem /= ci2;
                const int bi = ii >= a.Rp[i];
                bits |= bi << (d - 1 - i);
                erest += (ii - bi * a.Rp[i]) * stride;
                stride *= a.Rp[i];
            }
            xs0 = stride * nv;
            rp0 = a.Rp[0];
            xp0[j] = s_par[bits] + (int64_t)erest * nv + v;
            xp1[j] = s_par[bits | (1 << (d - 1))] + (int64_t)erest * nv + v;
        } else if (IN == MK_USER) {
            int rem = qcol[j] / nv;
            const int v = qcol[j] - rem * nv;
            int64_t ub = 0;
            for (int i = d - 1; i >= 1; --i) {
                const int bi = rem % a.cb[i];
                rem /= a.cb[i];
                ub += (int64_t)gt[goff[i] + bi] * a.user.gstride[i];
            }
            xp0[j] = a.user.p + ub * nv + v;
            gs0nv = a.user.gstride[0] * (int64_t)nv;
        }
    }

    // ---- per-column output
    int yoff[NC];
    cx<R> *yp0[NC], *yp1[NC];
    int rpl = 0;
    int64_t gslnv = 0;
    const int *gtl = gt + goff[k];   // tree order of the last mode (LeafOut)
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        yoff[j] = pcol[j] * o * post + qcol[j];
        yp0[j] = yp1[j] = nullptr;
        if (OUT == MK_PARENTS) {
            // post = nv: p = (a_0 .. a_{d-2}) over the combined dims 2 R'_i, q = v
            int rem = pcol[j], bits = 0, erest = 0, stride = a.Rp[d - 1];
            for (int i = d - 2; i >= 0; --i) {
                const int ci2 = 2 * a.Rp[i];
                const int ii = rem % ci2;
                rem /= ci2;
                const int bi = ii >= a.Rp[i];
                bits |= bi << (d - 1 - i);
                erest += (ii - bi * a.Rp[i]) * stride;
                stride *= a.Rp[i];
            }
            rpl = a.Rp[d - 1];
            yp0[j] = s_par[bits] + (int64_t)erest * nv + qcol[j];
            yp1[j] = s_par[bits | 1] + (int64_t)erest * nv + qcol[j];
        } else if (OUT == MK_USER) {
            // the last mode k of a LeafOut: every other mode is already at its leaf
            // size; p runs over the modes before k, q over the modes after k and v
            int rem = pcol[j];
            int64_t ub = 0;
            for (int i = k - 1; i >= 0; --i) {
                const int ai = rem % a.cb[i];
                rem /= a.cb[i];
                ub += (int64_t)gt[goff[i] + ai] * a.user.gstride[i];
            }
            int remq = qcol[j] / nv;
            const int v = qcol[j] - remq * nv;
            for (int i = d - 1; i > k; --i) {
                const int ai = remq % a.cb[i];
                remq /= a.cb[i];
                ub += (int64_t)gt[goff[i] + ai] * a.user.gstride[i];
            }
            yp0[j] = a.user.p + ub * nv + v;
            gslnv = a.user.gstride[k] * (int64_t)nv;
        }
    }

    auto store = [&](const cx<R> (&acc)[NC][OB], int a0, cx<R> *Y) {
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            if (!valid[j]) continue;
#pragma unroll
            for (int i = 0; i < OB; ++i) {
                const int aa = a0 + i;
                if (aa < o) {
                    if (OUT == MK_UNIT) Y[yoff[j] + aa * post] = acc[j][i];
                    else if (OUT == MK_PARENTS) {
                        if (aa < rpl) yp0[j][aa * nv] = acc[j][i];
                        else yp1[j][(aa - rpl) * nv] = acc[j][i];
                    } else {
                        yp0[j][(int64_t)gtl[aa] * gslnv] = acc[j][i];
                    }
                }
            }
        }
    };
    auto zero = [](cx<R> (&acc)[NC][OB]) {
#pragma unroll
        for (int j = 0; j < NC; ++j)
#pragma unroll
            for (int i = 0; i < OB; ++i) acc[j][i] = {R(0), R(0)};
    };

    if (IN == MK_PARENTS) {
        auto ld = [&](int j, int b) {
            const cx<R> *pp = b < rp0 ? xp0[j] + b * xs0 : xp1[j] + (b - rp0) * xs0;
            return *pp;
        };
        if (NC == 1 && m <= MODE_FIBER) {
            // the fiber is read once into registers and feeds all 2^d children
            cx<R> xf[MODE_FIBER];
#pragma unroll
            for (int b = 0; b < MODE_FIBER; ++b) xf[b] = b < m ? ld(0, b) : cx<R>{R(0), R(0)};
            for (int c = 0; c < nchild; ++c) {
                cx<R> *Y = s_out[c];
                const cx<R> *At = As + (int64_t)c * a.fsz;
                const int aend = (RK && !trans) ? s_rk[c] : lda;
                for (int a0 = 0; a0 < lda; a0 += OB) {
                    if (!mine(c, a0)) continue;
                    cx<R> acc[NC][OB];
                    zero(acc);
                    if constexpr (RK) {
                        // output pairs outside (one rank check each), the fiber inside
#pragma unroll
                        for (int i = 0; i < OB; i += 2) {
                            if (a0 + i >= aend) break;
                            const cx<R> *r = At + a0 + i;
#pragma unroll
                            for (int b = 0; b < MODE_FIBER; ++b) {
                                if (b >= m) break;
                                cx<R> u, w;
                                ld2(r + b * lda, u, w);
                                cmac(acc[0][i], u, xf[b]);
                                cmac(acc[0][i + 1], w, xf[b]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int b = 0; b < MODE_FIBER; ++b) {
                            if (b >= m) break;
                            const cx<R> *r = At + b * lda + a0;
#pragma unroll
                            for (int i = 0; i < OB; i += 2) {
                                cx<R> u, w;
                                ld2(r + i, u, w);
                                cmac(acc[0][i], u, xf[b]);
                                cmac(acc[0][i + 1], w, xf[b]);
                            }
                        }
                    }
                    store(acc, a0, Y);
                }
            }
        } else {
            for (int c = 0; c < nchild; ++c) {
                cx<R> *Y = s_out[c];
                const int aend = (RK && !trans) ? s_rk[c] : lda;
                const int mc = (RK && trans) ? min(m, s_rk[c]) : m;
                for (int a0 = 0; a0 < lda; a0 += OB) {
                    if (!mine(c, a0)) continue;
                    cx<R> acc[NC][OB];
                    zero(acc);
                    if (a0 < aend) mode_rows<R, OB, NC, RK>(acc, As + (int64_t)c * a.fsz, lda, a0, aend, mc, ld);
                    store(acc, a0, Y);
                }
            }
        }
    } else if (IN == MK_USER) {
        auto ld = [&](int j, int b) { return xp0[j][(int64_t)gt[b] * gs0nv]; };
        cx<R> *Y = s_out[0];
        const int aend = (RK && !trans) ? s_rk[0] : lda;
        const int mc = (RK && trans) ? min(m, s_rk[0]) : m;
        for (int a0 = SL ? sub * OB : 0; a0 < lda; a0 += SL ? S * OB : OB) {
            cx<R> acc[NC][OB];
            zero(acc);
            if (a0 < aend) mode_rows<R, OB, NC, RK>(acc, As, lda, a0, aend, mc, ld);
            store(acc, a0, Y);
        }
    } else {
        cx<R> *Y = s_out[0];
        for (int a0 = SL ? sub * OB : 0; a0 < lda; a0 += SL ? S * OB : OB) {
            cx<R> acc[NC][OB];
            zero(acc);
            for (int c = 0; c < nchild; ++c) {   // children in a fixed order (Gather)
                const cx<R> *X = s_in[c];
                const int aend = (RK && !trans) ? s_rk[c] : lda;
                const int mc = (RK && trans) ? min(m, s_rk[c]) : m;
                auto ld = [&](int j, int b) { return X[xoff[j] + b * post]; };
                if (a0 < aend) mode_rows<R, OB, NC, RK>(acc, As + (int64_t)c * a.fsz, lda, a0, aend, mc, ld);
            }
            store(acc, a0, Y);
        }
    }
    }   // column chunks
}

template <class R, int IN, int OUT, bool RK, bool SL>
cudaError_t launch_mode_ob(int ob, const ModeArgs<R> &a, cudaStream_t st) {
    void (*fn)(const ModeArgs<R>) = nullptr;
    switch (ob) {
        case 2: fn = k_mode<R, IN, OUT, 2, RK, SL>; break;
        case 4: fn = k_mode<R, IN, OUT, 4, RK, SL>; break;
        case 6: fn = k_mode<R, IN, OUT, 6, RK, SL>; break;
        case 8: fn = k_mode<R, IN, OUT, 8, RK, SL>; break;
        case 10: fn = k_mode<R, IN, OUT, 10, RK, SL>; break;
        case 12: fn = k_mode<R, IN, OUT, 12, RK, SL>; break;
        case 14: fn = k_mode<R, IN, OUT, 14, RK, SL>; break;
        case 16: fn = k_mode<R, IN, OUT, 16, RK, SL>; break;
        case 18: fn = k_mode<R, IN, OUT, 18, RK, SL>; break;
        case 20: fn = k_mode<R, IN, OUT, 20, RK, SL>; break;
        case 24: fn = k_mode<R, IN, OUT, 24, RK, SL>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = set_smem_once((const void *)fn, a.smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = a.nblk * a.gsplit;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    if (a.bt != 32 && a.bt != 64 && a.bt != MODE_THREADS) return cudaErrorInvalidValue;
    if (a.sub < 1 || (!SL && a.sub != 1) || a.bt % a.sub || (a.bt / a.sub) % 32) return cudaErrorInvalidValue;
    fn<<<(unsigned)blocks, (unsigned)a.bt, a.smem, st>>>(a);
    return cudaGetLastError();
}

// The per-mode launch of kinds (in_kind, out_kind), output rows per register
// chunk ob, rank bounds on (RK) or off, column slices (SL, a.sub > 1) or not;
// instantiated in tb_mode.cu (neither), tb_mode_rank.cu (RK), and
// tb_mode_slice.cu / tb_mode_slice_rank.cu (SL, complex64), which compile in
// parallel.
template <class R, bool RK, bool SL>
cudaError_t launch_mode_rk(int in_kind, int out_kind, int ob, const ModeArgs<R> &a, cudaStream_t st) {
    if (in_kind == MK_USER && out_kind == MK_UNIT) return launch_mode_ob<R, MK_USER, MK_UNIT, RK, SL>(ob, a, st);
    if (in_kind == MK_PARENTS && out_kind == MK_UNIT)
        return launch_mode_ob<R, MK_PARENTS, MK_UNIT, RK, SL>(ob, a, st);
    if (in_kind == MK_UNIT && out_kind == MK_UNIT) return launch_mode_ob<R, MK_UNIT, MK_UNIT, RK, SL>(ob, a, st);
    if (in_kind == MK_UNIT && out_kind == MK_PARENTS)
        return launch_mode_ob<R, MK_UNIT, MK_PARENTS, RK, SL>(ob, a, st);
    if (in_kind == MK_UNIT && out_kind == MK_USER) return launch_mode_ob<R, MK_UNIT, MK_USER, RK, SL>(ob, a, st);
    return cudaErrorInvalidValue;
}

}  // namespace tb

// Apply kernels of the tensor butterfly contraction (Alg. 2, Sec. 3.2).
//
// Every level pass works on tiles: a tile is the block F_{tau,s} (source side)
// or G_{t,nu} (target side) restricted to one tuple of segments (one node per
// mode), i.e. prod_k R_{l,k} entries with the nv right-hand sides innermost.
// A thread block stages its tiles in shared memory and contracts them mode by
// mode (the products prod_k x_k of Alg. 2) with the per-mode factor blocks
// staged beside them:
//
//   LeafIn  : F_{t0,s} = F(s) prod_k x_k V-bar^{s,k}                 (Alg. 2, step 1, l = 0)
//   Split   : F_{tau,s} = F_{p_tau,s} prod_k x_k diag_nu(W)          (Alg. 2, step 1, l > 0)
//             one block reads the 2^d parent tiles once and writes all 2^d children
//   core    : G_{t,s} = K(t-bar, s-bar) x_{d+1..2d} F_{t,s}          (Alg. 2, step 2)
//   Gather  : G_{t,p_nu} += G_{t,nu} prod_k x_k diag_tau(P)           (Alg. 2, step 3, l > 0)
//             one block sums the 2^d children in shared memory: no atomics,
//             deterministic order
//   LeafOut : G(t) = G_{t,s0} prod_k x_k U-bar^{t,k}                 (Alg. 2, step 3, l = 0)
//
// The adjoint K^H runs the same passes in reverse with conjugated factors:
// a Split with conj(P), a Gather with conj(W)^T, LeafIn with conj(U), LeafOut
// with conj(V)^T and the core with K(t-bar, s-bar)^H.
#include "tb_kernels.cuh"

namespace tb {

constexpr int AP_THREADS = 256;
constexpr int CORE_THREADS = 256;
constexpr int AB = 4;   // output rows per thread in the leaf passes

// Staged factors are transposed: At[b * lda + a] = A[a][b] with lda = o rounded
// up to a multiple of 4 and zero columns a >= o (see stage()).
TB_HD int lda_of(int o) { return (o + 3) & ~3; }

// dst[p][a][q] (=|+=) sum_b A[a][b] src[p][b][q] with A given transposed (At).
// Each item computes NR consecutive output rows a of one column (p, q); items
// run with q fastest, so a warp shares (p, a-block) whenever post >= 32 and its
// reads of At are broadcasts.
template <class R, int NR>
TB_DEV void mode_pass_rows(const cx<R> *__restrict__ src, cx<R> *__restrict__ dst, const cx<R> *__restrict__ At,
                           int pre, int mk, int ok, int post, bool acc) {
    const int nab = (ok + NR - 1) / NR, lda = lda_of(ok);
    const int items = pre * nab * post;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int q = it % post;
        const int r = it / post;
        const int ab = r % nab, p = r / nab;
        const int a0 = ab * NR;
        cx<R> c[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) c[i] = {R(0), R(0)};
        const cx<R> *s = src + (p * mk) * post + q;
        int acol[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) acol[i] = min(a0 + i, ok - 1);
#pragma unroll 2
        for (int b = 0; b < mk; ++b) {
            const cx<R> x = s[b * post];
            const cx<R> *arow = At + b * lda;
#pragma unroll
            for (int i = 0; i < NR; ++i) cmac(c[i], arow[acol[i]], x);
        }
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            if (a0 + i < ok) {
                const int idx = (p * ok + a0 + i) * post + q;
                dst[idx] = acc ? dst[idx] + c[i] : c[i];
            }
        }
    }
}

// Register-tiled form: each item computes 4 output rows x 2 adjacent columns
// from the transposed factor At[b][a] (row stride lda, a multiple of 4, zero
// padded), so one b step costs two vector loads of At, one vector load of the
// column pair and 8 complex FMAs.  Needs post even.
template <class R>
TB_DEV void mode_pass_tile(const cx<R> *__restrict__ src, cx<R> *__restrict__ dst, const cx<R> *__restrict__ At,
                           int lda, int pre, int mk, int ok, int post, bool acc) {
    const int nab = (ok + 3) / 4, nqb = post >> 1;
    const int items = pre * nab * nqb;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int qb = it % nqb;
        const int r = it / nqb;
        const int ab = r % nab, p = r / nab;
        const int a0 = ab * 4, q = 2 * qb;
        cx<R> c[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i) c[i][0] = c[i][1] = {R(0), R(0)};
        const cx<R> *s = src + (p * mk) * post + q;
        const cx<R> *ap = At + a0;
#pragma unroll 2
        for (int b = 0; b < mk; ++b) {
            const cx<R> x0 = s[b * post], x1 = s[b * post + 1];
            const cx<R> *arow = ap + b * lda;
            cx<R> av[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = arow[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                cmac(c[i][0], av[i], x0);
                cmac(c[i][1], av[i], x1);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (a0 + i < ok) {
                const int idx = (p * ok + a0 + i) * post + q;
                if (acc) {
                    dst[idx] = dst[idx] + c[i][0];
                    dst[idx + 1] = dst[idx + 1] + c[i][1];
                } else {
                    dst[idx] = c[i][0];
                    dst[idx + 1] = c[i][1];
                }
            }
        }
    }
}

// One mode product with the transposed factor At.  The register-tiled form is
// used when the column count is even and there is an item for every thread;
// otherwise the largest row block that still gives every thread an item.
template <class R>
TB_DEV void mode_pass(const cx<R> *__restrict__ src, cx<R> *__restrict__ dst, const cx<R> *__restrict__ At,
                      int pre, int mk, int ok, int post, bool acc) {
    const int cols = pre * post, T = blockDim.x;
    if ((post & 1) == 0 && (cols / 2) * ((ok + 3) / 4) >= T) {
        mode_pass_tile<R>(src, dst, At, lda_of(ok), pre, mk, ok, post, acc);
        return;
    }
    if (cols * ((ok + 7) / 8) >= T) mode_pass_rows<R, 8>(src, dst, At, pre, mk, ok, post, acc);
    else if (cols * ((ok + 3) / 4) >= T) mode_pass_rows<R, 4>(src, dst, At, pre, mk, ok, post, acc);
    else mode_pass_rows<R, 2>(src, dst, At, pre, mk, ok, post, acc);
}

// Passes k0 .. k1-1 of Y = X x_0 A_0 x_1 A_1 ... x_{d-1} A_{d-1}; X dims m[],
// Y dims o[], nvc innermost.  The output of pass k goes to Y for k = d-1 and to
// b0 / b1 (by parity of k) otherwise; `src` is the input of pass k0.
template <class R>
TB_DEV const cx<R> *mode_chain(int d, int k0, int k1, const int *m, const int *o, cx<R> *const *As,
                               const cx<R> *src, cx<R> *b0, cx<R> *b1, cx<R> *Y, int nvc, bool acc_last) {
    for (int k = k0; k < k1; ++k) {
        int pre = 1, post = nvc;
        for (int i = 0; i < k; ++i) pre *= o[i];
        for (int i = k + 1; i < d; ++i) post *= m[i];
        cx<R> *dst = (k == d - 1) ? Y : ((k & 1) ? b1 : b0);
        mode_pass<R>(src, dst, As[k], pre, m[k], o[k], post, acc_last && (k == d - 1));
        __syncthreads();
        src = dst;
    }
    return src;
}

template <class R>
TB_DEV void mode_chain(int d, const int *m, const int *o, cx<R> *const *As, const cx<R> *X, cx<R> *b0,
                       cx<R> *b1, cx<R> *Y, int nvc, bool acc_last) {
    mode_chain<R>(d, 0, d, m, o, As, X, b0, b1, Y, nvc, acc_last);
}

// First mode product of a source-leaf tile, read straight from the user tensor
// (gathered through the per-mode grid-index tables gt[k][b]) into dst.
template <class R>
TB_DEV void leaf_first_pass(int d, const int *m, const int *o, const cx<R> *A, const int *const *gt,
                            const int64_t *gstride, const cx<R> *__restrict__ user, int64_t nv, int64_t v0,
                            cx<R> *dst, int nvc) {
    int post = nvc;
    for (int i = 1; i < d; ++i) post *= m[i];
    const int mk = m[0], ok = o[0];
    const int nab = (ok + AB - 1) / AB;
    for (int it = threadIdx.x; it < nab * post; it += blockDim.x) {
        const int q = it % post, ab = it / post, a0 = ab * AB;
        int rq = q / nvc;
        const int v = q - rq * nvc;
        int64_t base = v0 + v;
        for (int k = d - 1; k >= 1; --k) {
            const int bk = rq % m[k];
            rq /= m[k];
            base += (int64_t)gt[k][bk] * gstride[k] * nv;
        }
        cx<R> c[AB];
#pragma unroll
        for (int i = 0; i < AB; ++i) c[i] = {R(0), R(0)};
        int acol[AB];
#pragma unroll
        for (int i = 0; i < AB; ++i) acol[i] = min(a0 + i, ok - 1);
        const int lda = lda_of(ok);
        for (int b = 0; b < mk; ++b) {
            const cx<R> x = user[base + (int64_t)gt[0][b] * gstride[0] * nv];
#pragma unroll
            for (int i = 0; i < AB; ++i) cmac(c[i], A[b * lda + acol[i]], x);
        }
#pragma unroll
        for (int i = 0; i < AB; ++i)
            if (a0 + i < ok) dst[(a0 + i) * post + q] = c[i];
    }
}

// Last mode product of a target-leaf tile, written straight to the user tensor
// (scattered through the grid-index tables).
template <class R>
TB_DEV void leaf_last_pass(int d, const int *m, const int *o, const cx<R> *A, const int *const *gt,
                           const int64_t *gstride, cx<R> *__restrict__ user, int64_t nv, int64_t v0,
                           const cx<R> *src, int nvc) {
    const int k = d - 1;
    int pre = 1;
    for (int i = 0; i < k; ++i) pre *= o[i];
    const int mk = m[k], ok = o[k], post = nvc;
    for (int it = threadIdx.x; it < pre * ok * post; it += blockDim.x) {
        const int v = it % post;
        const int r = it / post;
        const int a = r % ok, p = r / ok;
        cx<R> c = {R(0), R(0)};
        const cx<R> *s = src + p * mk * post + v;
        const int lda = lda_of(ok);
        for (int b = 0; b < mk; ++b) cmac(c, A[b * lda + a], s[b * post]);
        int64_t addr = (int64_t)gt[k][a] * gstride[k];
        int rp = p;
        for (int i = k - 1; i >= 0; --i) {
            const int ai = rp % o[i];
            rp /= o[i];
            addr += (int64_t)gt[i][ai] * gstride[i];
        }
        user[addr * nv + v0 + v] = c;
    }
}

// Raise a kernel's dynamic shared-memory limit once to the device maximum, so
// later launches (including those recorded into CUDA graphs) need no attribute
// calls.
cudaError_t set_smem_once(const void *fn, size_t smem) {
    static const void *done[64];
    static int ndone = 0;
    for (int i = 0; i < ndone; ++i)
        if (done[i] == fn) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    const int dyn_max = optin - (int)fa.sharedSizeBytes;   // static + dynamic <= opt-in limit
    if (smem > (size_t)dyn_max) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e == cudaSuccess && ndone < 64) done[ndone++] = fn;
    return e;
}

ChainSmem chain_smem(int d, const int *m, const int *o, int64_t nvc) {
    ChainSmem s{0, 0, 0, 0, 0};
    int64_t x = nvc, y = nvc;
    for (int k = 0; k < d; ++k) { x *= m[k]; y *= o[k]; }
    s.x = x;
    s.y = y;
    for (int k = 0; k + 1 < d; ++k) {
        int64_t t = nvc;
        for (int i = 0; i <= k; ++i) t *= o[i];
        for (int i = k + 1; i < d; ++i) t *= m[i];
        if (k & 1) s.b1 = s.b1 > t ? s.b1 : t;
        else s.b0 = s.b0 > t ? s.b0 : t;
    }
    for (int k = 0; k < d; ++k) s.a += (int64_t)m[k] * lda_of(o[k]);
    return s;
}

// Stage an r x c row-major factor block for a mode product that applies
// op(A) = A (o = r, m = c) or A^T (o = c, m = r), optionally conjugated, in
// the transposed layout dst[b * lda + a] = op(A)[a][b], lda = lda_of(o), with
// zero columns a in [o, lda).
template <class R>
TB_DEV void stage(cx<R> *dst, const cx<R> *__restrict__ src, int r, int c, bool trans, bool cj) {
    const int o = trans ? c : r, m = trans ? r : c, lda = lda_of(o);
    for (int e = threadIdx.x; e < m * lda; e += blockDim.x) {
        const int b = e / lda, a = e - b * lda;
        cx<R> v = {R(0), R(0)};
        if (a < o) {
            v = trans ? src[b * c + a] : src[a * c + b];
            if (cj) v.y = -v.y;
        }
        dst[e] = v;
    }
}

template <class R>
TB_DEV int64_t tile_index(const TileBuf<R> &b, int64_t F, int64_t M, int64_t sflat, int64_t nF, int d) {
    const int64_t blk = b.layout == 0 ? M * nF + F : F * b.nM + M;
    return (blk << (b.lgseg * d)) + sflat;
}

template <class R>
TB_DEV const cx<R> *fac_block(const FacRef<R> &f, int k, int64_t F, int64_t M, int sig, int d, int Lc) {
    int64_t j;
    if (!f.separable) j = ((F * f.nM + M) << f.lgseg) + sig;
    else {
        const int64_t Fk = (F >> (Lc * (d - 1 - k))) & ((1 << Lc) - 1);
        const int64_t Mk = (M >> (f.l * (d - 1 - k))) & ((1 << f.l) - 1);
        j = (((Fk << f.l) + Mk) << f.lgseg) + sig;
    }
    return f.A[k] + j * (int64_t)f.rows[k] * f.cols[k];
}

// ------------------------------------------------------------------ level pass
template <class R, Pass PASS, bool CONJ>
__global__ void __launch_bounds__(AP_THREADS, 2) k_level(const LevelArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R> *sm = reinterpret_cast<cx<R> *>(smraw);
    cx<R> *X = sm + a.offX, *B0 = sm + a.offB0, *B1 = sm + a.offB1, *Y = sm + a.offY, *Asm = sm + a.offA;
    const int d = a.d, Lc = a.Lc;
    // RHS chunks of one group are consecutive blocks, so the group's tiles are
    // re-read from L2 rather than DRAM when nv is split into several chunks
    const int64_t nch = (a.nv + a.nvc - 1) / a.nvc;
    const int64_t g = blockIdx.x / nch;
    const int64_t v0 = (int64_t)(blockIdx.x - g * nch) * a.nvc;
    const int nvc = (int)((a.nv - v0) < a.nvc ? (a.nv - v0) : a.nvc);
    const int tid = threadIdx.x;

    // segment tuple, multiset and mid-level block of this thread block
    const int lgs = (PASS == Pass::LeafIn || PASS == Pass::Split) ? a.out.lgseg : a.in.lgseg;
    const int64_t nsd = (int64_t)1 << (lgs * d);
    const int64_t sflat = g & (nsd - 1);
    const int64_t rest = g >> (lgs * d);
    int sig[MAXD];
    for (int k = 0; k < d; ++k) sig[k] = (int)((sflat >> (lgs * (d - 1 - k))) & ((1 << lgs) - 1));

    cx<R> *As[MAXD];
    {
        // staged factors: m x lda_of(o), with the factor block applied as is
        // (LeafIn, Split) or transposed (LeafOut, Gather)
        const bool tr = (PASS == Pass::LeafOut || PASS == Pass::Gather);
        int off = 0;
        for (int k = 0; k < d; ++k) {
            As[k] = Asm + off;
            const int ro = tr ? a.fac.cols[k] : a.fac.rows[k], rm = tr ? a.fac.rows[k] : a.fac.cols[k];
            off += rm * lda_of(ro);
        }
    }

    if (PASS == Pass::LeafIn || PASS == Pass::LeafOut) {
        const int64_t F = rest;
        // grid point of tile entry: axis k position F_k*nmid + sig_k*cb + b_k
        int m[MAXD], o[MAXD];
        for (int k = 0; k < d; ++k) {
            if (PASS == Pass::LeafIn) { m[k] = a.cb[k]; o[k] = a.out.R[k]; }
            else { m[k] = a.in.R[k]; o[k] = a.cb[k]; }
        }
        // grid index of leaf entry b along axis k
        __shared__ int gtab[MAXD][64];
        const int *gt[MAXD];
        for (int k = 0; k < d; ++k) {
            const int64_t Fk = (F >> (Lc * (d - 1 - k))) & ((1 << Lc) - 1);
            for (int b = tid; b < a.cb[k]; b += blockDim.x)
                gtab[k][b] = a.perm[k][Fk * a.nmid[k] + (int64_t)sig[k] * a.cb[k] + b];
            gt[k] = gtab[k];
            stage<R>(As[k], fac_block<R>(a.fac, k, F, 0, sig[k], d, Lc), a.fac.rows[k], a.fac.cols[k],
                     PASS == Pass::LeafOut, CONJ);
        }
        __syncthreads();
        if (PASS == Pass::LeafIn) {
            // pass 0 gathers from the user tensor; the leaf tile is never staged
            leaf_first_pass<R>(d, m, o, As[0], gt, a.user.gstride, a.user.p, a.nv, v0, d == 1 ? Y : B0, nvc);
            __syncthreads();
            mode_chain<R>(d, 1, d, m, o, As, B0, B0, B1, Y, nvc, false);
            const int64_t t = tile_index<R>(a.out, F, 0, sflat, a.nF, d);
            cx<R> *dst = a.out.p + t * a.out.tsize * a.nv + v0;
            for (int e = tid; e < a.out.tsize * nvc; e += blockDim.x) {
                const int v = e % nvc, b = e / nvc;
                dst[(int64_t)b * a.nv + v] = Y[e];
            }
        } else {
            const int64_t t = tile_index<R>(a.in, F, 0, sflat, a.nF, d);
            const cx<R> *src = a.in.p + t * a.in.tsize * a.nv + v0;
            for (int e = tid; e < a.in.tsize * nvc; e += blockDim.x) {
                const int v = e % nvc, b = e / nvc;
                X[e] = src[(int64_t)b * a.nv + v];
            }
            __syncthreads();
            // passes 0 .. d-2 in shared memory, the last one scatters to the user tensor
            const cx<R> *last = mode_chain<R>(d, 0, d - 1, m, o, As, X, B0, B1, Y, nvc, false);
            leaf_last_pass<R>(d, m, o, As[d - 1], gt, a.user.gstride, a.user.p, a.nv, v0, last, nvc);
        }
        return;
    }

    // Split / Gather: a group of 2^d tiles (F, multiset children of pM, sig)
    const int lvl = a.fac.l;                 // level of the factors (the finer multiset level)
    const int64_t nMp = (int64_t)1 << (d * (lvl - 1));
    const int64_t pM = rest % nMp, F = rest / nMp;
    int pMk[MAXD];
    for (int k = 0; k < d; ++k) pMk[k] = (int)((pM >> ((lvl - 1) * (d - 1 - k))) & ((1 << (lvl - 1)) - 1));
    const int nchild = 1 << d;

    if (PASS == Pass::Split) {
        // combined parent tile: dims 2 R'_k, child c of the parent segments at c_k R'_k
        int m[MAXD], o[MAXD];
        for (int k = 0; k < d; ++k) { m[k] = 2 * a.in.R[k]; o[k] = a.out.R[k]; }
        const int Tin = a.in.tsize;
        for (int e = tid; e < nchild * Tin * nvc; e += blockDim.x) {
            const int v = e % nvc;
            const int r = e / nvc;
            int b = r % Tin;
            const int c = r / Tin;
            int64_t sp = 0;
            int comb = 0, stride = 1;
            for (int k = d - 1; k >= 0; --k) {
                const int bk = b % a.in.R[k];
                b /= a.in.R[k];
                const int ck = (c >> (d - 1 - k)) & 1;
                comb += (ck * a.in.R[k] + bk) * stride;
                stride *= m[k];
            }
            for (int k = 0; k < d; ++k) sp = (sp << (lgs + 1)) | (2 * sig[k] + ((c >> (d - 1 - k)) & 1));
            const int64_t t = tile_index<R>(a.in, F, pM, sp, a.nF, d);
            const int bb = r % Tin;
            X[comb * nvc + v] = a.in.p[(t * Tin + bb) * a.nv + v0 + v];
        }
        for (int c = 0; c < nchild; ++c) {
            int64_t M = 0;
            for (int k = 0; k < d; ++k) M = (M << lvl) | (2 * pMk[k] + ((c >> (d - 1 - k)) & 1));
            for (int k = 0; k < d; ++k)
                stage<R>(As[k], fac_block<R>(a.fac, k, F, M, sig[k], d, Lc), a.fac.rows[k], a.fac.cols[k], false, CONJ);
            __syncthreads();
            mode_chain<R>(d, m, o, As, X, B0, B1, Y, nvc, false);
            const int64_t t = tile_index<R>(a.out, F, M, sflat, a.nF, d);
            cx<R> *dst = a.out.p + t * a.out.tsize * a.nv + v0;
            for (int e = tid; e < a.out.tsize * nvc; e += blockDim.x) {
                const int v = e % nvc, b = e / nvc;
                dst[(int64_t)b * a.nv + v] = Y[e];
            }
            __syncthreads();
        }
    } else {   // Gather
        int m[MAXD], o[MAXD];
        for (int k = 0; k < d; ++k) { m[k] = a.in.R[k]; o[k] = 2 * a.out.R[k]; }
        for (int c = 0; c < nchild; ++c) {
            int64_t M = 0;
            for (int k = 0; k < d; ++k) M = (M << lvl) | (2 * pMk[k] + ((c >> (d - 1 - k)) & 1));
            const int64_t t = tile_index<R>(a.in, F, M, sflat, a.nF, d);
            const cx<R> *src = a.in.p + t * a.in.tsize * a.nv + v0;
            for (int e = tid; e < a.in.tsize * nvc; e += blockDim.x) {
                const int v = e % nvc, b = e / nvc;
                X[e] = src[(int64_t)b * a.nv + v];
            }
            for (int k = 0; k < d; ++k)
                stage<R>(As[k], fac_block<R>(a.fac, k, F, M, sig[k], d, Lc), a.fac.rows[k], a.fac.cols[k], true, CONJ);
            __syncthreads();
            mode_chain<R>(d, m, o, As, X, B0, B1, Y, nvc, c > 0);
        }
        // scatter the combined output to the 2^d tiles (F, pM, 2 sig + e) one level up
        const int Tout = a.out.tsize;
        for (int e = tid; e < nchild * Tout * nvc; e += blockDim.x) {
            const int v = e % nvc;
            const int r = e / nvc;
            int b = r % Tout;
            const int c = r / Tout;
            int comb = 0, stride = 1;
            for (int k = d - 1; k >= 0; --k) {
                const int bk = b % a.out.R[k];
                b /= a.out.R[k];
                const int ck = (c >> (d - 1 - k)) & 1;
                comb += (ck * a.out.R[k] + bk) * stride;
                stride *= o[k];
            }
            int64_t sp = 0;
            for (int k = 0; k < d; ++k) sp = (sp << (lgs + 1)) | (2 * sig[k] + ((c >> (d - 1 - k)) & 1));
            const int64_t t = tile_index<R>(a.out, F, pM, sp, a.nF, d);
            a.out.p[(t * Tout + (r % Tout)) * a.nv + v0 + v] = Y[comb * nvc + v];
        }
    }
}

template <class R>
cudaError_t launch_level(Pass pass, bool conj, const LevelArgs<R> &a, cudaStream_t st) {
    const int64_t nchunks = (a.nv + a.nvc - 1) / a.nvc;
    dim3 grid((unsigned)(a.nblocks * nchunks));
    void (*fn)(const LevelArgs<R>) = nullptr;
#define TB_PICK(P)                                                  \
    fn = conj ? k_level<R, P, true> : k_level<R, P, false>;
    switch (pass) {
        case Pass::LeafIn: TB_PICK(Pass::LeafIn) break;
        case Pass::Split: TB_PICK(Pass::Split) break;
        case Pass::Gather: TB_PICK(Pass::Gather) break;
        case Pass::LeafOut: TB_PICK(Pass::LeafOut) break;
    }
#undef TB_PICK
    cudaError_t e = set_smem_once((const void *)fn, a.smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, AP_THREADS, a.smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- dense core
// Forward: G_{t,s}[a] = sum_b C[a][b] F_{t,s}[b] on compact core indices; a warp
// per core row, lanes over b, warp-shuffle reduction.  Adjoint: thread per b.
template <class R, int NVC>
__global__ void __launch_bounds__(CORE_THREADS) k_core_dense(const CoreApplyArgs<R> a, int adjoint) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R> *Xc = reinterpret_cast<cx<R> *>(smraw);
    const int d = a.d;
    const int64_t nch = (a.nv + a.nvc - 1) / a.nvc;
    const int64_t p = blockIdx.x / nch;
    const int64_t v0 = (int64_t)(blockIdx.x - p * nch) * a.nvc;
    const int nvc = (int)((a.nv - v0) < a.nvc ? (a.nv - v0) : a.nvc);
    int rt[MAXD], rs[MAXD];
    int Mt = 1, Ms = 1;
    for (int k = 0; k < d; ++k) {
        rt[k] = a.dims[p * 2 * d + k];
        rs[k] = a.dims[p * 2 * d + d + k];
        Mt *= rt[k];
        Ms *= rs[k];
    }
    const cx<R> *C = a.core + a.off[p];
    // forward: in = source tile (dims in.R, compact rs), out = target tile (dims out.R, compact rt)
    const int *rin = adjoint ? rt : rs;
    const int *rout = adjoint ? rs : rt;
    const int Min = adjoint ? Mt : Ms, Mout = adjoint ? Ms : Mt;
    const cx<R> *src = a.in.p + p * a.in.tsize * a.nv + v0;
    cx<R> *dst = a.out.p + p * a.out.tsize * a.nv + v0;
    for (int e = threadIdx.x; e < Min * nvc; e += blockDim.x) {
        const int v = e % nvc;
        int b = e / nvc, pos = 0, stride = 1;
        for (int k = d - 1; k >= 0; --k) {
            pos += (b % rin[k]) * stride;
            b /= rin[k];
            stride *= a.in.R[k];
        }
        Xc[e] = src[(int64_t)pos * a.nv + v];
    }
    for (int e = threadIdx.x; e < a.out.tsize * nvc; e += blockDim.x) {
        const int v = e % nvc, b = e / nvc;
        dst[(int64_t)b * a.nv + v] = {R(0), R(0)};
    }
    __syncthreads();
    auto outpos = [&](int idx) {
        int pos = 0, stride = 1;
        for (int k = d - 1; k >= 0; --k) {
            pos += (idx % rout[k]) * stride;
            idx /= rout[k];
            stride *= a.out.R[k];
        }
        return pos;
    };
    if (!adjoint) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int row = warp; row < Mout; row += nw) {
            cx<R> acc[NVC];
#pragma unroll
            for (int v = 0; v < NVC; ++v) acc[v] = {R(0), R(0)};
            const cx<R> *Crow = C + (int64_t)row * Ms;
            for (int b = lane; b < Ms; b += 32) {
                const cx<R> c = Crow[b];
#pragma unroll
                for (int v = 0; v < NVC; ++v)
                    if (v < nvc) cmac(acc[v], c, Xc[b * nvc + v]);
            }
#pragma unroll
            for (int v = 0; v < NVC; ++v) {
                for (int o = 16; o > 0; o >>= 1) {
                    acc[v].x += __shfl_xor_sync(0xffffffffu, acc[v].x, o);
                    acc[v].y += __shfl_xor_sync(0xffffffffu, acc[v].y, o);
                }
            }
            if (lane == 0) {
                const int pos = outpos(row);
#pragma unroll
                for (int v = 0; v < NVC; ++v)
                    if (v < nvc) dst[(int64_t)pos * a.nv + v] = acc[v];
            }
        }
    } else {
        for (int col = threadIdx.x; col < Mout; col += blockDim.x) {
            cx<R> acc[NVC];
#pragma unroll
            for (int v = 0; v < NVC; ++v) acc[v] = {R(0), R(0)};
            for (int row = 0; row < Min; ++row) {
                const cx<R> c = C[(int64_t)row * Ms + col];
#pragma unroll
                for (int v = 0; v < NVC; ++v)
                    if (v < nvc) cmac_conj(acc[v], c, Xc[row * nvc + v]);
            }
            const int pos = outpos(col);
#pragma unroll
            for (int v = 0; v < NVC; ++v)
                if (v < nvc) dst[(int64_t)pos * a.nv + v] = acc[v];
        }
    }
}

template <class R>
cudaError_t launch_core_dense(bool adjoint, const CoreApplyArgs<R> &a, cudaStream_t st) {
    const int64_t nchunks = (a.nv + a.nvc - 1) / a.nvc;
    dim3 grid((unsigned)(a.P * nchunks));
    void (*fn)(const CoreApplyArgs<R>, int);
    if (a.nvc <= 1) fn = k_core_dense<R, 1>;
    else if (a.nvc <= 4) fn = k_core_dense<R, 4>;
    else if (a.nvc <= 8) fn = k_core_dense<R, 8>;
    else fn = k_core_dense<R, 16>;
    cudaError_t e = set_smem_once((const void *)fn, a.smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, CORE_THREADS, a.smem, st>>>(a, adjoint ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------ Kronecker core
// For a kernel that is a product over modes, K(t-bar, s-bar) = kron_k K_k and the
// core contraction is a mode-product chain with the per-mode factors.
template <class R, bool ADJ>
__global__ void __launch_bounds__(CORE_THREADS) k_core_kron(const CoreApplyArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R> *sm = reinterpret_cast<cx<R> *>(smraw);
    cx<R> *X = sm + a.offX, *B0 = sm + a.offB0, *B1 = sm + a.offB1, *Y = sm + a.offY, *Asm = sm + a.offA;
    const int d = a.d;
    const int64_t nch = (a.nv + a.nvc - 1) / a.nvc;
    const int64_t p = blockIdx.x / nch;
    const int64_t v0 = (int64_t)(blockIdx.x - p * nch) * a.nvc;
    const int nvc = (int)((a.nv - v0) < a.nvc ? (a.nv - v0) : a.nvc);
    const int64_t nb = (int64_t)1 << a.Lc;
    const int64_t nF = (int64_t)1 << (a.Lc * d);
    const int64_t t = p / nF, s = p % nF;
    int m[MAXD], o[MAXD];
    cx<R> *As[MAXD];
    int off = 0;
    for (int k = 0; k < d; ++k) {
        m[k] = ADJ ? a.Rt[k] : a.Rs[k];
        o[k] = ADJ ? a.Rs[k] : a.Rt[k];
        As[k] = Asm + off;
        off += m[k] * lda_of(o[k]);
        const int64_t tk = (t >> (a.Lc * (d - 1 - k))) & (nb - 1), sk = (s >> (a.Lc * (d - 1 - k))) & (nb - 1);
        stage<R>(As[k], a.kron[k] + (tk * nb + sk) * a.Rt[k] * a.Rs[k], a.Rt[k], a.Rs[k], ADJ, ADJ);
    }
    const cx<R> *src = a.in.p + p * a.in.tsize * a.nv + v0;
    for (int e = threadIdx.x; e < a.in.tsize * nvc; e += blockDim.x) {
        const int v = e % nvc, b = e / nvc;
        X[e] = src[(int64_t)b * a.nv + v];
    }
    __syncthreads();
    mode_chain<R>(d, m, o, As, X, B0, B1, Y, nvc, false);
    cx<R> *dst = a.out.p + p * a.out.tsize * a.nv + v0;
    for (int e = threadIdx.x; e < a.out.tsize * nvc; e += blockDim.x) {
        const int v = e % nvc, b = e / nvc;
        dst[(int64_t)b * a.nv + v] = Y[e];
    }
}

template <class R>
cudaError_t launch_core_kron(bool adjoint, const CoreApplyArgs<R> &a, cudaStream_t st) {
    const int64_t nchunks = (a.nv + a.nvc - 1) / a.nvc;
    dim3 grid((unsigned)(a.P * nchunks));
    void (*fn)(const CoreApplyArgs<R>) = adjoint ? k_core_kron<R, true> : k_core_kron<R, false>;
    cudaError_t e = set_smem_once((const void *)fn, a.smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, CORE_THREADS, a.smem, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_level<float>(Pass, bool, const LevelArgs<float> &, cudaStream_t);
template cudaError_t launch_level<double>(Pass, bool, const LevelArgs<double> &, cudaStream_t);
template cudaError_t launch_core_dense<float>(bool, const CoreApplyArgs<float> &, cudaStream_t);
template cudaError_t launch_core_dense<double>(bool, const CoreApplyArgs<double> &, cudaStream_t);
template cudaError_t launch_core_kron<float>(bool, const CoreApplyArgs<float> &, cudaStream_t);
template cudaError_t launch_core_kron<double>(bool, const CoreApplyArgs<double> &, cudaStream_t);

}  // namespace tb

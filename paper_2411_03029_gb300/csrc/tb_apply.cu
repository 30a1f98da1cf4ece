// Mid-level core contraction on CUDA cores (Alg. 2, step 2):
//   G_{t,s} = K(t-bar, s-bar) x_{d+1..2d} F_{t,s}
// for the complex128 / complex64 apply precisions (the split-BF16 tensor-core
// form lives in tb_core_tc.cu), in two forms: a dense core per pair (t, s)
// stored with compact ranks, and, for kernels that are a product over modes,
// the Kronecker form K = kron_k K_k applied as a mode-product chain on a tile
// staged in shared memory.  The adjoint uses K(t-bar, s-bar)^H.
//
// The level passes (Alg. 2, steps 1 and 3) run as per-mode launches in
// tb_mode.cu.
#include "tb_kernels.cuh"

namespace tb {

constexpr int CORE_THREADS = 256;

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
// column pair and 8 complex FMAs.  Needs post even and 16-byte aligned src / At.
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
        const cx<R> *arow = At + a0;
#pragma unroll 4
        for (int b = 0; b < mk; ++b) {
            cx<R> x0, x1, av[4];
            ld2(s, x0, x1);
            ld2(arow, av[0], av[1]);
            ld2(arow + 2, av[2], av[3]);
            s += post;
            arow += lda;
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
    {
        const int64_t nF = (int64_t)1 << (a.Lc * d);
        const int64_t f = adjoint ? p / nF : p % nF;   // the pair's input-side multiset
        if (f < a.pf0 || f >= a.pf1) return;
    }
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

// Forward core for one right-hand side, complex64: G_{t,s}[a] = sum_b C[a][b] F_{t,s}[b].
// A warp takes CR_ROWS core rows at a time; lane l takes columns l, l + 32, ..
// and accumulates all CR_ROWS rows, reading each row coalesced (32 consecutive
// entries per load, CR_ROWS independent loads in flight per lane).  A
// transposed butterfly reduction (CR_ROWS - 1 exchanges per component within
// each half-warp, then one across the halves) leaves row r0 + l's sum in lanes
// l and l + 16.  Columns of a row are summed in the same order for every row:
// deterministic.
constexpr int CR_ROWS = 16;

template <class R>
__global__ void __launch_bounds__(CORE_THREADS, 3) k_core_rows(const CoreApplyArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R> *Xc = reinterpret_cast<cx<R> *>(smraw);
    const int d = a.d;
    const int64_t p = blockIdx.x;
    {
        const int64_t f = p % ((int64_t)1 << (a.Lc * d));   // the pair's source multiset
        if (f < a.pf0 || f >= a.pf1) return;
    }
    int rt[MAXD], rs[MAXD];
    int Mt = 1, Ms = 1;
    for (int k = 0; k < d; ++k) {
        rt[k] = a.dims[p * 2 * d + k];
        rs[k] = a.dims[p * 2 * d + d + k];
        Mt *= rt[k];
        Ms *= rs[k];
    }
    const cx<R> *C = a.core + a.off[p];
    const cx<R> *src = a.in.p + p * a.in.tsize * a.nv;
    cx<R> *dst = a.out.p + p * a.out.tsize * a.nv;
    for (int b = threadIdx.x; b < Ms; b += blockDim.x) {
        int q = b, pos = 0, stride = 1;
        for (int k = d - 1; k >= 0; --k) {
            pos += (q % rs[k]) * stride;
            q /= rs[k];
            stride *= a.in.R[k];
        }
        Xc[b] = src[(int64_t)pos * a.nv];
    }
    for (int e = threadIdx.x; e < a.out.tsize; e += blockDim.x) dst[(int64_t)e * a.nv] = {R(0), R(0)};
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nk = (Ms + 31) >> 5;
    for (int r0 = warp * CR_ROWS; r0 < Mt; r0 += nw * CR_ROWS) {
        cx<R> acc[CR_ROWS];
#pragma unroll
        for (int j = 0; j < CR_ROWS; ++j) acc[j] = {R(0), R(0)};
        const int nr = Mt - r0 < CR_ROWS ? Mt - r0 : CR_ROWS;
        for (int k = 0; k < nk; ++k) {
            const int b = lane + 32 * k;
            const bool live = b < Ms;
            const cx<R> *col = C + (int64_t)r0 * Ms + b;
            const cx<R> xk = live ? Xc[b] : cx<R>{R(0), R(0)};
            cx<R> c[CR_ROWS];
#pragma unroll
            for (int j = 0; j < CR_ROWS; ++j) {
                // the core is read once per apply: streaming loads (evict first)
                float2 v = make_float2(0.f, 0.f);
                if (live && j < nr) v = __ldcs(reinterpret_cast<const float2 *>(col + (int64_t)j * Ms));
                c[j] = cx<R>{v.x, v.y};
            }
#pragma unroll
            for (int j = 0; j < CR_ROWS; ++j) cmac(acc[j], c[j], xk);
        }
        // transposed reduction within each half-warp: after the step with offset
        // o, lane l keeps the partial sums of the rows whose bit o equals lane bit o
#pragma unroll
        for (int o = CR_ROWS / 2; o >= 1; o >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int j = 0; j < o; ++j) {
                const cx<R> send = up ? acc[j] : acc[j + o];
                const cx<R> keep = up ? acc[j + o] : acc[j];
                cx<R> got;
                got.x = __shfl_xor_sync(0xffffffffu, send.x, o);
                got.y = __shfl_xor_sync(0xffffffffu, send.y, o);
                acc[j] = {keep.x + got.x, keep.y + got.y};
            }
        }
        acc[0].x += __shfl_xor_sync(0xffffffffu, acc[0].x, 16);
        acc[0].y += __shfl_xor_sync(0xffffffffu, acc[0].y, 16);
        if (lane < nr) {
            int q = r0 + lane, pos = 0, stride = 1;
            for (int k = d - 1; k >= 0; --k) {
                pos += (q % rt[k]) * stride;
                q /= rt[k];
                stride *= a.out.R[k];
            }
            dst[(int64_t)pos * a.nv] = acc[0];
        }
    }
}

// Forward core for one RHS with the entries of K(t-bar, s-bar) evaluated on
// the fly (no core bytes read), same row batches and reduction as k_core_rows.
// The block builds per-row and per-column tables of the pair's skeleton points
// (integer grid coordinates, and for the Radon kernel c(x) and |xi| as FP32
// double-floats from FP64), then each entry costs integer arithmetic, one
// residual-corrected sqrt and one sincospif:
//   sqrt(D) = s + (D - s^2) / (2 s)  (D an exact integer in FP32, the residual by FMA),
//   phase = cyc (s + s_lo) as a double-float product (Dekker: p = c s and its
//   exact error fma(c, s, -p)), reduced to (-1/2, 1/2] cycles before sincospif.
template <int KIND>
__global__ void __launch_bounds__(CORE_THREADS, 3) k_core_regen(const CoreApplyArgs<float> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int d = a.d;
    const int64_t p = blockIdx.x;
    {
        const int64_t f = p % ((int64_t)1 << (a.Lc * d));   // the pair's source multiset
        if (f < a.pf0 || f >= a.pf1) return;
    }
    int rt[MAXD], rs[MAXD];
    int Mt = 1, Ms = 1;
    for (int k = 0; k < d; ++k) {
        rt[k] = a.dims[p * 2 * d + k];
        rs[k] = a.dims[p * 2 * d + d + k];
        Mt *= rt[k];
        Ms *= rs[k];
    }
    // shared tables: X (Ms), column ints (Ms x d), column float pair (Ms), row ints (Mt x d), row float pair (Mt)
    cx<float> *Xc = reinterpret_cast<cx<float> *>(smraw);
    float2 *colf = reinterpret_cast<float2 *>(Xc + a.offX);
    float2 *rowf = colf + a.offX;
    int *coli = reinterpret_cast<int *>(rowf + a.offB0);
    int *rowi = coli + (int64_t)a.offX * d;
    const CoreRegen &g = a.rg;
    const int64_t t = p / g.nF, s = p - t * g.nF;
    const int64_t jt = t * g.nF + s, js = s * g.nF + t;
    const cx<float> *src = a.in.p + p * a.in.tsize * a.nv;
    cx<float> *dst = a.out.p + p * a.out.tsize * a.nv;
    for (int b = threadIdx.x; b < Ms; b += blockDim.x) {
        int q = b, pos = 0, stride = 1;
        double xx = 0.0;
        for (int k = d - 1; k >= 0; --k) {
            const int bk = q % rs[k];
            q /= rs[k];
            pos += bk * stride;
            stride *= a.in.R[k];
            const int j = g.sskel[k][js * g.scap[k] + bk];
            const int v = KIND == TB_KERNEL_HELMHOLTZ ? j + g.off[k] : j + g.xi0[k];
            coli[(int64_t)b * d + k] = v;
            xx += (double)v * v;
        }
        Xc[b] = src[(int64_t)pos * a.nv];
        if (KIND == TB_KERNEL_RADON) {
            const double nr = sqrt(xx);
            const float hi = (float)nr;
            colf[b] = make_float2(hi, (float)(nr - hi));
        }
    }
    for (int r = threadIdx.x; r < Mt; r += blockDim.x) {
        int q = r;
        double sp = 1.0;
        for (int k = d - 1; k >= 0; --k) {
            const int ak = q % rt[k];
            q /= rt[k];
            const int i = g.tskel[k][jt * g.tcap[k] + ak];
            rowi[(int64_t)r * d + k] = i;
            if (KIND == TB_KERNEL_RADON) sp *= sinpi(2.0 * g.xs[k][i]);
        }
        if (KIND == TB_KERNEL_RADON) {
            const double c = g.ra + g.rb * sp;
            const float hi = (float)c;
            rowf[r] = make_float2(hi, (float)(c - hi));
        }
    }
    for (int e = threadIdx.x; e < a.out.tsize; e += blockDim.x) dst[(int64_t)e * a.nv] = {0.f, 0.f};
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nk = (Ms + 31) >> 5;
    for (int r0 = warp * CR_ROWS; r0 < Mt; r0 += nw * CR_ROWS) {
        cx<float> acc[CR_ROWS];
#pragma unroll
        for (int j = 0; j < CR_ROWS; ++j) acc[j] = {0.f, 0.f};
        const int nr = Mt - r0 < CR_ROWS ? Mt - r0 : CR_ROWS;
        for (int k = 0; k < nk; ++k) {
            const int b = lane + 32 * k;
            const bool live = b < Ms;
            const int bb = live ? b : 0;
            const cx<float> xk = live ? Xc[b] : cx<float>{0.f, 0.f};
            int cj[MAXD];
            for (int m = 0; m < d; ++m) cj[m] = coli[(int64_t)bb * d + m];
            const float2 cf = KIND == TB_KERNEL_RADON ? colf[bb] : make_float2(0.f, 0.f);
#pragma unroll 4
            for (int j = 0; j < CR_ROWS; ++j) {
                if (j >= nr) break;
                const int r = r0 + j;
                float sn, cs, amp = 1.f;
                if (KIND == TB_KERNEL_HELMHOLTZ) {
                    int D = g.hp2;
                    for (int m = 0; m < d; ++m) {
                        const int dd = rowi[(int64_t)r * d + m] - cj[m];
                        D += dd * dd;
                    }
                    const float Df = (float)D;
                    const float sq = sqrtf(Df);
                    const float slo = fmaf(-sq, sq, Df) / (2.f * sq);
                    const float ph = g.cyc_hi * sq;
                    const float er = fmaf(g.cyc_hi, sq, -ph);
                    const float lo = fmaf(g.cyc_hi, slo, fmaf(g.cyc_lo, sq, er));
                    const float f = (ph - rintf(ph)) + lo;
                    sincospif(2.f * f, &sn, &cs);
                    amp = g.inv_h / sq;
                } else {
                    int num = 0;
                    for (int m = 0; m < d; ++m) num += rowi[(int64_t)r * d + m] * cj[m];
                    int md = num % g.n;
                    if (md < 0) md += g.n;
                    const float f1 = (float)md / (float)g.n;
                    const float2 rc = rowf[r];
                    const float ph = rc.x * cf.x;
                    const float er = fmaf(rc.x, cf.x, -ph);
                    const float lo = fmaf(rc.x, cf.y, fmaf(rc.y, cf.x, er));
                    float f = f1 + ((ph - rintf(ph)) + lo);
                    f -= rintf(f);
                    sincospif(2.f * f, &sn, &cs);
                }
                const cx<float> kv = {live ? cs * amp : 0.f, live ? sn * amp : 0.f};
                cmac(acc[j], kv, xk);
            }
        }
#pragma unroll
        for (int o = CR_ROWS / 2; o >= 1; o >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int j = 0; j < o; ++j) {
                const cx<float> send = up ? acc[j] : acc[j + o];
                const cx<float> keep = up ? acc[j + o] : acc[j];
                cx<float> got;
                got.x = __shfl_xor_sync(0xffffffffu, send.x, o);
                got.y = __shfl_xor_sync(0xffffffffu, send.y, o);
                acc[j] = {keep.x + got.x, keep.y + got.y};
            }
        }
        acc[0].x += __shfl_xor_sync(0xffffffffu, acc[0].x, 16);
        acc[0].y += __shfl_xor_sync(0xffffffffu, acc[0].y, 16);
        if (lane < nr) {
            int q = r0 + lane, pos = 0, stride = 1;
            for (int k = d - 1; k >= 0; --k) {
                pos += (q % rt[k]) * stride;
                q /= rt[k];
                stride *= a.out.R[k];
            }
            dst[(int64_t)pos * a.nv] = acc[0];
        }
    }
}

cudaError_t launch_core_regen(const CoreApplyArgs<float> &a, cudaStream_t st) {
    void (*fn)(const CoreApplyArgs<float>) = nullptr;
    if (a.rg.kind == TB_KERNEL_HELMHOLTZ) fn = k_core_regen<TB_KERNEL_HELMHOLTZ>;
    else if (a.rg.kind == TB_KERNEL_RADON) fn = k_core_regen<TB_KERNEL_RADON>;
    else return cudaErrorInvalidValue;
    cudaError_t e = set_smem_once((const void *)fn, a.smem);
    if (e != cudaSuccess) return e;
    fn<<<(unsigned)a.P, CORE_THREADS, a.smem, st>>>(a);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_core_rows(const CoreApplyArgs<R> &a, cudaStream_t st) {
    cudaError_t e = set_smem_once((const void *)k_core_rows<R>, a.smem);
    if (e != cudaSuccess) return e;
    k_core_rows<R><<<(unsigned)a.P, CORE_THREADS, a.smem, st>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_core_rows<float>(const CoreApplyArgs<float> &, cudaStream_t);

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

template cudaError_t launch_core_dense<float>(bool, const CoreApplyArgs<float> &, cudaStream_t);
template cudaError_t launch_core_dense<double>(bool, const CoreApplyArgs<double> &, cudaStream_t);
template cudaError_t launch_core_kron<float>(bool, const CoreApplyArgs<float> &, cudaStream_t);
template cudaError_t launch_core_kron<double>(bool, const CoreApplyArgs<double> &, cudaStream_t);

}  // namespace tb

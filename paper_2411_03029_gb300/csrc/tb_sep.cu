// Apply of a separable tensor butterfly (kernel = product of per-mode
// factors, e.g. the Fourier kernel of Sec. 3.2.1 / 4.3).
//
// With separable factors (see the separable reading of Eqs. tensorID_BF_V /
// transfer W in the construction) every transfer, interpolation and core block
// acts on one mode, so the tensor butterfly of Eq. (butterfly_tensor) is the
// tensor product over modes of 1-D butterfly chains
//     B_k = U_k P_k,1 .. P_k,Lc  K_k  W_k,Lc .. W_k,1 V_k ,
// and u = f x_1 B_1 x_2 ... x_d B_d.  Each step is a small sparse matrix (CSR)
// on the 1-D index of its mode.  Three forms apply the chains:
//   - k_sep_pass: a thread block stages a tile that holds complete fibers
//     along a few consecutive modes (and a contiguous run of the trailing
//     modes and right-hand sides) and applies those modes' steps one after
//     another in shared memory;
//   - k_sep_fiber: one pass per mode, each thread's fiber in a shared-memory
//     column, the steps as packed nonzero streams;
//   - k_sep_regf / k_sep_reg / k_sep_reg2: one pass per mode (or per pair of
//     modes) with the fibers in registers, for modes whose ranks equal the
//     leaf size, where every step is a compile-time pattern of dense blocks
//     (sepr_col) and V, U^T fold into the load and store positions.
#include "tb_kernels.cuh"

namespace tb {

constexpr int SEP_THREADS = 256;

template <class R>
__global__ void __launch_bounds__(SEP_THREADS) k_sep_pass(const SepPassArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R> *A = reinterpret_cast<cx<R> *>(smraw);
    cx<R> *B = A + a.buf;
    const int64_t blk = blockIdx.x;
    const int64_t o = blk / a.nchunks, ch = blk - o * a.nchunks;
    const int64_t i0 = ch * a.ic;
    const int ic = (int)((a.inner - i0) < a.ic ? (a.inner - i0) : a.ic);
    int ext[MAXD];
    int64_t P = 1;
    for (int k = a.k0; k <= a.k1; ++k) {
        ext[k] = a.n[k];
        P *= a.n[k];
    }
    const cx<R> *src = a.in + o * P * a.inner + i0;
    for (int64_t e = threadIdx.x; e < P * ic; e += blockDim.x) {
        const int64_t p = e / ic, i = e - p * ic;
        A[e] = src[p * a.inner + i];
    }
    __syncthreads();
    for (int k = a.k0; k <= a.k1; ++k) {
        for (int s = 0; s < a.nsteps[k]; ++s) {
            const SepStep<R> S = a.steps[a.step0[k] + s];
            int pre = 1, post = ic;
            for (int j = a.k0; j < k; ++j) pre *= ext[j];
            for (int j = k + 1; j <= a.k1; ++j) post *= ext[j];
            const int items = pre * S.n_out * post;
            for (int it = threadIdx.x; it < items; it += blockDim.x) {
                const int q = it % post;
                const int r2 = it / post;
                const int r = r2 % S.n_out, p = r2 / S.n_out;
                cx<R> acc = {R(0), R(0)};
                const int j1 = S.rowptr[r + 1];
                const cx<R> *row = A + (p * S.n_in) * post + q;
                for (int j = S.rowptr[r]; j < j1; ++j) cmac(acc, S.val[j], row[S.col[j] * post]);
                B[(p * S.n_out + r) * post + q] = acc;
            }
            __syncthreads();
            cx<R> *t = A;
            A = B;
            B = t;
            ext[k] = S.n_out;
        }
    }
    cx<R> *dst = a.out + o * P * a.inner + i0;
    for (int64_t e = threadIdx.x; e < P * ic; e += blockDim.x) {
        const int64_t p = e / ic, i = e - p * ic;
        dst[p * a.inner + i] = A[e];
    }
}

template <class R>
cudaError_t launch_sep_pass(const SepPassArgs<R> &a, cudaStream_t st) {
    cudaError_t e = set_smem_once((const void *)k_sep_pass<R>, a.smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = a.outer * a.nchunks;
    k_sep_pass<R><<<(unsigned)blocks, SEP_THREADS, a.smem, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_sep_pass<float>(const SepPassArgs<float> &, cudaStream_t);
template cudaError_t launch_sep_pass<double>(const SepPassArgs<double> &, cudaStream_t);

// Thread-per-fiber form: each thread owns one (fiber along mode k, RHS) pair
// and keeps the fiber in its own column of two shared buffers (column-major
// per thread: entry e of thread t at e * T + t, conflict-free), so the steps
// of the chain need no block-wide synchronisation.  Each step runs as its
// packed row-ordered nonzero stream (value, column, end of row), copied to
// shared memory with the column pre-scaled by T and read as broadcasts: one
// 16-byte load, one operand load and four FMAs per nonzero.
template <class R>
__global__ void k_sep_fiber(const SepFiberArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int T = blockDim.x, t = threadIdx.x;
    cx<R> *b0 = reinterpret_cast<cx<R> *>(smraw);
    cx<R> *b1 = b0 + (size_t)a.maxext * T;
    SepNz<R> *spk = reinterpret_cast<SepNz<R> *>(b1 + (size_t)a.maxext * T);
    __shared__ int s_po[40];   // per-step offsets into spk
    if (t == 0) {
        int po = 0;
        for (int s = 0; s < a.nsteps; ++s) {
            s_po[s] = po;
            po += a.steps[s].npk;
        }
    }
    __syncthreads();
    for (int s = 0; s < a.nsteps; ++s) {
        const SepStep<R> S = a.steps[s];
        for (int i = t; i < S.npk; i += T) {
            SepNz<R> e = S.nz[i];
            e.col *= T;
            spk[s_po[s] + i] = e;
        }
    }
    __syncthreads();
    const int64_t gid = (int64_t)blockIdx.x * T + t;
    const bool live = gid < a.outer * a.inner;
    const int64_t o = live ? gid / a.inner : 0, q = live ? gid - o * a.inner : 0;
    const int64_t base = o * a.nk * a.inner + q;
    if (live)
        for (int i = 0; i < a.nk; ++i) b0[i * T + t] = a.in[base + (int64_t)i * a.inner];
    cx<R> *src = b0 + t, *dst = b1 + t;
    for (int s = 0; s < a.nsteps; ++s) {
        const SepNz<R> *P = spk + s_po[s];
        const int n = a.steps[s].npk;
        cx<R> acc = {R(0), R(0)};
        cx<R> *dp = dst;
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            const SepNz<R> e = P[j];
            cmac(acc, e.v, src[e.col]);
            if (e.last) {
                *dp = acc;
                dp += T;
                acc = {R(0), R(0)};
            }
        }
        cx<R> *tmp = src;
        src = dst;
        dst = tmp;
    }
    if (live)
        for (int i = 0; i < a.nk; ++i) a.out[base + (int64_t)i * a.inner] = src[i * T];
}

template <class R>
cudaError_t launch_sep_fiber(const SepFiberArgs<R> &a, cudaStream_t st) {
    cudaError_t e = set_smem_once((const void *)k_sep_fiber<R>, a.smem);
    if (e != cudaSuccess) return e;
    const int64_t total = a.outer * a.inner;
    const int64_t blocks = (total + a.threads - 1) / a.threads;
    k_sep_fiber<R><<<(unsigned)blocks, a.threads, a.smem, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_sep_fiber<float>(const SepFiberArgs<float> &, cudaStream_t);
template cudaError_t launch_sep_fiber<double>(const SepFiberArgs<double> &, cudaStream_t);

// Register-resident chain of one mode (ranks equal to the leaf size; see
// sepr_col).  One thread owns one fiber (o, q) at a time: it loads the N
// entries through the load positions (tree order and the permutation V),
// applies the dense-block steps with the fiber in registers and the step
// coefficients read from shared memory as warp-wide broadcasts, and stores
// through the store positions (U^T and tree order).  The adjoint applies the
// conjugate-transposed steps in reverse, scattering into its output registers;
// load and store positions swap roles.  Threads walk the fibers with a grid
// stride, and when N <= 16 the next fiber's loads are issued before the
// current fiber's arithmetic.
constexpr int SEPR_THREADS = 128;
// padding (complex entries) between the rows of a fused pair's shared tile:
// phase 1 writes runs of Q entries from N Q apart, and the pad spreads them
// over both halves of the banks
constexpr int SEPR2_PAD = 8;

// Complex coefficients from shared memory.  The asm is volatile so that the
// loads stay inside the fiber loop: hoisting the loop-invariant coefficients
// into registers would spill.  Pairs need 16-byte alignment (an even entry
// offset for complex64).  The host branches let a CPU harness run the same
// step code on host arrays.
TB_HD void sepr_lds2(const cx<float> *p, cx<float> &a, cx<float> &b) {
#ifdef __CUDA_ARCH__
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(a.x), "=f"(a.y), "=f"(b.x), "=f"(b.y) : "r"(s));
#else
    a = p[0];
    b = p[1];
#endif
}
TB_HD void sepr_lds1(const cx<float> *p, cx<float> &a) {
#ifdef __CUDA_ARCH__
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(a.x), "=f"(a.y) : "r"(s));
#else
    a = p[0];
#endif
}
TB_HD void sepr_lds1(const cx<double> *p, cx<double> &a) {
#ifdef __CUDA_ARCH__
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(a.x), "=d"(a.y) : "r"(s));
#else
    a = p[0];
#endif
}
TB_HD void sepr_lds2(const cx<double> *p, cx<double> &a, cx<double> &b) {
    sepr_lds1(p, a);
    sepr_lds1(p + 1, b);
}

// One step of the chain: y = S x (forward, gather over each row's inputs) or
// y = S^H x (adjoint, scatter of each row's conjugated coefficients).  Rows of
// even width read their coefficients in pairs, odd widths one at a time.
template <class R, int LC, int RK, bool ADJ>
TB_HD void sepr_step(const cx<R> *__restrict__ cs, int st, const cx<R> (&x)[RK << (2 * LC)],
                     cx<R> (&y)[RK << (2 * LC)]) {
    constexpr int N = RK << (2 * LC);
    const int K = sepr_width(LC, RK, st);
    const cx<R> *c = cs + sepr_off(LC, RK, st);
    if (!ADJ) {
#pragma unroll
        for (int e = 0; e < N; ++e) {
            cx<R> acc = {R(0), R(0)};
            if (K % 2 == 0) {
#pragma unroll
                for (int j = 0; j < K; j += 2) {
                    cx<R> u, w;
                    sepr_lds2(c + e * K + j, u, w);
                    cmac(acc, u, x[sepr_col(LC, RK, st, e, j)]);
                    cmac(acc, w, x[sepr_col(LC, RK, st, e, j + 1)]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    cx<R> u;
                    sepr_lds1(c + e * K + j, u);
                    cmac(acc, u, x[sepr_col(LC, RK, st, e, j)]);
                }
            }
            y[e] = acc;
        }
    } else {
#pragma unroll
        for (int e = 0; e < N; ++e) y[e] = {R(0), R(0)};
#pragma unroll
        for (int e = 0; e < N; ++e) {
            if (K % 2 == 0) {
#pragma unroll
                for (int j = 0; j < K; j += 2) {
                    cx<R> u, w;
                    sepr_lds2(c + e * K + j, u, w);
                    cmac_conj(y[sepr_col(LC, RK, st, e, j)], u, x[e]);
                    cmac_conj(y[sepr_col(LC, RK, st, e, j + 1)], w, x[e]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    cx<R> u;
                    sepr_lds1(c + e * K + j, u);
                    cmac_conj(y[sepr_col(LC, RK, st, e, j)], u, x[e]);
                }
            }
        }
    }
}

template <class R, int LC, int RK, bool ADJ>
TB_HD void sepr_chain(const cx<R> *__restrict__ cs, cx<R> (&x)[RK << (2 * LC)]) {
    constexpr int N = RK << (2 * LC);
    cx<R> y[N];
    if (!ADJ) {
#pragma unroll
        for (int st = 0; st <= 2 * LC; st += 2) {
            sepr_step<R, LC, RK, false>(cs, st, x, y);
            if (st + 1 > 2 * LC) {
#pragma unroll
                for (int e = 0; e < N; ++e) x[e] = y[e];
                break;
            }
            sepr_step<R, LC, RK, false>(cs, st + 1, y, x);
        }
    } else {
#pragma unroll
        for (int st = 2 * LC; st >= 0; st -= 2) {
            sepr_step<R, LC, RK, true>(cs, st, x, y);
            if (st - 1 < 0) {
#pragma unroll
                for (int e = 0; e < N; ++e) x[e] = y[e];
                break;
            }
            sepr_step<R, LC, RK, true>(cs, st - 1, y, x);
        }
    }
}

// ---- complex64 with paired FP32 FMAs (fma.rn.f32x2, two lanes per
// instruction).  Coefficients are float4 (re, re, im, im) forward and
// (re, re, im, -im) adjoint, one 16-byte shared load each, feeding F fibers.
// Forward (gather): A = sum (re, re) * x, B = sum (im, im) * x over a row, then
// y = (A.x - B.y, A.y + B.x).  Adjoint (scatter):
// y[col] += (re, re) * x + (im, -im) * (x.y, x.x) = conj(c) x.
TB_HD float4 seprf_lds(const float4 *p) {
#ifdef __CUDA_ARCH__
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(s));
    return v;
#else
    return *p;
#endif
}
TB_HD float2 seprf_fma2(float2 a, float2 b, float2 c) {
#ifdef __CUDA_ARCH__
    return __ffma2_rn(a, b, c);
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}

template <int LC, int RK, bool ADJ, int F, int ST>
TB_HD void seprf_step(const float4 *__restrict__ cs, const float2 (&x)[F][RK << (2 * LC)],
                      float2 (&y)[F][RK << (2 * LC)]) {
    constexpr int N = RK << (2 * LC);
    constexpr int K = sepr_width(LC, RK, ST);
    const float4 *c = cs + sepr_off(LC, RK, ST);
    if constexpr (!ADJ) {
#pragma unroll
        for (int e = 0; e < N; ++e) {
            float2 A[F], B[F];
#pragma unroll
            for (int f = 0; f < F; ++f) A[f] = B[f] = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const float4 cc = seprf_lds(c + e * K + j);
                const float2 cr = make_float2(cc.x, cc.y), ci = make_float2(cc.z, cc.w);
                const int col = sepr_col(LC, RK, ST, e, j);
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    A[f] = seprf_fma2(cr, x[f][col], A[f]);
                    B[f] = seprf_fma2(ci, x[f][col], B[f]);
                }
            }
#pragma unroll
            for (int f = 0; f < F; ++f) y[f][e] = make_float2(A[f].x - B[f].y, A[f].y + B[f].x);
        }
    } else {
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
            for (int e = 0; e < N; ++e) y[f][e] = make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < N; ++e) {
            float2 xs[F];
#pragma unroll
            for (int f = 0; f < F; ++f) xs[f] = make_float2(x[f][e].y, x[f][e].x);
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const float4 cc = seprf_lds(c + e * K + j);
                const float2 cr = make_float2(cc.x, cc.y), ci = make_float2(cc.z, cc.w);
                const int col = sepr_col(LC, RK, ST, e, j);
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    y[f][col] = seprf_fma2(cr, x[f][e], y[f][col]);
                    y[f][col] = seprf_fma2(ci, xs[f], y[f][col]);
                }
            }
        }
    }
}

// steps I .. 2 Lc of the chain (forward order; the adjoint runs them
// reversed), ping-ponging between the two register arrays; the step index is
// a template argument so every register index is a compile-time constant
template <int LC, int RK, bool ADJ, int F, int I>
TB_HD void seprf_chain_from(const float4 *__restrict__ cs, float2 (&x)[F][RK << (2 * LC)],
                            float2 (&y)[F][RK << (2 * LC)]) {
    if constexpr (I <= 2 * LC) {
        seprf_step<LC, RK, ADJ, F, ADJ ? 2 * LC - I : I>(cs, x, y);
        seprf_chain_from<LC, RK, ADJ, F, I + 1>(cs, y, x);
    }
}

template <int LC, int RK, bool ADJ, int F>
TB_HD void seprf_chain(const float4 *__restrict__ cs, float2 (&x)[F][RK << (2 * LC)]) {
    constexpr int N = RK << (2 * LC);
    float2 y[F][N];
    seprf_chain_from<LC, RK, ADJ, F, 0>(cs, x, y);
    // 2 Lc + 1 steps: the result is in y
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
        for (int e = 0; e < N; ++e) x[f][e] = y[f][e];
}

// Per-mode register chain, complex64 paired-FMA form: each thread takes F
// fibers (f, f + T, ..., consecutive threads on consecutive fibers) and
// issues all F N loads before it stages the block's coefficients, so the
// loads are in flight during the staging.  One batch per thread (no
// grid-stride loop): the load / store offsets, kernel parameters, are then
// read where they are used instead of being held in registers.
template <int LC, int RK, bool ADJ, int F, int MINB>
__global__ void __launch_bounds__(SEPR_THREADS, MINB) k_sep_regf(const SepRegArgs<float> a) {
    constexpr int N = RK << (2 * LC);
    constexpr int NC = sepr_ncoef(LC, RK);
    __shared__ __align__(16) float4 cs[NC];
    const int *ldo = ADJ ? a.sto : a.ldo;
    const int *sto = ADJ ? a.ldo : a.sto;
    const int64_t total = a.outer * a.inner, inner = a.inner;
    const int64_t f0 = (int64_t)blockIdx.x * blockDim.x * F + threadIdx.x;
    const float2 *in = reinterpret_cast<const float2 *>(a.in);
    float2 *out = reinterpret_cast<float2 *>(a.out);
    float2 x[F][N];
    int64_t base[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const int64_t fi = f0 + (int64_t)f * blockDim.x;
        const int64_t o = fi / inner;
        base[f] = fi < total ? o * N * inner + (fi - o * inner) : -1;
    }
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
        for (int p = 0; p < N; ++p) x[f][p] = base[f] >= 0 ? in[base[f] + ldo[p]] : make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < NC; i += blockDim.x) cs[i] = a.cf4[i];
    __syncthreads();
    seprf_chain<LC, RK, ADJ, F>(cs, x);
#pragma unroll
    for (int f = 0; f < F; ++f)
        if (base[f] >= 0)
#pragma unroll
            for (int p = 0; p < N; ++p) out[base[f] + sto[p]] = x[f][p];
}

template <class R, int LC, int RK, bool ADJ, int MINB>
__global__ void __launch_bounds__(SEPR_THREADS, MINB) k_sep_reg(const SepRegArgs<R> a) {
    constexpr int N = RK << (2 * LC);
    constexpr int NC = sepr_ncoef(LC, RK);
    constexpr bool PF = N * sizeof(R) <= 64;
    __shared__ __align__(16) cx<R> cs[NC];
    for (int i = threadIdx.x; i < NC; i += blockDim.x) cs[i] = a.coef[i];
    __syncthreads();
    const int *ldo = ADJ ? a.sto : a.ldo;   // offsets the input is read from
    const int *sto = ADJ ? a.ldo : a.sto;   // offsets the output is written to
    const int64_t total = a.outer * a.inner;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t inner = a.inner;
    auto base = [&](int64_t f) {
        const int64_t o = f / inner;
        return o * N * inner + (f - o * inner);
    };
    auto load = [&](cx<R> (&x)[N], int64_t f) {
        const cx<R> *src = a.in + base(f);
#pragma unroll
        for (int p = 0; p < N; ++p) x[p] = src[ldo[p]];
    };
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    cx<R> xn[N];
    if (PF && f < total) load(xn, f);
    for (; f < total; f += stride) {
        cx<R> x[N];
        if (PF) {
#pragma unroll
            for (int p = 0; p < N; ++p) x[p] = xn[p];
            if (f + stride < total) load(xn, f + stride);
        } else {
            load(x, f);
        }
        sepr_chain<R, LC, RK, ADJ>(cs, x);
        cx<R> *dst = a.out + base(f);
#pragma unroll
        for (int p = 0; p < N; ++p) dst[sto[p]] = x[p];
    }
}

// Fused pair of modes (SepReg2Args): phase 1 applies mode kb to the fibers
// (o, i_ka = r, q) read from global memory and writes them to the shared tile
// in grid order; phase 2 applies mode ka to the fibers (o, i_kb = r, q) read
// from the tile and writes global memory.  Thread t = (r, qi) in both phases;
// the tile is (i_ka N + i_kb) Q + qi, so each warp's shared accesses are runs
// of Q consecutive entries.  Threads past the end of the inner range compute
// on zeros and store nothing.
template <class R, int LC, int RK, bool ADJ>
TB_HD void sepr2_phase1(const SepReg2Args<R> &a, const cx<R> *csb, cx<R> *tile, int64_t blk, int t) {
    constexpr int N = RK << (2 * LC);
    const int lq = a.lq, qi = t & ((1 << lq) - 1), r = t >> lq;
    const int64_t o = blk / a.nchunks, inner = a.inner;
    const int64_t q = ((blk - o * a.nchunks) << lq) + qi;
    const bool valid = q < inner;
    const int *ldb = ADJ ? a.st_b : a.ld_b, *stb = ADJ ? a.ld_b : a.st_b;
    cx<R> x[N];
    const cx<R> *src = a.in + ((o * N + r) * N) * inner + q;
#pragma unroll
    for (int p = 0; p < N; ++p) x[p] = valid ? src[(int64_t)ldb[p] * inner] : cx<R>{R(0), R(0)};
    sepr_chain<R, LC, RK, ADJ>(csb, x);
#pragma unroll
    for (int p = 0; p < N; ++p) tile[((r * N + stb[p]) << lq) + qi] = x[p];
}

template <class R, int LC, int RK, bool ADJ>
TB_HD void sepr2_phase2(const SepReg2Args<R> &a, const cx<R> *csa, const cx<R> *tile, int64_t blk, int t) {
    constexpr int N = RK << (2 * LC);
    const int lq = a.lq, qi = t & ((1 << lq) - 1), r = t >> lq;
    const int64_t o = blk / a.nchunks, inner = a.inner;
    const int64_t q = ((blk - o * a.nchunks) << lq) + qi;
    const int *lda = ADJ ? a.st_a : a.ld_a, *sta = ADJ ? a.ld_a : a.st_a;
    cx<R> x[N];
#pragma unroll
    for (int p = 0; p < N; ++p) x[p] = tile[((lda[p] * N + r) << lq) + qi];
    sepr_chain<R, LC, RK, ADJ>(csa, x);
    if (q < inner) {
        cx<R> *dst = a.out + (o * N * N + r) * inner + q;
#pragma unroll
        for (int p = 0; p < N; ++p) dst[(int64_t)sta[p] * N * inner] = x[p];
    }
}

// complex64 phases of the fused pair with the paired-FMA chain
template <int LC, int RK, bool ADJ>
TB_HD void seprf2_phase1(const SepReg2Args<float> &a, const float4 *csb, float2 *tile, int64_t blk, int t) {
    constexpr int N = RK << (2 * LC);
    const int lq = a.lq, qi = t & ((1 << lq) - 1), r = t >> lq;
    const int64_t o = blk / a.nchunks, inner = a.inner;
    const int64_t q = ((blk - o * a.nchunks) << lq) + qi;
    const bool valid = q < inner;
    const int *ldb = ADJ ? a.st_b : a.ld_b, *stb = ADJ ? a.ld_b : a.st_b;
    float2 x[1][N];
    const float2 *src = reinterpret_cast<const float2 *>(a.in) + ((o * N + r) * N) * inner + q;
#pragma unroll
    for (int p = 0; p < N; ++p) x[0][p] = valid ? src[(int64_t)ldb[p] * inner] : make_float2(0.f, 0.f);
    seprf_chain<LC, RK, ADJ, 1>(csb, x);
    const int pitch = (N << lq) + SEPR2_PAD;
#pragma unroll
    for (int p = 0; p < N; ++p) tile[r * pitch + (stb[p] << lq) + qi] = x[0][p];
}

template <int LC, int RK, bool ADJ>
TB_HD void seprf2_phase2(const SepReg2Args<float> &a, const float4 *csa, const float2 *tile, int64_t blk, int t) {
    constexpr int N = RK << (2 * LC);
    const int lq = a.lq, qi = t & ((1 << lq) - 1), r = t >> lq;
    const int64_t o = blk / a.nchunks, inner = a.inner;
    const int64_t q = ((blk - o * a.nchunks) << lq) + qi;
    const int *lda = ADJ ? a.st_a : a.ld_a, *sta = ADJ ? a.ld_a : a.st_a;
    const int pitch = (N << lq) + SEPR2_PAD;
    float2 x[1][N];
#pragma unroll
    for (int p = 0; p < N; ++p) x[0][p] = tile[lda[p] * pitch + (r << lq) + qi];
    seprf_chain<LC, RK, ADJ, 1>(csa, x);
    if (q < inner) {
        float2 *dst = reinterpret_cast<float2 *>(a.out) + (o * N * N + r) * inner + q;
#pragma unroll
        for (int p = 0; p < N; ++p) dst[(int64_t)sta[p] * N * inner] = x[0][p];
    }
}

template <int LC, int RK, bool ADJ>
__global__ void __launch_bounds__(SEPR_THREADS, 4) k_sep_reg2f(const SepReg2Args<float> a) {
    constexpr int NC = sepr_ncoef(LC, RK);
    extern __shared__ __align__(16) unsigned char smraw[];
    float4 *csb = reinterpret_cast<float4 *>(smraw);
    float4 *csa = csb + NC;
    float2 *tile = reinterpret_cast<float2 *>(csa + NC);
    for (int i = threadIdx.x; i < NC; i += blockDim.x) {
        csb[i] = a.cf4_b[i];
        csa[i] = a.cf4_a[i];
    }
    __syncthreads();
    seprf2_phase1<LC, RK, ADJ>(a, csb, tile, blockIdx.x, threadIdx.x);
    __syncthreads();
    seprf2_phase2<LC, RK, ADJ>(a, csa, tile, blockIdx.x, threadIdx.x);
}

template <class R, int LC, int RK, bool ADJ>
__global__ void __launch_bounds__(SEPR_THREADS, 4) k_sep_reg2(const SepReg2Args<R> a) {
    constexpr int NC = sepr_ncoef(LC, RK);
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R> *csb = reinterpret_cast<cx<R> *>(smraw);
    cx<R> *csa = csb + NC;
    cx<R> *tile = csa + NC;
    for (int i = threadIdx.x; i < NC; i += blockDim.x) {
        csb[i] = a.coef_b[i];
        csa[i] = a.coef_a[i];
    }
    __syncthreads();
    sepr2_phase1<R, LC, RK, ADJ>(a, csb, tile, blockIdx.x, threadIdx.x);
    __syncthreads();
    sepr2_phase2<R, LC, RK, ADJ>(a, csa, tile, blockIdx.x, threadIdx.x);
}

template <class R, int LC, int RK, int MINB>
static cudaError_t launch_sep_reg_t(bool adjoint, const SepRegArgs<R> &a, cudaStream_t st) {
    void (*fn)(const SepRegArgs<R>) =
        adjoint ? k_sep_reg<R, LC, RK, true, MINB> : k_sep_reg<R, LC, RK, false, MINB>;
    const int64_t total = a.outer * a.inner;
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + SEPR_THREADS - 1) / SEPR_THREADS;
    if (a.blocks > 0 && a.blocks < blocks) blocks = a.blocks;
    if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    fn<<<(unsigned)blocks, SEPR_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

template <class R, int LC, int RK>
static cudaError_t launch_sep_reg2_t(bool adjoint, const SepReg2Args<R> &a, cudaStream_t st) {
    void (*fn)(const SepReg2Args<R>) = adjoint ? k_sep_reg2<R, LC, RK, true> : k_sep_reg2<R, LC, RK, false>;
    constexpr int N = RK << (2 * LC);
    const int threads = N << a.lq;
    if (threads > SEPR_THREADS || threads < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(2 * sepr_ncoef(LC, RK) + N * N * (1 << a.lq)) * sizeof(cx<R>);
    cudaError_t e = set_smem_once((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = a.outer * a.nchunks;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    fn<<<(unsigned)blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <class R>
bool sep_reg_supported(int lc, int rk) {
    if (lc != 1) return false;
    if (sizeof(R) == 8) return rk == 1 || rk == 2;
    return rk == 1 || rk == 2 || rk == 4 || rk == 8;
}

template <class R>
cudaError_t launch_sep_reg(bool adjoint, int variant, const SepRegArgs<R> &a, cudaStream_t st) {
    if (!sep_reg_supported<R>(a.lc, a.rk)) return cudaErrorInvalidValue;
    switch (a.rk) {
        case 1: return launch_sep_reg_t<R, 1, 1, 3>(adjoint, a, st);
        case 2: return launch_sep_reg_t<R, 1, 2, 3>(adjoint, a, st);
        default: break;
    }
    (void)variant;
    return cudaErrorInvalidValue;
}

template <class R>
cudaError_t launch_sep_reg2(bool adjoint, const SepReg2Args<R> &a, cudaStream_t st) {
    if (!sep_reg_supported<R>(a.lc, a.rk)) return cudaErrorInvalidValue;
    switch (a.rk) {
        case 1: return launch_sep_reg2_t<R, 1, 1>(adjoint, a, st);
        case 2: return launch_sep_reg2_t<R, 1, 2>(adjoint, a, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int LC, int RK, int F, int MINB>
static cudaError_t launch_sep_regf_t(bool adjoint, const SepRegArgs<float> &a, cudaStream_t st) {
    void (*fn)(const SepRegArgs<float>) =
        adjoint ? k_sep_regf<LC, RK, true, F, MINB> : k_sep_regf<LC, RK, false, F, MINB>;
    const int64_t total = a.outer * a.inner;
    if (total <= 0) return cudaSuccess;
    const int64_t blocks = (total + (int64_t)SEPR_THREADS * F - 1) / ((int64_t)SEPR_THREADS * F);
    if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    fn<<<(unsigned)blocks, SEPR_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

template <int LC, int RK>
static cudaError_t launch_sep_reg2f_t(bool adjoint, const SepReg2Args<float> &a, cudaStream_t st) {
    void (*fn)(const SepReg2Args<float>) = adjoint ? k_sep_reg2f<LC, RK, true> : k_sep_reg2f<LC, RK, false>;
    constexpr int N = RK << (2 * LC);
    const int threads = N << a.lq;
    if (threads > SEPR_THREADS || threads < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * sepr_ncoef(LC, RK) * sizeof(float4) +
                        (size_t)N * ((N << a.lq) + SEPR2_PAD) * sizeof(float2);
    cudaError_t e = set_smem_once((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = a.outer * a.nchunks;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    fn<<<(unsigned)blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

// complex64: the paired-FMA form with two fibers per thread up to N = 16
// (variant 0, 3 resident blocks per SM) or one (variant 2, 4 blocks), and
// the scalar form with prefetch (variant 1), for rk up to 8
template <>
cudaError_t launch_sep_reg<float>(bool adjoint, int variant, const SepRegArgs<float> &a, cudaStream_t st) {
    if (!sep_reg_supported<float>(a.lc, a.rk)) return cudaErrorInvalidValue;
    if (variant == 0) {
        switch (a.rk) {
            case 1: return launch_sep_regf_t<1, 1, 2, 3>(adjoint, a, st);
            case 2: return launch_sep_regf_t<1, 2, 2, 3>(adjoint, a, st);
            case 4: return launch_sep_regf_t<1, 4, 2, 3>(adjoint, a, st);
            case 8: return launch_sep_regf_t<1, 8, 1, 3>(adjoint, a, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (variant == 2) {
        switch (a.rk) {
            case 1: return launch_sep_regf_t<1, 1, 1, 4>(adjoint, a, st);
            case 2: return launch_sep_regf_t<1, 2, 1, 4>(adjoint, a, st);
            case 4: return launch_sep_regf_t<1, 4, 1, 4>(adjoint, a, st);
            case 8: return launch_sep_regf_t<1, 8, 1, 3>(adjoint, a, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (a.rk) {
        case 1: return launch_sep_reg_t<float, 1, 1, 3>(adjoint, a, st);
        case 2: return launch_sep_reg_t<float, 1, 2, 3>(adjoint, a, st);
        case 4: return launch_sep_reg_t<float, 1, 4, 3>(adjoint, a, st);
        case 8: return launch_sep_reg_t<float, 1, 8, 2>(adjoint, a, st);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_sep_reg2<float>(bool adjoint, const SepReg2Args<float> &a, cudaStream_t st) {
    if (!sep_reg_supported<float>(a.lc, a.rk)) return cudaErrorInvalidValue;
    switch (a.rk) {
        case 1: return launch_sep_reg2f_t<1, 1>(adjoint, a, st);
        case 2: return launch_sep_reg2f_t<1, 2>(adjoint, a, st);
        case 4: return launch_sep_reg2f_t<1, 4>(adjoint, a, st);
        case 8: return launch_sep_reg2f_t<1, 8>(adjoint, a, st);
        default: return cudaErrorInvalidValue;
    }
}

template bool sep_reg_supported<float>(int, int);
template bool sep_reg_supported<double>(int, int);
template cudaError_t launch_sep_reg<double>(bool, int, const SepRegArgs<double> &, cudaStream_t);
template cudaError_t launch_sep_reg2<double>(bool, const SepReg2Args<double> &, cudaStream_t);

}  // namespace tb

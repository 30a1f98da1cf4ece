// Apply of a separable tensor butterfly (kernel = product of per-mode
// factors, e.g. the Fourier kernel of Sec. 3.2.1 / 4.3).
//
// With separable factors (see the separable reading of Eqs. tensorID_BF_V /
// transfer W in the construction) every transfer, interpolation and core block
// acts on one mode, so the tensor butterfly of Eq. (butterfly_tensor) is the
// tensor product over modes of 1-D butterfly chains
//     B_k = U_k P_k,1 .. P_k,Lc  K_k  W_k,Lc .. W_k,1 V_k ,
// and u = f x_1 B_1 x_2 ... x_d B_d.  A thread block stages a tile that holds
// complete fibers along a few consecutive modes (and a contiguous run of the
// trailing modes and right-hand sides), and applies the step matrices of those
// modes one after another in shared memory.  Each step is a small sparse
// matrix (CSR) on the 1-D index of its mode.
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

template <class R, int LC, int RK, bool ADJ>
__global__ void __launch_bounds__(SEPR_THREADS, (RK << (2 * LC)) * sizeof(R) <= 64 ? 3 : 2)
    k_sep_reg(const SepRegArgs<R> a) {
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

template <class R, int LC, int RK>
static cudaError_t launch_sep_reg_t(bool adjoint, const SepRegArgs<R> &a, cudaStream_t st) {
    void (*fn)(const SepRegArgs<R>) = adjoint ? k_sep_reg<R, LC, RK, true> : k_sep_reg<R, LC, RK, false>;
    const int64_t total = a.outer * a.inner;
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + SEPR_THREADS - 1) / SEPR_THREADS;
    if (a.blocks > 0 && a.blocks < blocks) blocks = a.blocks;
    if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    fn<<<(unsigned)blocks, SEPR_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

template <class R>
bool sep_reg_supported(int lc, int rk) {
    if (lc != 1) return false;
    if (sizeof(R) == 8) return rk == 1 || rk == 2;
    return rk == 1 || rk == 2 || rk == 4 || rk == 8;
}

template <class R>
cudaError_t launch_sep_reg(bool adjoint, const SepRegArgs<R> &a, cudaStream_t st) {
    if (!sep_reg_supported<R>(a.lc, a.rk)) return cudaErrorInvalidValue;
    switch (a.rk) {
        case 1: return launch_sep_reg_t<R, 1, 1>(adjoint, a, st);
        case 2: return launch_sep_reg_t<R, 1, 2>(adjoint, a, st);
        default: break;
    }
    return cudaErrorInvalidValue;
}

// the longer fibers are instantiated for complex64 only
template <>
cudaError_t launch_sep_reg<float>(bool adjoint, const SepRegArgs<float> &a, cudaStream_t st) {
    if (!sep_reg_supported<float>(a.lc, a.rk)) return cudaErrorInvalidValue;
    switch (a.rk) {
        case 1: return launch_sep_reg_t<float, 1, 1>(adjoint, a, st);
        case 2: return launch_sep_reg_t<float, 1, 2>(adjoint, a, st);
        case 4: return launch_sep_reg_t<float, 1, 4>(adjoint, a, st);
        case 8: return launch_sep_reg_t<float, 1, 8>(adjoint, a, st);
        default: return cudaErrorInvalidValue;
    }
}

template bool sep_reg_supported<float>(int, int);
template bool sep_reg_supported<double>(int, int);
template cudaError_t launch_sep_reg<double>(bool, const SepRegArgs<double> &, cudaStream_t);

}  // namespace tb

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

}  // namespace tb

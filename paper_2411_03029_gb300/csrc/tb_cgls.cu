// Vector kernels of the device-resident least-squares solver (tb_cgls).
//
// CGLS (conjugate gradients on the normal equations K^H K x = K^H b) solves
// min_x ||K x - b||_2 for each right-hand-side column independently; the
// inversion of generalized Radon data is the use the paper gives these
// operators (Sec. 4.2).  The forward and adjoint butterflies are the library's
// own applies; the kernels here do the vector updates and the per-column
// squared norms.  Every scalar of the iteration (gamma = ||s||^2, alpha, beta,
// the residual history) lives in device memory and is read by the kernels that
// need it, so an iteration has no host round trip and can be captured once as
// a CUDA graph and replayed.
//
// Layout: N x nv complex entries with the RHS index innermost (the apply's
// layout), so entry e belongs to column e % nv.  A block has J = blockDim / nv
// row lanes per column; a thread keeps one column for the whole launch (the
// grid's row stride is a multiple of nv), so alpha / beta are read once.
// Norms: each thread sums |a_e|^2 in FP64, the block reduces its threads of a
// column in a fixed order into partial[block][column], and a single-block
// kernel sums the partials over blocks in order: deterministic, no atomics.
#include "tb_kernels.cuh"

namespace tb {
namespace {

constexpr int CG_THREADS = 256;
constexpr int CG_BLOCKS = 304;   // two per SM on GB300; the partial sums have this many rows

struct Lanes {
    int v, j, J;   // column, row lane, lanes per column
};

TB_DEV Lanes lanes(int nv) {
    const int J = blockDim.x / nv;
    return {(int)(threadIdx.x % nv), (int)(threadIdx.x / nv), J};
}

// Write the block's per-column sums of `acc` (threads with t < J nv) to partial[blockIdx.x][v].
TB_DEV void block_column_sums(double acc, int nv, int J, double *partial) {
    __shared__ double red[1024];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < J; ++j) s += red[j * nv + v];
        partial[(int64_t)blockIdx.x * nv + v] = s;
    }
}

template <class R>
__global__ void __launch_bounds__(1024) k_cgls_sqnorm(const cx<R> *__restrict__ a, int64_t rows, int nv,
                                                       double *partial) {
    const Lanes L = lanes(nv);
    double acc = 0.0;
    if (L.j < L.J) {
        const int64_t stride = (int64_t)gridDim.x * L.J;
        for (int64_t r = (int64_t)blockIdx.x * L.J + L.j; r < rows; r += stride) {
            const cx<R> z = a[r * nv + L.v];
            acc += (double)z.x * z.x + (double)z.y * z.y;
        }
    }
    block_column_sums(acc, nv, L.J, partial);
}

// x += alpha_v p, r -= alpha_v q; partial sums of |r|^2 of the updated r.
template <class R>
__global__ void __launch_bounds__(1024) k_cgls_xr(cx<R> *__restrict__ x, cx<R> *__restrict__ r,
                                                   const cx<R> *__restrict__ p, const cx<R> *__restrict__ q,
                                                   const CglsScalars *__restrict__ sc, int64_t rows, int nv,
                                                   double *partial) {
    const Lanes L = lanes(nv);
    double acc = 0.0;
    if (L.j < L.J) {
        const R al = (R)sc[L.v].alpha;
        const int64_t stride = (int64_t)gridDim.x * L.J;
        for (int64_t i = (int64_t)blockIdx.x * L.J + L.j; i < rows; i += stride) {
            const int64_t e = i * nv + L.v;
            const cx<R> pe = p[e], qe = q[e];
            cx<R> xe = x[e], re = r[e];
            xe.x = fma(al, pe.x, xe.x);
            xe.y = fma(al, pe.y, xe.y);
            re.x = fma(-al, qe.x, re.x);
            re.y = fma(-al, qe.y, re.y);
            x[e] = xe;
            r[e] = re;
            acc += (double)re.x * re.x + (double)re.y * re.y;
        }
    }
    block_column_sums(acc, nv, L.J, partial);
}

// r = b - q; partial sums of |r|^2.
template <class R>
__global__ void __launch_bounds__(1024) k_cgls_sub(cx<R> *__restrict__ r, const cx<R> *__restrict__ b,
                                                    const cx<R> *__restrict__ q, int64_t rows, int nv,
                                                    double *partial) {
    const Lanes L = lanes(nv);
    double acc = 0.0;
    if (L.j < L.J) {
        const int64_t stride = (int64_t)gridDim.x * L.J;
        for (int64_t i = (int64_t)blockIdx.x * L.J + L.j; i < rows; i += stride) {
            const int64_t e = i * nv + L.v;
            const cx<R> be = b[e], qe = q[e];
            const cx<R> re = {be.x - qe.x, be.y - qe.y};
            r[e] = re;
            acc += (double)re.x * re.x + (double)re.y * re.y;
        }
    }
    block_column_sums(acc, nv, L.J, partial);
}

// p = s + beta_v p
template <class R>
__global__ void __launch_bounds__(1024) k_cgls_p(cx<R> *__restrict__ p, const cx<R> *__restrict__ s,
                                                  const CglsScalars *__restrict__ sc, int64_t rows, int nv) {
    const Lanes L = lanes(nv);
    if (L.j >= L.J) return;
    const R be = (R)sc[L.v].beta;
    const int64_t stride = (int64_t)gridDim.x * L.J;
    for (int64_t i = (int64_t)blockIdx.x * L.J + L.j; i < rows; i += stride) {
        const int64_t e = i * nv + L.v;
        const cx<R> se = s[e];
        cx<R> pe = p[e];
        pe.x = fma(be, pe.x, se.x);
        pe.y = fma(be, pe.y, se.y);
        p[e] = pe;
    }
}

// Sum the partials of each column over the blocks (in block order) and update
// the iteration's scalars:
//   CG_GAMMA0   gamma = ||s||^2 (start)
//   CG_ALPHA    delta = ||q||^2, alpha = gamma / delta (0 when delta = 0)
//   CG_BETA     beta = ||s_new||^2 / gamma (0 when gamma = 0), gamma = ||s_new||^2
//   CG_RESID    hist[count][v] = ||r||, then count += 1 (kept below `cap` rows)
__global__ void k_cgls_finalize(const double *__restrict__ partial, int nblocks, int nv, int mode,
                                CglsScalars *sc, double *hist, int *count, int cap) {
    __shared__ int s_row;
    if (threadIdx.x == 0) s_row = mode == CG_RESID ? *count : 0;
    __syncthreads();
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * nv + v];
        CglsScalars c = sc[v];
        if (mode == CG_GAMMA0) {
            c.gamma = s;
        } else if (mode == CG_ALPHA) {
            c.delta = s;
            c.alpha = s > 0.0 ? c.gamma / s : 0.0;
        } else if (mode == CG_BETA) {
            c.beta = c.gamma > 0.0 ? s / c.gamma : 0.0;
            c.gamma = s;
        } else if (s_row < cap) {
            hist[(int64_t)s_row * nv + v] = sqrt(s);
        }
        sc[v] = c;
    }
    __syncthreads();
    if (mode == CG_RESID && threadIdx.x == 0 && s_row < cap) *count = s_row + 1;
}

dim3 cg_block(int nv) {
    const int J = nv <= CG_THREADS ? CG_THREADS / nv : 1;
    return dim3((unsigned)(J * nv));
}

}  // namespace

int cgls_blocks() { return CG_BLOCKS; }
int cgls_max_nv() { return 1024; }

template <class R>
cudaError_t launch_cgls_sqnorm(const cx<R> *a, int64_t rows, int nv, double *partial, cudaStream_t st) {
    k_cgls_sqnorm<R><<<CG_BLOCKS, cg_block(nv), 0, st>>>(a, rows, nv, partial);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_cgls_xr(cx<R> *x, cx<R> *r, const cx<R> *p, const cx<R> *q, const CglsScalars *sc, int64_t rows,
                           int nv, double *partial, cudaStream_t st) {
    k_cgls_xr<R><<<CG_BLOCKS, cg_block(nv), 0, st>>>(x, r, p, q, sc, rows, nv, partial);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_cgls_sub(cx<R> *r, const cx<R> *b, const cx<R> *q, int64_t rows, int nv, double *partial,
                            cudaStream_t st) {
    k_cgls_sub<R><<<CG_BLOCKS, cg_block(nv), 0, st>>>(r, b, q, rows, nv, partial);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_cgls_p(cx<R> *p, const cx<R> *s, const CglsScalars *sc, int64_t rows, int nv, cudaStream_t st) {
    k_cgls_p<R><<<CG_BLOCKS, cg_block(nv), 0, st>>>(p, s, sc, rows, nv);
    return cudaGetLastError();
}

cudaError_t launch_cgls_finalize(const double *partial, int nv, int mode, CglsScalars *sc, double *hist, int *count,
                                 int cap, cudaStream_t st) {
    k_cgls_finalize<<<1, 256, 0, st>>>(partial, CG_BLOCKS, nv, mode, sc, hist, count, cap);
    return cudaGetLastError();
}

#define TB_CGLS_INST(R)                                                                                       \
    template cudaError_t launch_cgls_sqnorm<R>(const cx<R> *, int64_t, int, double *, cudaStream_t);          \
    template cudaError_t launch_cgls_xr<R>(cx<R> *, cx<R> *, const cx<R> *, const cx<R> *, const CglsScalars *, \
                                           int64_t, int, double *, cudaStream_t);                             \
    template cudaError_t launch_cgls_sub<R>(cx<R> *, const cx<R> *, const cx<R> *, int64_t, int, double *,    \
                                            cudaStream_t);                                                    \
    template cudaError_t launch_cgls_p<R>(cx<R> *, const cx<R> *, const CglsScalars *, int64_t, int, cudaStream_t);
TB_CGLS_INST(float)
TB_CGLS_INST(double)

}  // namespace tb

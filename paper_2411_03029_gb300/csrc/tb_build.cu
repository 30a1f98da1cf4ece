// Construction kernels of the tensor butterfly (Alg. 1, Sec. 3.2).
//
//  * k_interp_decomp: one thread block per interpolative decomposition.  It
//    forms the proxy matrix of Eq. (tensorID_BF_V) / (transfer W) (or the
//    target-side mirror, Eqs. tensorID_BF_U / transfer P) row chunk by row
//    chunk with FP64 kernel phases, folds each chunk into a running
//    triangular factor by Householder reflections (so the proxy matrix is never
//    stored), runs a column-pivoted QR on that factor, truncates at the
//    smallest rank r with ||R22||_F <= eps ||A||_F (Sec. 2.1), and solves
//    R11 T = R12 for the interpolation coefficients.
//  * k_core_eval: the mid-level skeleton cores K(t-bar, s-bar) of Alg. 1 step 3.
//  * k_kron_eval: per-mode factors of the core when the kernel is a product
//    over modes (the core is then their Kronecker product, Eq. tuckerID).
#include <cstdio>

#include "tb_kernels.cuh"

namespace tb {

constexpr int ID_THREADS = 128;
constexpr int ID_CHUNK = 32;   // proxy rows folded per step
constexpr int ID_NCMAX = 64;   // candidate columns per ID

TB_DEV uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// A bijection of [0, 2^bits) (odd multipliers, additions and xor-shifts are
// each invertible modulo 2^bits): the row permutation of one mode in the
// Latin-hypercube proxy design.  Multipliers and offsets are drawn from the
// salt, so the permutations of different modes are unrelated; a fixed
// multiplier with a salted offset would make them shifted copies of one
// permutation, a correlated design that loses accuracy in the IDs.
TB_DEV uint32_t perm_bits(uint32_t q, uint32_t salt, int bits) {
    const uint32_t mask = (bits >= 32) ? 0xffffffffu : ((1u << bits) - 1u);
    const int s1 = bits / 2 + 1, s2 = (bits + 1) / 2;
    uint32_t x = q;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const uint32_t km = mix32(salt + 0x9E3779B9u * (uint32_t)(2 * r));
        const uint32_t ka = mix32(salt + 0x9E3779B9u * (uint32_t)(2 * r + 1));
        x = (x * (km | 1u) + ka) & mask;
        x ^= x >> ((r & 1) ? s2 : s1);
    }
    return x;
}

TB_DEV c128 cdiv(c128 a, c128 b) {
    double inv = 1.0 / norm2(b);
    return {(a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv};
}

// Block-wide reduction of one double into lane 0 of warp 0 (result broadcast
// through `slot`).
TB_DEV double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

__global__ void __launch_bounds__(ID_THREADS)
k_interp_decomp(const IdArgs a) {
    extern __shared__ __align__(16) unsigned char id_smem[];
    const int64_t id = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
    if (id >= a.nids) return;
    const int tid = threadIdx.x, bd = blockDim.x;
    const int d = a.d, l = a.l, Lc = a.Lc;

    __shared__ int cand[ID_NCMAX], piv[ID_NCMAX], ipiv[ID_NCMAX];
    __shared__ int rsize[2 * MAXD], rstart[2 * MAXD], rmode[2 * MAXD], rside[2 * MAXD];
    __shared__ uint32_t rsalt[2 * MAXD];
    __shared__ int64_t rstride[2 * MAXD];
    __shared__ double red[33];
    __shared__ double cn[ID_NCMAX];
    __shared__ c128 hh[2];      // v0, beta
    __shared__ double hcoef;
    __shared__ int flags[4];    // skip, stop, rank, pivot
    __shared__ int sh_k, sh_nc, sh_r1, sh_nrows, sh_nrm, sh_exh;
    __shared__ int64_t sh_j;
    __shared__ int sh_F[MAXD], sh_M[MAXD];

    // ---------------------------------------------------------- decode the ID
    if (tid == 0) {
        const int nseg = 1 << (Lc - l);
        int k, sg;
        int64_t j;
        int64_t r = id;
        sg = (int)(r % nseg);
        r /= nseg;
        if (!a.separable) {
            k = (int)(r % d);
            r /= d;
            const int64_t nM = ipow2(d * l);
            const int64_t M = r % nM, F = r / nM;
            for (int m = 0; m < d; ++m) {
                sh_M[m] = (int)((M >> (l * (d - 1 - m))) & ((1 << l) - 1));
                sh_F[m] = (int)((F >> (Lc * (d - 1 - m))) & ((1 << Lc) - 1));
            }
            j = (F * nM + M) * nseg + sg;
        } else {
            const int Mk = (int)(r % (1 << l));
            r >>= l;
            const int Fk = (int)(r % (1 << Lc));
            k = (int)(r >> Lc);
            for (int m = 0; m < d; ++m) { sh_M[m] = 0; sh_F[m] = 0; }
            sh_M[k] = Mk;
            sh_F[k] = Fk;
            j = ((int64_t)Fk * (1 << l) + Mk) * nseg + sg;
        }
        sh_k = k;
        sh_j = j;
        // candidates of mode k
        int nc = 0, r1 = 0;
        if (l == 0) {
            const int64_t base = (int64_t)sh_F[k] * (a.n[k] >> Lc) + (int64_t)sg * a.cb[k];
            nc = a.cb[k];
            for (int c = 0; c < nc; ++c) cand[c] = a.perm[k][base + c];
        } else {
            int64_t jp;
            if (!a.separable) {
                const int64_t nMp = ipow2(d * (l - 1));
                int64_t pM = 0;
                for (int m = 0; m < d; ++m) pM = (pM << (l - 1)) | (sh_M[m] >> 1);
                int64_t F = 0;
                for (int m = 0; m < d; ++m) F = (F << Lc) | sh_F[m];
                jp = (F * nMp + pM) * (2 * nseg) + 2 * sg;
            } else {
                jp = ((int64_t)sh_F[k] * (1 << (l - 1)) + (sh_M[k] >> 1)) * (2 * nseg) + 2 * sg;
            }
            const int *ps = a.pskel[k];
            const int pc = a.pcap[k];
            r1 = a.prank[k][jp];
            const int r2 = a.prank[k][jp + 1];
            for (int c = 0; c < r1; ++c) cand[nc++] = ps[jp * pc + c];
            for (int c = 0; c < r2; ++c) cand[nc++] = ps[(jp + 1) * pc + c];
        }
        sh_nc = nc;
        sh_r1 = r1;
        // proxy row design: row modes and node extents
        int nrm = 0;
        if (!a.separable) {
            for (int m = 0; m < d; ++m) {   // other side, nodes at level l
                rmode[nrm] = m; rside[nrm] = 1;
                rsize[nrm] = (int)(a.n[m] >> l);
                rstart[nrm] = sh_M[m] * rsize[nrm];
                ++nrm;
            }
            for (int m = 0; m < d; ++m) {   // own side, mid-level nodes except mode k
                if (m == k) continue;
                rmode[nrm] = m; rside[nrm] = 0;
                rsize[nrm] = (int)(a.n[m] >> Lc);
                rstart[nrm] = sh_F[m] * rsize[nrm];
                ++nrm;
            }
        } else {
            rmode[0] = k; rside[0] = 1;
            rsize[0] = (int)(a.n[k] >> l);
            rstart[0] = sh_M[k] * rsize[0];
            nrm = 1;
        }
        double tot = 1.0;
        for (int q = 0; q < nrm; ++q) tot *= (double)rsize[q];
        int exh = tot <= (double)a.rows_cap;
        int nrows = exh ? (int)tot : a.rows_cap;
        int64_t st = 1;
        for (int q = nrm - 1; q >= 0; --q) { rstride[q] = st; st *= rsize[q]; }
        for (int q = 0; q < nrm; ++q)
            rsalt[q] = mix32(a.seed ^ mix32((uint32_t)(id * 2654435761ull) + 977u * q + 131071u * a.side + 7919u * l));
        sh_nrm = nrm;
        sh_nrows = nrows;
        sh_exh = exh;
    }
    __syncthreads();
    const int k = sh_k, nc = sh_nc, nrm = sh_nrm, nrows = sh_nrows, exh = sh_exh;
    const int64_t j = sh_j;

    c128 *Rm = reinterpret_cast<c128 *>(id_smem);   // nc x nc, leading dim nc
    c128 *B = Rm + nc * nc;                          // ID_CHUNK x nc

    for (int e = tid; e < nc * nc; e += bd) Rm[e] = {0.0, 0.0};
    __syncthreads();

    // ---------------------------------------------- stream the proxy matrix
    for (int q0 = 0; q0 < nrows; q0 += ID_CHUNK) {
        for (int e = tid; e < ID_CHUNK * nc; e += bd) {
            const int i = e / nc, c = e - i * nc;
            const int q = q0 + i;
            c128 val = {0.0, 0.0};
            if (q < nrows) {
                double xo[MAXD], xw[MAXD];   // other-side / own-side point
                for (int m = 0; m < d; ++m) { xo[m] = a.oth[m][0]; xw[m] = a.own[m][0]; }
                for (int rm = 0; rm < nrm; ++rm) {
                    int pos;
                    if (exh) pos = (int)((q / rstride[rm]) % rsize[rm]);
                    else {
                        const uint32_t h = perm_bits((uint32_t)q, rsalt[rm], a.rows_bits);
                        pos = (int)(((2ull * h + 1ull) * (uint64_t)rsize[rm]) >> (a.rows_bits + 1));
                    }
                    const int m = rmode[rm];
                    const int g = a.perm[m][rstart[rm] + pos];
                    if (rside[rm]) xo[m] = a.oth[m][g];
                    else xw[m] = a.own[m][g];
                }
                xw[k] = a.own[k][cand[c]];
                val = (a.side == 0) ? eval_kernel(a.ks, d, xo, xw) : eval_kernel(a.ks, d, xw, xo);
            }
            B[i * nc + c] = val;
        }
        __syncthreads();
        // fold [Rm; B] -> Rm by Householder reflections, column by column
        for (int jc = 0; jc < nc; ++jc) {
            if (tid < 32) {
                double s = 0.0;
                for (int i = tid; i < ID_CHUNK; i += 32) s += norm2(B[i * nc + jc]);
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (tid == 0) {
                    if (s == 0.0) flags[0] = 1;
                    else {
                        const c128 al = Rm[jc * nc + jc];
                        const double na = sqrt(norm2(al));
                        const double nr = sqrt(na * na + s);
                        c128 beta = (na == 0.0) ? c128{-nr, 0.0} : c128{-nr * al.x / na, -nr * al.y / na};
                        c128 v0 = al - beta;
                        hh[0] = v0;
                        hh[1] = beta;
                        hcoef = 2.0 / (norm2(v0) + s);
                        flags[0] = 0;
                    }
                }
            }
            __syncthreads();
            if (!flags[0]) {
                const c128 v0 = hh[0];
                const double cf = hcoef;
                for (int m = jc + 1 + tid; m < nc; m += bd) {
                    c128 w = {0.0, 0.0};
                    cmac_conj(w, v0, Rm[jc * nc + m]);
                    for (int i = 0; i < ID_CHUNK; ++i) cmac_conj(w, B[i * nc + jc], B[i * nc + m]);
                    w = cf * w;
                    Rm[jc * nc + m] = Rm[jc * nc + m] - w * v0;
                    for (int i = 0; i < ID_CHUNK; ++i) B[i * nc + m] = B[i * nc + m] - w * B[i * nc + jc];
                }
            }
            __syncthreads();
            if (!flags[0]) {
                if (tid == 0) Rm[jc * nc + jc] = hh[1];
                for (int i = tid; i < ID_CHUNK; i += bd) B[i * nc + jc] = {0.0, 0.0};
            }
            __syncthreads();
        }
    }

    // ------------------------------------ column-pivoted QR of the factor
    double part = 0.0;
    for (int e = tid; e < nc * nc; e += bd) part += norm2(Rm[e]);
    const double total2 = block_sum(part, red);
    const double thr = a.tol * a.tol * total2;
    int rcap = nc < a.cap[k] ? nc : a.cap[k];
    if (rcap > a.rank_max) rcap = a.rank_max;
    for (int c = tid; c < nc; c += bd) piv[c] = c;
    if (tid == 0) { flags[1] = 0; flags[2] = nc; }
    __syncthreads();
    for (int jc = 0; jc < nc; ++jc) {
        for (int m = jc + tid; m < nc; m += bd) {
            double s = 0.0;
            for (int i = jc; i < nc; ++i) s += norm2(Rm[i * nc + m]);
            cn[m] = s;
        }
        __syncthreads();
        if (tid == 0) {
            double trail = 0.0;
            int p = jc;
            double best = -1.0;
            for (int m = jc; m < nc; ++m) {
                trail += cn[m];
                if (cn[m] > best) { best = cn[m]; p = m; }
            }
            if (total2 == 0.0 && jc == 1) { flags[1] = 1; flags[2] = 1; }
            else if (jc > 0 && trail <= thr) { flags[1] = 1; flags[2] = jc; }
            else if (jc == rcap) {
                flags[1] = 1;
                flags[2] = jc;
                atomicMax(a.err, 2);   // rank cap exceeded
            }
            flags[3] = p;
            if (!flags[1] && p != jc) { int t = piv[jc]; piv[jc] = piv[p]; piv[p] = t; }
        }
        __syncthreads();
        if (flags[1]) break;
        const int p = flags[3];
        if (p != jc)
            for (int i = tid; i < nc; i += bd) {
                c128 t = Rm[i * nc + jc];
                Rm[i * nc + jc] = Rm[i * nc + p];
                Rm[i * nc + p] = t;
            }
        __syncthreads();
        if (tid < 32) {
            double s = 0.0;
            for (int i = jc + 1 + tid; i < nc; i += 32) s += norm2(Rm[i * nc + jc]);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (tid == 0) {
                if (s == 0.0) flags[0] = 1;
                else {
                    const c128 al = Rm[jc * nc + jc];
                    const double na = sqrt(norm2(al));
                    const double nr = sqrt(na * na + s);
                    c128 beta = (na == 0.0) ? c128{-nr, 0.0} : c128{-nr * al.x / na, -nr * al.y / na};
                    hh[0] = al - beta;
                    hh[1] = beta;
                    hcoef = 2.0 / (norm2(hh[0]) + s);
                    flags[0] = 0;
                }
            }
        }
        __syncthreads();
        if (!flags[0]) {
            const c128 v0 = hh[0];
            const double cf = hcoef;
            for (int m = jc + 1 + tid; m < nc; m += bd) {
                c128 w = {0.0, 0.0};
                cmac_conj(w, v0, Rm[jc * nc + m]);
                for (int i = jc + 1; i < nc; ++i) cmac_conj(w, Rm[i * nc + jc], Rm[i * nc + m]);
                w = cf * w;
                Rm[jc * nc + m] = Rm[jc * nc + m] - w * v0;
                for (int i = jc + 1; i < nc; ++i) Rm[i * nc + m] = Rm[i * nc + m] - w * Rm[i * nc + jc];
            }
        }
        __syncthreads();
        if (!flags[0]) {
            if (tid == 0) Rm[jc * nc + jc] = hh[1];
            for (int i = jc + 1 + tid; i < nc; i += bd) Rm[i * nc + jc] = {0.0, 0.0};
        }
        __syncthreads();
    }
    const int r = flags[2];
    const bool degenerate = (total2 == 0.0);

    // ----------------------- interpolation coefficients T = R11^{-1} R12
    for (int m = r + tid; m < nc; m += bd) {
        for (int i = r - 1; i >= 0; --i) {
            c128 t = Rm[i * nc + m];
            for (int q = i + 1; q < r; ++q) t = t - Rm[i * nc + q] * Rm[q * nc + m];
            Rm[i * nc + m] = degenerate ? c128{0.0, 0.0} : cdiv(t, Rm[i * nc + i]);
        }
    }
    for (int c = tid; c < nc; c += bd) ipiv[piv[c]] = c;
    __syncthreads();

    // ----------------------------------------------------------- outputs
    const int cap = a.cap[k], cin = a.cin[k];
    if (tid == 0) a.rank[k][j] = r;
    for (int s = tid; s < cap; s += bd) a.skel[k][j * cap + s] = (s < r) ? cand[piv[s]] : -1;
    c128 *V = a.fac[k] + j * (int64_t)cap * cin;
    const int r1 = sh_r1, pR = (l > 0) ? a.pR[k] : 0;
    for (int e = tid; e < cap * cin; e += bd) {
        const int row = e / cin, col = e - row * cin;
        int c = -1;
        if (l == 0) c = (col < nc) ? col : -1;
        else if (col < pR) c = (col < r1) ? col : -1;
        else {
            const int q = col - pR;
            c = (r1 + q < nc) ? r1 + q : -1;
        }
        c128 v = {0.0, 0.0};
        if (c >= 0 && row < r) {
            const int jp = ipiv[c];
            if (jp < r) v = (jp == row) ? c128{1.0, 0.0} : c128{0.0, 0.0};
            else v = Rm[row * nc + jp];
        }
        V[e] = v;
    }
}

// ------------------------------------------------------------ mid-level cores
__global__ void k_core_eval(const CoreArgs a) {
    const int64_t p = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
    if (p >= a.P) return;
    const int d = a.d;
    const int *dims = a.dims + p * 2 * d;
    int rt[MAXD], rs[MAXD];
    int64_t Mt = 1, Ms = 1;
    for (int k = 0; k < d; ++k) {
        rt[k] = dims[k];
        rs[k] = dims[d + k];
        Mt *= rt[k];
        Ms *= rs[k];
    }
    const int64_t t = p / a.nF, s = p % a.nF;
    const int64_t jt = t * a.nF + s, js = s * a.nF + t;   // level-Lc block indices
    const int64_t off = a.off[p];
    for (int64_t e = threadIdx.x; e < Mt * Ms; e += blockDim.x) {
        int64_t ia = e / Ms, ib = e - ia * Ms;
        double x[MAXD], y[MAXD];
        for (int k = d - 1; k >= 0; --k) {
            const int ak = (int)(ia % rt[k]);
            ia /= rt[k];
            const int bk = (int)(ib % rs[k]);
            ib /= rs[k];
            x[k] = a.xs[k][a.tskel[k][jt * a.tcap[k] + ak]];
            y[k] = a.ys[k][a.sskel[k][js * a.scap[k] + bk]];
        }
        const c128 v = eval_kernel(a.ks, d, x, y);
        if (a.out64) a.out64[off + e] = v;
        if (a.out32) a.out32[off + e] = {(float)v.x, (float)v.y};
    }
}

// Per-mode core factors K_k(t-bar_k, s-bar_k), zero-padded to Rt x Rs, for a
// kernel that is a product over modes (evaluated as the 1-D kernel).
__global__ void k_kron_eval(const KronArgs a) {
    const int nb = 1 << a.Lc;
    const int64_t blk = blockIdx.x;   // (t_k, s_k)
    if (blk >= (int64_t)nb * nb) return;
    const int tk = (int)(blk / nb), sk = (int)(blk % nb);
    const int64_t jt = (int64_t)tk * nb + sk, js = (int64_t)sk * nb + tk;
    const int rt = a.trank[jt], rs = a.srank[js];
    for (int e = threadIdx.x; e < a.Rt * a.Rs; e += blockDim.x) {
        const int ia = e / a.Rs, ib = e - ia * a.Rs;
        c128 v = {0.0, 0.0};
        if (ia < rt && ib < rs) {
            const double x = a.xk[a.tskel[jt * a.tcap + ia]];
            const double y = a.yk[a.sskel[js * a.scap + ib]];
            v = eval_kernel(a.ks, 1, &x, &y);
        }
        if (a.out64) a.out64[blk * a.Rt * a.Rs + e] = v;
        if (a.out32) a.out32[blk * a.Rt * a.Rs + e] = {(float)v.x, (float)v.y};
    }
}

__global__ void k_to_c64(const c128 *in, c64 *out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = {(float)in[i].x, (float)in[i].y};
}

// ------------------------------------------------------------- launchers
cudaError_t launch_interp_decomp(const IdArgs &a, cudaStream_t st) {
    const size_t smem = (size_t)(a.ncmax * a.ncmax + ID_CHUNK * a.ncmax) * sizeof(c128);
    cudaError_t e = set_smem_once((const void *)k_interp_decomp, smem);
    if (e != cudaSuccess) return e;
    const int64_t gx = a.nids < 65535 ? a.nids : 65535;
    dim3 grid((unsigned)gx, (unsigned)((a.nids + gx - 1) / gx));
    k_interp_decomp<<<grid, ID_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_core_eval(const CoreArgs &a, cudaStream_t st) {
    const int64_t gx = a.P < 65535 ? a.P : 65535;
    dim3 grid((unsigned)gx, (unsigned)((a.P + gx - 1) / gx));
    k_core_eval<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_kron_eval(const KronArgs &a, cudaStream_t st) {
    const int nb = 1 << a.Lc;
    k_kron_eval<<<nb * nb, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_to_c64(const c128 *in, c64 *out, int64_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_to_c64<<<(unsigned)blocks, 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

int id_max_columns() { return ID_NCMAX; }

}  // namespace tb

// Mid-level core contraction G_{t,s} = K(t-bar, s-bar) x_{d+1..2d} F_{t,s}
// (Alg. 2, step 2) on the tcgen05 tensor cores in two-term split BF16 with
// FP32 accumulation in tensor memory.
//
// Real form.  With the core stored as interleaved (re, im) pairs, a core row
// is a real row of length 2 M_s, and for each RHS v the two real rows
//     A_re[v] = ( Re x_k, -Im x_k )_k      A_im[v] = ( Im x_k, Re x_k )_k
// give Re G[n][v] = <C_row n, A_re[v]> and Im G[n][v] = <C_row n, A_im[v]>.
// So G^T = A (M x 2Ms) * C^T with M = 2 nv, a tensor-core product
// D[m][n] = sum_k A[m][k] B[n][k] whose B operand is the core itself, K-major.
//
// Split BF16.  C = Ch + Cl and x = xh + xl in BF16 (hi = rn(v), lo = rn(v - hi)).
// A holds the rows of xh (rows 0..31) and xl (rows 32..63); two products with
// B = Ch and B = Cl land in two TMEM accumulators, and the four partial
// products xh Ch + xl Ch + xh Cl + xl Cl are summed in FP32 in the epilogue.
//
// Core storage (built once by k_core_tile): per pair, row tiles of up to 128
// core rows (rows padded to 16) and K-chunks of 32 complex columns (columns
// padded to 32).  Each (tile, chunk) block holds rows x 128 B of Ch followed by
// rows x 128 B of Cl, in the 128-byte-swizzled layout the MMA reads from
// shared memory, so one bulk copy moves a block.
//
// Pipeline.  One 256-thread block per SM walks its work items (pair, row
// tile); K-chunks stream through 4 shared-memory stages with bulk copies
// issued two chunks ahead.  Every wait on an mbarrier is bounded: on expiry
// the block records TB_ETIMEOUT in the error word, drains its outstanding
// copies (again bounded), frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "tb_kernels.cuh"

namespace tb {

namespace tc {

constexpr int NT = 128;             // core rows per work item (MMA N)
constexpr int KC = 32;              // complex core columns per K-chunk (64 BF16 = 128 B)
constexpr int STAGES = 4;
constexpr int AHEAD = 2;            // chunks prefetched ahead of the MMA
constexpr int THREADS = 256;
constexpr int A_BYTES = 128 * 128;  // 128 rows x 128 B
constexpr int B_BYTES = 2 * NT * 128;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_BYTES = 32 * NT * 4;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_BYTES + 1024;
constexpr uint32_t TMEM_COLS = 2 * NT;   // D_hi at [0, NT), D_lo at [NT, 2 NT)
constexpr long long SPIN_LIMIT = 1ll << 26;

TB_DEV uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

TB_DEV void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
TB_DEV void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
TB_DEV bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the barrier phase did not complete within the limit.
TB_DEV bool mbar_wait(uint64_t *bar, uint32_t phase) {
    for (long long i = 0; i < SPIN_LIMIT; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}
TB_DEV void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
TB_DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
TB_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
TB_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (stride byte offset), descriptor version 1.
TB_DEV uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused with a 128 B swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // version
    d |= (uint64_t)2 << 61;               // swizzle 128 B
    return d;
}
// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, M = 128.
TB_HD uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
TB_DEV void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
TB_DEV void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
TB_DEV void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of (row, byte-in-row) in a 128 B-swizzled K-major tile
TB_HD uint32_t swz(uint32_t row, uint32_t byte) {
    return row * 128u + ((((byte >> 4) ^ (row & 7u)) << 4) | (byte & 15u));
}

TB_DEV uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

}  // namespace tc

// Compact multi-index -> position in a padded tile.
TB_DEV int compact_to_padded(int idx, int d, const int *r, const int *R) {
    int pos = 0, stride = 1;
    for (int k = d - 1; k >= 0; --k) {
        pos += (idx % r[k]) * stride;
        idx /= r[k];
        stride *= R[k];
    }
    return pos;
}

// ---------------------------------------------------------------- build: tiling
__global__ void k_core_tile(const CoreTileArgs a) {
    using namespace tc;
    const int64_t it = blockIdx.x;
    if (it >= a.nitems) return;
    const CoreItem item = a.items[it];
    const int p = item.pair, d = a.d;
    int Mt = 1, Ms = 1;
    for (int k = 0; k < d; ++k) {
        Mt *= a.dims[(int64_t)p * 2 * d + k];
        Ms *= a.dims[(int64_t)p * 2 * d + d + k];
    }
    // rows of this operator: forward C (Mt x Ms), adjoint C^H (Ms x Mt)
    const int nrows = a.adjoint ? Ms : Mt, ncols = a.adjoint ? Mt : Ms;
    const int64_t off = a.core_off[p];
    unsigned char *base = a.out + item.boff;
    const int rows = item.rows;
    for (int64_t e = threadIdx.x; e < (int64_t)item.nkc * rows * KC; e += blockDim.x) {
        const int kk = (int)(e % KC);
        const int64_t t = e / KC;
        const int r = (int)(t % rows);
        const int kc = (int)(t / rows);
        const int n = item.tile * NT + r, k = kc * KC + kk;
        double re = 0.0, im = 0.0;
        if (n < nrows && k < ncols) {
            const int64_t ci = a.adjoint ? off + (int64_t)k * Ms + n : off + (int64_t)n * Ms + k;
            if (a.c128) { re = a.c128[ci].x; im = a.c128[ci].y; }
            else { re = a.c64[ci].x; im = a.c64[ci].y; }
            if (a.adjoint) im = -im;
        }
        const __nv_bfloat16 hr = __double2bfloat16(re), hi = __double2bfloat16(im);
        const __nv_bfloat16 lr = __double2bfloat16(re - (double)__bfloat162float(hr));
        const __nv_bfloat16 li = __double2bfloat16(im - (double)__bfloat162float(hi));
        unsigned char *blk = base + (int64_t)kc * rows * 256;
        const uint32_t o = swz((uint32_t)r, (uint32_t)(4 * kk));
        __nv_bfloat162 h2, l2;
        h2.x = hr; h2.y = hi;
        l2.x = lr; l2.y = li;
        *reinterpret_cast<__nv_bfloat162 *>(blk + o) = h2;
        *reinterpret_cast<__nv_bfloat162 *>(blk + (int64_t)rows * 128 + o) = l2;
    }
}

cudaError_t launch_core_tile(const CoreTileArgs &a, cudaStream_t st) {
    if (a.nitems == 0) return cudaSuccess;
    k_core_tile<<<(unsigned)a.nitems, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ the apply
__global__ void __launch_bounds__(tc::THREADS, 1) k_core_tc(const CoreTcArgs a) {
    using namespace tc;
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES], mma_bar[STAGES];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int d = a.d;
    float *epi = reinterpret_cast<float *>(sm + STAGES * STAGE_BYTES);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&mma_bar[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_sh = 0;
    }
    // A rows 64..127 stay zero; rows 0..63 are rewritten for every chunk
    for (int s = 0; s < STAGES; ++s)
        for (int i = tid; i < A_BYTES / 16; i += THREADS)
            reinterpret_cast<uint4 *>(sm + s * STAGE_BYTES)[i] = make_uint4(0, 0, 0, 0);
    fence_proxy_async();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    // chunk streams: "copy" runs AHEAD chunks in front of "compute"
    struct Cursor {
        int64_t item;
        int kc;
    };
    auto next = [&](Cursor c) {
        if (++c.kc >= a.items[c.item].nkc) {
            c.kc = 0;
            c.item += gridDim.x;
        }
        return c;
    };
    Cursor cp{(int64_t)blockIdx.x, 0}, cm{(int64_t)blockIdx.x, 0};
    int64_t g_copy = 0, g = 0;   // chunks issued / computed by this block
    bool ok = true;
    auto issue = [&](Cursor c, int64_t gi) {
        // stage reuse: MMAs of chunk gi - STAGES must have drained it
        const int s = (int)(gi % STAGES);
        if (gi >= STAGES && !mbar_wait(&mma_bar[s], (uint32_t)(((gi - STAGES) / STAGES) & 1))) return false;
        if (tid == 0) {
            const CoreItem it = a.items[c.item];
            const uint32_t bytes = (uint32_t)it.rows * 256u;
            mbar_expect_tx(&full_bar[s], bytes);
            bulk_g2s(sm + s * STAGE_BYTES + A_BYTES, a.tiles + it.boff + (int64_t)c.kc * bytes, bytes, &full_bar[s]);
        }
        return true;
    };
    for (int i = 0; i < AHEAD && cp.item < a.nitems && ok; ++i) {
        ok = issue(cp, g_copy);
        ++g_copy;
        cp = next(cp);
    }

    // the two (k, v) input values this thread converts for a chunk; loaded one
    // chunk ahead so their L2 latency overlaps the previous chunk's work
    constexpr int PER = KC * 16 / THREADS;
    auto load_x = [&](Cursor c, cx<float> *x) {
#pragma unroll
        for (int i = 0; i < PER; ++i) x[i] = cx<float>{0.f, 0.f};
        if (c.item >= a.nitems) return;
        const int pp = a.items[c.item].pair;
        int r[MAXD], M = 1;
        for (int k = 0; k < d; ++k) {
            r[k] = a.dims[(int64_t)pp * 2 * d + (a.adjoint ? k : d + k)];
            M *= r[k];
        }
        const cx<float> *xin = a.in + (int64_t)pp * a.in_tsize * a.nv;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = tid + i * THREADS;
            const int v = e & 15, k = c.kc * KC + (e >> 4);
            if (v < a.nvc && k < M)
                x[i] = xin[(int64_t)compact_to_padded(k, d, r, a.in_R) * a.nv + a.v0 + v];
        }
    };
    cx<float> xcur[PER], xnxt[PER];
    load_x(cm, xcur);

    while (ok && cm.item < a.nitems) {
        const CoreItem it = a.items[cm.item];
        const int p = it.pair;
        int rout[MAXD];
        int Mout = 1;
        for (int k = 0; k < d; ++k) {
            rout[k] = a.dims[(int64_t)p * 2 * d + (a.adjoint ? d + k : k)];
            Mout *= rout[k];
        }
        const int s = (int)(g % STAGES);
        // prefetch
        if (cp.item < a.nitems) {
            ok = issue(cp, g_copy);
            ++g_copy;
            cp = next(cp);
        }
        if (__syncthreads_or(!ok)) { ok = false; break; }
        load_x(next(cm), xnxt);
        // build A for this chunk: rows v / 16+v (x_hi re/im), 32+v / 48+v (x_lo)
        unsigned char *A = sm + s * STAGE_BYTES;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = tid + i * THREADS;
            const int v = e & 15, kk = e >> 4;
            const float xr = xcur[i].x, xi = xcur[i].y;
            const float hr = __bfloat162float(__float2bfloat16_rn(xr));
            const float hi = __bfloat162float(__float2bfloat16_rn(xi));
            const float lr = xr - hr, li = xi - hi;
            const uint32_t b = 4u * kk;
            *reinterpret_cast<uint32_t *>(A + swz(v, b)) = pack_bf16(hr, -hi);
            *reinterpret_cast<uint32_t *>(A + swz(16 + v, b)) = pack_bf16(hi, hr);
            *reinterpret_cast<uint32_t *>(A + swz(32 + v, b)) = pack_bf16(lr, -li);
            *reinterpret_cast<uint32_t *>(A + swz(48 + v, b)) = pack_bf16(li, lr);
        }
        fence_proxy_async();
        __syncthreads();
        ok = mbar_wait(&full_bar[s], (uint32_t)((g / STAGES) & 1));
        if (__syncthreads_or(!ok)) { ok = false; break; }
        if (tid == 0) {
            tc_fence_after();
            const uint32_t ab = smem_u32(A), bh = ab + A_BYTES, bl = bh + (uint32_t)it.rows * 128u;
            const uint32_t idesc = idesc_bf16(it.rows);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint32_t acc = (cm.kc > 0 || ks > 0) ? 1u : 0u;
                const uint32_t koff = 32u * ks;
                mma_bf16(tmem, sdesc(ab + koff), sdesc(bh + koff), idesc, acc);
                mma_bf16(tmem + NT, sdesc(ab + koff), sdesc(bl + koff), idesc, acc);
            }
            mma_commit(&mma_bar[s]);
        }
        const bool last = (cm.kc + 1 == it.nkc);
        const int64_t gdone = g;
        ++g;
        cm = next(cm);
#pragma unroll
        for (int i = 0; i < PER; ++i) xcur[i] = xnxt[i];
        if (!last) continue;

        // ------------------------------------------------------- epilogue
        ok = mbar_wait(&mma_bar[s], (uint32_t)((gdone / STAGES) & 1));
        if (__syncthreads_or(!ok)) { ok = false; break; }
        tc_fence_after();
        const int wq = warp & 3;   // TMEM lane quarter this warp may read
        const int ngrp = it.rows / 16;
        // pass 1: lanes 32..63 (x_lo rows) -> epi; pass 2: lanes 0..31 add
        for (int pass = 0; pass < 2; ++pass) {
            if (wq == 1 - pass) {
                for (int gq = (warp >> 2); gq < ngrp; gq += 2) {
                    float dh[16], dl[16];
                    const uint32_t taddr = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(16 * gq);
                    tmem_ld16(taddr, dh);
                    tmem_ld16(taddr + NT, dl);
                    float *row = epi + lane * NT + 16 * gq;
#pragma unroll
                    for (int c = 0; c < 16; ++c) row[c] = (pass == 0) ? dh[c] + dl[c] : row[c] + dh[c] + dl[c];
                }
            }
            tc_fence_before();
            __syncthreads();
        }
        // write G rows of this tile: G[n][v] = epi[v][n] + i epi[16+v][n]
        cx<float> *out = a.out + (int64_t)p * a.out_tsize * a.nv;
        const int nbase = it.tile * NT;
        for (int e = tid; e < it.rows * 16; e += THREADS) {
            const int v = e & 15, nl = e >> 4;
            const int n = nbase + nl;
            if (v < a.nvc && n < Mout) {
                const int pos = compact_to_padded(n, d, rout, a.out_R);
                out[(int64_t)pos * a.nv + a.v0 + v] = cx<float>{epi[v * NT + nl], epi[(16 + v) * NT + nl]};
            }
        }
        if (it.tile == 0) {   // zero the padded entries no compact index reaches
            for (int64_t e = tid; e < (int64_t)a.out_tsize * a.nvc; e += THREADS) {
                int b = (int)(e / a.nvc), pad = 0;
                const int v = (int)(e - (int64_t)b * a.nvc);
                const int64_t idx = (int64_t)b * a.nv + a.v0 + v;
                for (int k = d - 1; k >= 0; --k) {
                    if (b % a.out_R[k] >= rout[k]) pad = 1;
                    b /= a.out_R[k];
                }
                if (pad) out[idx] = cx<float>{0.f, 0.f};
            }
        }
        __syncthreads();
    }

    if (!ok) {
        if (tid == 0) atomicExch(a.err, (int)TB_ETIMEOUT);
        // drain the copies this block issued and that may still be landing
        for (int64_t gi = (g_copy > STAGES ? g_copy - STAGES : 0); gi < g_copy; ++gi)
            mbar_wait(&full_bar[gi % STAGES], (uint32_t)((gi / STAGES) & 1));
        if (g > 0) mbar_wait(&mma_bar[(g - 1) % STAGES], (uint32_t)(((g - 1) / STAGES) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

int core_tc_rows_per_item() { return tc::NT; }
int core_tc_cols_per_chunk() { return tc::KC; }

cudaError_t launch_core_tc(const CoreTcArgs &a, cudaStream_t st) {
    if (a.nitems == 0) return cudaSuccess;
    cudaError_t e = set_smem_once((const void *)k_core_tc, tc::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = a.nitems < sms ? a.nitems : sms;
    k_core_tc<<<(unsigned)grid, tc::THREADS, tc::SMEM_BYTES, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tb

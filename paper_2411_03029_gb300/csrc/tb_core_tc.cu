// Mid-level core contraction G_{t,s} = K(t-bar, s-bar) x_{d+1..2d} F_{t,s}
// (Alg. 2, step 2) on the tcgen05 tensor cores in two-term split BF16 with
// FP32 accumulation in tensor memory.
//
// Real form.  With the core stored as interleaved (re, im) pairs, a core row
// is a real row of length 2 M_s, and for each RHS v the two real rows
//     B_re[v] = ( Re x_k, -Im x_k )_k      B_im[v] = ( Im x_k, Re x_k )_k
// give Re G[n][v] = <C_row n, B_re[v]> and Im G[n][v] = <C_row n, B_im[v]>.
// So G = C B^T, a tensor-core product D[m][n] = sum_k A[m][k] B[n][k] whose A
// operand is a tile of up to 128 core rows (K-major, MMA M = 128) and whose B
// operand holds 64 rows: B_re, B_im of x_hi (rows 0..31) and of x_lo (32..63)
// for 16 right-hand sides (MMA N = 64).
//
// Split BF16.  C = Ch + Cl and x = xh + xl in BF16 (hi = rn(v), lo = rn(v - hi)).
// The products Ch B^T and Cl B^T land in two 64-column TMEM accumulators and
// the epilogue sums the four partial products xh Ch + xl Ch + xh Cl + xl Cl in
// FP32.
//
// Core storage (built once by k_core_tile): per pair, row tiles of up to 128
// core rows (rows padded to 16) and K-chunks of 32 complex columns (columns
// padded to 32).  Each (tile, chunk) block holds rows x 128 B of Ch followed by
// rows x 128 B of Cl, in the 128-byte-swizzled K-major layout the MMA reads
// from shared memory, so one bulk copy moves a block.
//
// Pipeline.  One 384-thread block per SM walks its work items (pair, row tile)
// with warp-specialised roles that meet at mbarriers:
//   warp 0       streams the core K-chunks into STAGES shared-memory stages
//                (cp.async.bulk, completion counted in bytes);
//   warps 8..11  load the matching 32 x 16 input values (CONV_AHEAD chunks ahead,
//                through a build-time table of padded input positions), split
//                them into BF16 pairs and write the B rows of the stage;
//   warp 1       issues the MMAs of a chunk once both halves of its stage have
//                landed and releases the stage with tcgen05.commit;
//   warps 4..7   drain a finished item's accumulator from tensor memory and
//                write its rows of G.  Accumulators are double-buffered, so
//                the next item's MMAs overlap the drain;
//   warps 2..3   zero the padded entries of each pair's output tile.
// Every mbarrier wait is bounded.  A role whose wait expires records
// TB_ETIMEOUT and raises a block-wide abort flag that ends the other roles'
// waits; the block then waits, again bounded, for its copies and MMAs in
// flight, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "tb_kernels.cuh"
#include "tb_tc.cuh"

namespace tb {

namespace tc {

constexpr int NT = 128;                    // core rows per work item (MMA M)
constexpr int KC = 32;                     // complex core columns per K-chunk (64 BF16 = 128 B)
constexpr int NB = 64;                     // B rows (MMA N)
constexpr int STAGES = 5;
constexpr int THREADS = 384;
constexpr int CORE_BYTES = 2 * NT * 128;   // Ch tile then Cl tile
constexpr int X_BYTES = NB * 128;
constexpr int STAGE_BYTES = CORE_BYTES + X_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr uint32_t ACC_COLS = 128;         // D_h at [0, 64), D_l at [64, 128)
constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
constexpr int EPI_WARP0 = 4;               // warps 4..7: one per TMEM lane quarter
constexpr int CONV_WARP0 = 8;              // warps 8..11
constexpr int PAD_WARP0 = 2;               // warps 2..3
constexpr int NEPI = 128, NCONV = 128, NPAD = 64;
#ifndef TB_CONV_AHEAD
#define TB_CONV_AHEAD 3
#endif
constexpr int CONV_AHEAD = TB_CONV_AHEAD;   // input chunks the converters keep in flight
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
    __shared__ __align__(8) uint64_t full_bar[STAGES], xfull_bar[STAGES], empty_bar[STAGES];
    __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int d = a.d;
    const volatile int *abort = &abort_sh;
    auto give_up = [&]() {
        if (atomicExch(&abort_sh, 1) == 0) atomicExch(a.err, (int)TB_ETIMEOUT);
    };

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&xfull_bar[s], NCONV);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf_bar[b], 1);
            mbar_init(&acce_bar[b], NEPI);
        }
        mbar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_sh = 0;
    }
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
    int64_t issued = 0;   // producer: chunks whose copy was issued

    if (warp == 0) {
        // ------------------------------------------------ core chunk producer
        if (lane == 0) {
            bool ok = true;
            for (int64_t item = blockIdx.x; ok && item < a.nitems; item += gridDim.x) {
                const CoreItem it = a.items[item];
                const uint32_t bytes = (uint32_t)it.rows * 256u;
                const unsigned char *src = a.tiles + it.boff;
                for (int kc = 0; kc < it.nkc; ++kc) {
                    const int s = (int)(issued % STAGES);
                    if (issued >= STAGES &&
                        !mbar_wait(&empty_bar[s], (uint32_t)((issued / STAGES - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full_bar[s], bytes);
                    bulk_g2s(sm + s * STAGE_BYTES, src + (int64_t)kc * bytes, bytes, &full_bar[s]);
                    ++issued;
                }
            }
            if (!ok) give_up();
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int64_t gi = 0, ni = 0;
            bool ok = true;
            const uint32_t idesc = idesc_bf16(NB);
            for (int64_t item = blockIdx.x; ok && item < a.nitems; item += gridDim.x, ++ni) {
                const CoreItem it = a.items[item];
                const int b = (int)(ni & 1);
                if (ni >= 2 && !mbar_wait(&acce_bar[b], (uint32_t)(((ni >> 1) - 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dh = tmem + (uint32_t)b * ACC_COLS, dl = dh + 64u;
                for (int kc = 0; kc < it.nkc; ++kc, ++gi) {
                    const int s = (int)(gi % STAGES);
                    const uint32_t ph = (uint32_t)((gi / STAGES) & 1);
                    if (!mbar_wait(&full_bar[s], ph, abort) || !mbar_wait(&xfull_bar[s], ph, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ch = smem_u32(sm + s * STAGE_BYTES);
                    const uint32_t cl = ch + (uint32_t)it.rows * 128u, xb = ch + CORE_BYTES;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                        const uint32_t koff = 32u * ks;
                        mma_bf16(dh, sdesc(ch + koff), sdesc(xb + koff), idesc, acc);
                        mma_bf16(dl, sdesc(cl + koff), sdesc(xb + koff), idesc, acc);
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) break;
                mma_commit(&accf_bar[b]);
            }
            if (!ok) give_up();
            // completes once every MMA issued above has finished
            mma_commit(&done_bar);
            mbar_wait(&done_bar, 0);
        }
    } else if (warp >= CONV_WARP0) {
        // ------------------------------------------- input split into BF16 rows
        const int t = tid - CONV_WARP0 * 32;
        const int kq = t >> 4, v = t & 15;   // columns 4 kq .. 4 kq + 3 of a chunk, RHS v
        const bool vlive = v < a.nvc;
        // Look-ahead cursor over (item, chunk).  The padded positions of the
        // cursor's four columns (a build-time table, -1 past the pair's last
        // column) are loaded one call before the values that use them, and the
        // item after the cursor's is fetched one item early, so no value load
        // waits on a table or item load issued in the same call.
        int64_t litem = blockIdx.x;
        int lkc = 0;
        CoreItem lit, lnext;
        if (litem < a.nitems) lit = a.items[litem];
        if (litem + gridDim.x < a.nitems) lnext = a.items[litem + gridDim.x];
        int4 lps = make_int4(-1, -1, -1, -1);
        auto load_pos = [&]() {
            if (litem < a.nitems) lps = *reinterpret_cast<const int4 *>(a.xpos + lit.xpos + lkc * KC + 4 * kq);
        };
        load_pos();
        auto load_next = [&](cx<float> *x) {
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = cx<float>{0.f, 0.f};
            if (litem >= a.nitems) return;
            const cx<float> *base = a.in + (int64_t)lit.pair * a.in_tsize * a.nv + a.v0 + v;
            if (vlive) {
                if (lps.x >= 0) x[0] = base[(int64_t)lps.x * a.nv];
                if (lps.y >= 0) x[1] = base[(int64_t)lps.y * a.nv];
                if (lps.z >= 0) x[2] = base[(int64_t)lps.z * a.nv];
                if (lps.w >= 0) x[3] = base[(int64_t)lps.w * a.nv];
            }
            if (++lkc >= lit.nkc) {
                lkc = 0;
                litem += gridDim.x;
                if (litem < a.nitems) {
                    lit = lnext;
                    if (litem + gridDim.x < a.nitems) lnext = a.items[litem + gridDim.x];
                }
            }
            load_pos();   // for the next call
        };
        // CONV_AHEAD chunks of values in flight, in fixed registers (the loop
        // below is unrolled, so no value that may still be loading is copied)
        cx<float> xb[CONV_AHEAD][4];
#pragma unroll
        for (int u = 0; u < CONV_AHEAD; ++u) load_next(xb[u]);
        int64_t item = blockIdx.x, gi = 0;
        int kc = 0, nkc = item < a.nitems ? a.items[item].nkc : 0;
        bool ok = true;
        auto step = [&](cx<float> *x) -> bool {
            if (item >= a.nitems) return false;
            const int s = (int)(gi % STAGES);
            if (gi >= STAGES && !mbar_wait(&empty_bar[s], (uint32_t)((gi / STAGES - 1) & 1), abort)) {
                ok = false;
                return false;
            }
            unsigned char *X = sm + s * STAGE_BYTES + CORE_BYTES;
            // rows v, 16 + v, 32 + v, 48 + v; bytes 16 kq .. 16 kq + 15 (columns 4 kq .. 4 kq + 3)
            uint32_t w[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float xr = x[i].x, xi = x[i].y;
                const float hr = __bfloat162float(__float2bfloat16_rn(xr));
                const float hi = __bfloat162float(__float2bfloat16_rn(xi));
                const float lr_ = xr - hr, li = xi - hi;
                w[0][i] = pack_bf16(hr, -hi);
                w[1][i] = pack_bf16(hi, hr);
                w[2][i] = pack_bf16(lr_, -li);
                w[3][i] = pack_bf16(li, lr_);
            }
#pragma unroll
            for (int f = 0; f < 4; ++f)
                *reinterpret_cast<uint4 *>(X + swz(16 * f + v, 16u * kq)) = make_uint4(w[f][0], w[f][1], w[f][2], w[f][3]);
            fence_proxy_async();   // generic-proxy writes -> visible to the MMA
            mbar_arrive(&xfull_bar[s]);
            ++gi;
            load_next(x);   // the chunk CONV_AHEAD ahead
            if (++kc >= nkc) {
                kc = 0;
                item += gridDim.x;
                if (item < a.nitems) nkc = a.items[item].nkc;
            }
            return true;
        };
        for (bool more = true; more;) {
#pragma unroll
            for (int u = 0; u < CONV_AHEAD; ++u)
                if (more) more = step(xb[u]);
        }
        if (!ok) give_up();
    } else if (warp >= EPI_WARP0) {
        // --------------------------------------------------------- epilogue
        const int q = warp & 3;   // the TMEM lane quarter this warp may read
        int64_t ni = 0;
        for (int64_t item = blockIdx.x; item < a.nitems; item += gridDim.x, ++ni) {
            const CoreItem it = a.items[item];
            const int b = (int)(ni & 1);
            // warp-uniform outcome: the TMEM loads below are warp-collective
            if (!__all_sync(0xffffffffu, mbar_wait(&accf_bar[b], (uint32_t)((ni >> 1) & 1), abort))) {
                give_up();
                break;
            }
            tc_fence_after();
            float re[16], im[16], c[32];
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)b * ACC_COLS;
            tmem_ld32(taddr, c);   // Ch against the x_hi rows
#pragma unroll
            for (int v = 0; v < 16; ++v) { re[v] = c[v]; im[v] = c[16 + v]; }
#pragma unroll
            for (int part = 1; part < 4; ++part) {   // Ch x_lo, Cl x_hi, Cl x_lo
                tmem_ld32(taddr + 32u * part, c);
#pragma unroll
                for (int v = 0; v < 16; ++v) { re[v] += c[v]; im[v] += c[16 + v]; }
            }
            tc_fence_before();
            mbar_arrive(&acce_bar[b]);

            const int p = it.pair;
            int Mout = 1;
            for (int k = 0; k < d; ++k) Mout *= it.rout[k];
            cx<float> *out = a.out + (int64_t)p * a.out_tsize * a.nv;
            const int nl = 32 * q + lane, n = it.tile * NT + nl;
            if (nl < it.rows && n < Mout) {
                const int pos = compact_to_padded(n, d, it.rout, a.out_R);
                cx<float> *o = out + (int64_t)pos * a.nv + a.v0;
                if ((a.nv & 1) == 0 && (a.v0 & 1) == 0) {   // 16-byte aligned pairs
#pragma unroll
                    for (int v = 0; v < 16; v += 2) {
                        if (v + 1 < a.nvc)
                            *reinterpret_cast<float4 *>(o + v) = make_float4(re[v], im[v], re[v + 1], im[v + 1]);
                        else if (v < a.nvc)
                            o[v] = cx<float>{re[v], im[v]};
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < 16; ++v)
                        if (v < a.nvc) o[v] = cx<float>{re[v], im[v]};
                }
            }
        }
    } else if (warp >= PAD_WARP0) {
        // ------------------------------ zero the padded entries of the output
        // A pair's output tile has padded R_k positions in every mode; the
        // compact entries (index < r_k in every mode) are written by the
        // epilogue, the rest must read as zero.  This role walks the block's
        // items with tile 0 (one per pair) and clears the others, one 16-RHS
        // run per entry, independently of the MMA pipeline.  Skipped when the
        // output buffer keeps zeros there from one apply to the next.
        const int pt = tid - PAD_WARP0 * 32;
        int inner = 1;
        for (int k = 1; k < d; ++k) inner *= a.out_R[k];
        const bool vec = (a.nv & 1) == 0;
        for (int64_t item = blockIdx.x; a.zero_pad && item < a.nitems && !*abort; item += gridDim.x) {
            const CoreItem it = a.items[item];
            if (it.tile != 0) continue;
            const int *rout = it.rout;
            cx<float> *out = a.out + (int64_t)it.pair * a.out_tsize * a.nv + a.v0;
            for (int j = pt; j < inner; j += NPAD) {
                int rem = j;
                bool pin = false;   // padded in some mode k >= 1
                for (int k = d - 1; k >= 1; --k) {
                    if (rem % a.out_R[k] >= rout[k]) pin = true;
                    rem /= a.out_R[k];
                }
                for (int b0 = pin ? 0 : rout[0]; b0 < a.out_R[0]; ++b0) {
                    cx<float> *o = out + ((int64_t)b0 * inner + j) * a.nv;
                    int v = 0;
                    if (vec)
                        for (; v + 1 < a.nvc; v += 2) *reinterpret_cast<float4 *>(o + v) = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (; v < a.nvc; ++v) o[v] = cx<float>{0.f, 0.f};
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (tid == 0 && abort_sh) {
        // after a give-up, the copies of the last STAGES chunks may still be landing
        for (int64_t gi = (issued > STAGES ? issued - STAGES : 0); gi < issued; ++gi)
            mbar_wait(&full_bar[gi % STAGES], (uint32_t)((gi / STAGES) & 1));
    }
    if (warp == 0) {
        __syncwarp();
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

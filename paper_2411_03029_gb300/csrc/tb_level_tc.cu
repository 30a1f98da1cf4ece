// Level passes of the apply (Alg. 2, steps 1 and 3) on the tcgen05 tensor
// cores: one persistent launch per pass, complex64 data, each mode product a
// two-term split-BF16 tensor-core product with FP32 accumulation in tensor
// memory.
//
// A level pass applies to every unit a chain of d mode products with the
// unit's own factor blocks (V / W on the source side, U^T / P^T on the target
// side; the unit of each pass is described in tb_mode.cu).  Step i of a chain
// contracts mode k = order[i]:
//     Y[.., o', ..] = sum_{i_k} op(A)[o', i_k] X[.., i_k, ..].
// With the rows of the step's operand X the entries of the other modes times
// the vc right-hand sides of the work item, and each complex value stored as
// an (re, im) pair, this is the real product D = X B^T with
//     B[2 o'][2 i] = Re a, B[2 o'][2 i + 1] = -Im a,
//     B[2 o' + 1][2 i] = Im a, B[2 o' + 1][2 i + 1] = Re a      (a = op(A)[o', i]),
// so D[r][2 o'] = Re y, D[r][2 o' + 1] = Im y.  X = Xh + Xl and B = Bh + Bl in
// BF16 (hi = rn(v), lo = rn(v - hi)).  The operand stores each complex value
// as (hi re, hi im, lo re, lo im), i.e. K runs over [Xh | Xl] interleaved per
// value, and two MMAs per K-step accumulate in one TMEM accumulator
//     X B1^T = Xh Bh + Xl Bh    (B1 = Bh repeated for the lo slots)
//     X B2^T = Xh Bl            (B2 = Bl, zero for the lo slots),
// dropping only Xl Bl (below 2^-16 relative).  Operands live in shared memory
// in the 32-byte-swizzled K-major layout (tb_tc.cuh), 128-row tiles (MMA
// M = 128), N = 2 o padded to 16, K padded to 4 complex per K-step (the
// padded columns are zero in both operands).
//
// Block: two warpgroups of 128 threads, one block per SM, 512 TMEM columns
// (256 per warpgroup).  A warpgroup runs chains: it stages the chain's factor
// operands, then per step one thread issues the MMAs and commits to the
// warpgroup's mbarrier, and the 128 threads (thread = TMEM lane = operand row)
// read the accumulator and write the next step's operand, split into BF16
// pairs, into the same buffer (the step's MMAs have completed).  The other
// warpgroup's work overlaps each wait.  The rows of a step's operand
// enumerate its other modes in an order the host picks per step (the one
// whose 8-byte accumulator stores into the next operand, simulated for one
// warp, take the fewest shared-memory wavefronts).
//  * LeafIn / LeafOut: each warpgroup takes its own work items (a leaf tile
//    and a chunk of vc RHS).
//  * Split: the block takes an item (a group of 2^d children, vc RHS) and
//    stages the combined parent tile once as the step-0 operand shared by
//    both warpgroups; warpgroup g runs children g, g + 2, ...
//  * Gather: warpgroup g runs children g, g + 2, ..., each from its own child
//    tile, and accumulates the last step of all its children in one TMEM
//    accumulator (the last step's rows are the same for every child); at the
//    end of the item the block adds the two warpgroups' accumulators and
//    writes the 2^d parent tiles.  The sum order is fixed: deterministic.
// Every mbarrier wait is bounded; a warpgroup whose wait expires records
// TB_ETIMEOUT, stops issuing MMAs and runs its loops to the end without them,
// so every barrier is still reached; before freeing tensor memory each
// warpgroup waits (bounded) for its last MMAs.
#include "tb_kernels.cuh"
#include "tb_tc.cuh"

namespace tb {

namespace {

constexpr int LT_THREADS = 256;
constexpr uint32_t LT_TMEM_COLS = 512, LT_WG_COLS = 256;
constexpr int LT_MAXCH = 8;

TB_DEV float2 zero2() { return make_float2(0.f, 0.f); }

// Per-mode indices (d <= 3) addressed by a run-time mode: selects on three
// registers instead of a local array.
struct I3 {
    int v0, v1, v2;
    TB_DEV int get(int j) const { return j == 0 ? v0 : (j == 1 ? v1 : v2); }
    TB_DEV void set(int j, int x) {
        if (j == 0) v0 = x;
        else if (j == 1) v1 = x;
        else v2 = x;
    }
};

}  // namespace

__global__ void __launch_bounds__(LT_THREADS, 1) k_level_tc(const LevelTcArgs A) {
    using namespace tc;
    const LevelArgs &a = A.L;
    extern __shared__ __align__(16) unsigned char lt_raw[];
    // the operand area starts at the next 1024-byte boundary; indexing lt_raw
    // keeps every store in the shared state space (no aliasing with the
    // global loads, which may then be issued ahead of them)
    const uint32_t pad = (1024u - (smem_u32(lt_raw) & 1023u)) & 1023u;
    unsigned char *sm = lt_raw + pad;
    const uint32_t sbase = smem_u32(lt_raw) + pad;
    __shared__ __align__(8) uint64_t mbar[2], dbar[2];
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_wg[2];
    __shared__ const cx<float> *s_fac[LT_MAXCH][LTC_MAXD];
    __shared__ const float2 *s_in[LT_MAXCH];
    __shared__ float2 *s_out[LT_MAXCH];
    __shared__ float2 *s_par[LT_MAXCH];

    const int tid = threadIdx.x, wg = tid >> 7, wt = tid & 127, q = (tid >> 5) & 3, lane = tid & 31;
    const int d = a.d, vc = a.vc, lvc = a.lvc;
    const bool leaf = a.pass == 0 || a.pass == 3;
    const int nchild = leaf ? 1 : (1 << d);
    I3 goff{0, 0, 0};   // offset of each mode's leaf table
    int gtab = 0;
    for (int i = 0; i < d; ++i) {
        goff.set(i, gtab);
        gtab += a.cb[i];
    }

    if (tid == 0) {
        for (int g = 0; g < 2; ++g) {
            mbar_init(&mbar[g], 1);
            mbar_init(&dbar[g], 1);
            abort_wg[g] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(LT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh + (uint32_t)wg * LT_WG_COLS;
    const uint32_t woff = A.wg_off[wg];                  // this warpgroup's operand buffer (offset in sm)
    const uint32_t foff = woff + A.fac_off;              // its factor operands
    int64_t *gstr = reinterpret_cast<int64_t *>(sm + woff + A.tab_off);   // leaf tables
    int *gt = reinterpret_cast<int *>(gstr + gtab);
    volatile int *abt = &abort_wg[wg];
    uint32_t phase = 0;   // parity of this warpgroup's next MMA completion
    auto st8 = [&](uint32_t off, uint2 v) { *reinterpret_cast<uint2 *>(sm + off) = v; };

    // ---------------------------------------------------------------- item
    // Pointers of item g into the slots [slot, slot + nchild): factor blocks,
    // output / input tiles and (groups) the 2^d parent tiles; leaf tables of
    // grid indices.  Run by 64 threads, j = 0..63.
    auto decode = [&](int64_t g, int slot, int j) {
        const int Lc = a.Lc, lgs = a.lgs, lvl = a.lvl;
        const int64_t sflat = g & (((int64_t)1 << (lgs * d)) - 1);
        const int64_t rest = g >> (lgs * d);
        int sig[LTC_MAXD], pMk[LTC_MAXD];
        for (int i = 0; i < d; ++i) sig[i] = (int)((sflat >> (lgs * (d - 1 - i))) & ((1 << lgs) - 1));
        int64_t F = rest, pM = 0;
        if (!leaf) {
            const int64_t nMp = (int64_t)1 << (d * (lvl - 1));
            pM = rest & (nMp - 1);
            F = rest >> (d * (lvl - 1));
            for (int i = 0; i < d; ++i) pMk[i] = (int)((pM >> ((lvl - 1) * (d - 1 - i))) & ((1 << (lvl - 1)) - 1));
        }
        if (j < nchild) {
            int64_t M = 0;
            if (!leaf)
                for (int i = 0; i < d; ++i) M = (M << lvl) | (2 * pMk[i] + ((j >> (d - 1 - i)) & 1));
            for (int k = 0; k < d; ++k) s_fac[slot + j][k] = fac_block<float>(a.fac, k, F, M, sig[k], d, Lc);
            if (a.pass == 0 || a.pass == 1)
                s_out[slot + j] = reinterpret_cast<float2 *>(a.lout.p + tile_index<float>(a.lout, F, M, sflat, a.nF, d) *
                                                                            a.lout.tsize * a.nv);
            else
                s_in[slot + j] = reinterpret_cast<const float2 *>(
                    a.lin.p + tile_index<float>(a.lin, F, M, sflat, a.nF, d) * a.lin.tsize * a.nv);
        }
        if (!leaf && j < (1 << d)) {
            int64_t sp = 0;
            for (int i = 0; i < d; ++i) sp = (sp << (lgs + 1)) | (2 * sig[i] + ((j >> (d - 1 - i)) & 1));
            const TileBuf<float> &tb = a.pass == 1 ? a.lin : a.lout;
            s_par[j] = reinterpret_cast<float2 *>(tb.p + tile_index<float>(tb, F, pM, sp, a.nF, d) * tb.tsize * a.nv);
        }
        if (leaf) {
            for (int i = 0; i < d; ++i) {
                const int64_t Fi = (F >> (Lc * (d - 1 - i))) & ((1 << Lc) - 1);
                for (int b = j; b < a.cb[i]; b += 64) {
                    const int gi = a.perm[i][Fi * a.nmid[i] + (int64_t)sig[i] * a.cb[i] + b];
                    gt[goff.get(i) + b] = gi;
                    gstr[goff.get(i) + b] = (int64_t)gi * a.user.gstride[i];
                }
            }
        }
    };

    // Row r of step S -> the index of each of its other modes; returns the RHS.
    auto row_idx = [&](const LtcStep &S, int r, I3 &idx) -> int {
        const int v = r & (vc - 1);
        int rest = r >> lvc;
        for (int j = S.nod - 1; j >= 0; --j) {
            const int dj = S.od[j];
            const int t = rest / dj;
            idx.set(S.om[j], rest - t * dj);
            rest = t;
        }
        return v;
    };

    // ------------------------------------------------- step-0 operand staging
    // The input of the chain (C order over the input dims m_k, vc RHS
    // innermost) as the operand of step 0: thread t of nt owns rows t, t + nt,
    // ...; it loads the row's m inputs along mode k0, eight at a time with all
    // eight in flight, and writes them split, zeros in the padded K columns.
    auto stage_a0 = [&](int c, uint32_t aoff, int t, int nt, int v0, int nvc) {
        const LtcStep &S = A.st[0];
        const int k0 = S.k, m0 = S.m, kpad = S.ks * 4;
        const uint32_t a_rs = S.a_rs;
        I3 istr{1, 1, 1};   // entry stride of each mode in the input's C order
        for (int k = d - 2; k >= 0; --k) istr.set(k, istr.get(k + 1) * a.m[k + 1]);
        for (int r = t; r < S.rows; r += nt) {
            I3 idx{0, 0, 0};
            const int v = row_idx(S, r, idx);
            const bool live = v < nvc;
            const int64_t col = (int64_t)v0 + v;
            // base of the row's fiber along mode k0 and the step between entries
            const float2 *src = nullptr;
            int64_t stp = 0;
            const float2 *src1 = nullptr;   // Split: second parent along mode k0
            int half = m0;
            if (a.pass == 0) {
                int64_t ub = 0;
                for (int j = 0; j < d; ++j)
                    if (j != k0) ub += gstr[goff.get(j) + idx.get(j)];
                src = reinterpret_cast<const float2 *>(a.user.p) + ub * a.nv + col;
            } else if (a.pass == 1) {
                int bits = 0, er = 0, es = 1, ek = 0;
                for (int j = d - 1; j >= 0; --j) {
                    if (j == k0) {
                        ek = es;
                    } else {
                        const int ij = idx.get(j), bj = ij >= a.Rp[j];
                        bits |= bj << (d - 1 - j);
                        er += (ij - bj * a.Rp[j]) * es;
                    }
                    es *= a.Rp[j];
                }
                half = a.Rp[k0];
                src = s_par[bits] + (int64_t)er * a.nv + col;   // bit of mode k0 clear
                src1 = s_par[bits | (1 << (d - 1 - k0))] + (int64_t)er * a.nv + col;
                stp = (int64_t)ek * a.nv;
            } else {
                int e = 0;
                for (int j = 0; j < d; ++j)
                    if (j != k0) e += idx.get(j) * istr.get(j);
                src = s_in[c] + (int64_t)e * a.nv + col;
                stp = (int64_t)istr.get(k0) * a.nv;
            }
            const int64_t *gk = gstr + goff.get(k0);
            // the whole fiber first (up to 32 values in flight), then the stores
            float2 x[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                x[u] = zero2();
                if (u >= m0 || !live) continue;
                const float2 *p;
                if (a.pass == 0) p = src + gk[u] * a.nv;
                else if (a.pass == 1) p = u < half ? src + u * stp : src1 + (u - half) * stp;
                else p = src + u * stp;
                x[u] = __ldg(p);
            }
#pragma unroll
            for (int u = 0; u < 32; ++u)
                if (u < kpad)
                    st8(aoff + (uint32_t)(u >> 2) * a_rs + sw32c((uint32_t)r, (uint32_t)(u & 3)),
                        split_pair(x[u].x, x[u].y));
        }
    };

    // ------------------------------------------------------ factor staging
    // B1, B2 of every step of child c (rows 2 o', 2 o' + 1 of the split real
    // form of op(A), zero beyond o and m).  Thread wt takes K column
    // ii = 4 s + (wt & 3) and output rows o' = wt >> 2, + 32, ...
    auto stage_b = [&](int slot) {
        for (int i = 0; i < d; ++i) {
            const LtcStep &S = A.st[i];
            const int k = S.k, nO = S.np >> 1, cols = a.fac.cols[k], ks = S.ks, o = S.o, m = S.m;
            const uint32_t b_rs = S.b_rs, b_half = S.b_half;
            const cx<float> *src = s_fac[slot][k];
            const uint32_t bb = foff + S.b_off;
            const int per = (nO + 31) >> 5;   // output rows per thread and K-step (MMA N <= 256: <= 4)
            const int trans = a.trans, conj = a.conj;
            for (int s0 = 0; s0 < ks; s0 += 8) {
                // loads of up to 8 K-steps x 4 output rows first (one round), then the stores
                cx<float> f[8][4];
#pragma unroll
                for (int sj = 0; sj < 8; ++sj)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int ii = 4 * (s0 + sj) + (wt & 3), oo = (wt >> 2) + 32 * j;
                        const bool ok = s0 + sj < ks && j < per && oo < o && ii < m;
                        f[sj][j] = ok ? (trans ? src[ii * cols + oo] : src[oo * cols + ii]) : cx<float>{0.f, 0.f};
                    }
#pragma unroll
                for (int sj = 0; sj < 8; ++sj) {
                    if (s0 + sj >= ks) break;
                    const int ii = 4 * (s0 + sj) + (wt & 3);
                    const uint32_t reg = bb + (uint32_t)(s0 + sj) * b_rs;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int oo = (wt >> 2) + 32 * j;
                        if (j >= per || oo >= nO) continue;
                        const float fy = conj ? -f[sj][j].y : f[sj][j].y;
                        const uint2 re = split_pair(f[sj][j].x, -fy), im = split_pair(fy, f[sj][j].x);
                        const uint32_t a0 = reg + sw32c((uint32_t)(2 * oo), (uint32_t)(ii & 3));
                        const uint32_t a1 = reg + sw32c((uint32_t)(2 * oo + 1), (uint32_t)(ii & 3));
                        st8(a0, make_uint2(re.x, re.x));            // B1: hi for the hi and lo slots
                        st8(a1, make_uint2(im.x, im.x));
                        st8(a0 + b_half, make_uint2(re.y, 0u));     // B2: lo for the hi slots
                        st8(a1 + b_half, make_uint2(im.y, 0u));
                    }
                }
            }
        }
    };

    // ------------------------------------------------------------- one step
    // MMAs of step i (operand at aoff), then the wait for them.
    auto mma_step = [&](int i, uint32_t aoff, bool acc_in) {
        const LtcStep &S = A.st[i];
        fence_proxy_async();   // this thread's operand writes -> visible to the MMA
        wg_sync(wg);
        if (wt == 0 && !*abt) {
            tc_fence_after();
            const uint32_t bb = sbase + foff + S.b_off, ab = sbase + aoff;
            const int tiles = S.tiles, ks = S.ks, np = S.np;
            const uint32_t a_rs = S.a_rs, b_rs = S.b_rs, b_half = S.b_half, dcol = tmem + S.tcol, idesc = S.idesc;
            for (int t = 0; t < tiles; ++t) {
                const uint32_t dt = dcol + (uint32_t)(t * np);
                for (int s = 0; s < ks; ++s) {
                    const uint64_t ad = sdesc32(ab + (uint32_t)s * a_rs + (uint32_t)t * 4096u);
                    const uint32_t b1 = bb + (uint32_t)s * b_rs;
                    mma_bf16_nc(dt, ad, sdesc32(b1), idesc, (s > 0 || acc_in) ? 1u : 0u);
                    mma_bf16_nc(dt, ad, sdesc32(b1 + b_half), idesc, 1u);
                }
            }
            mma_commit(&mbar[wg]);
        }
        // only the issuing thread polls the mbarrier; the others wait at the
        // warpgroup barrier, which takes no issue slots
        if (wt == 0) {
            if (!mbar_wait(&mbar[wg], phase, abt)) {
                if (atomicExch(&abort_wg[wg], 1) == 0 && A.err) atomicExch(A.err, (int)TB_ETIMEOUT);
            }
            tc_fence_before();
        }
        phase ^= 1u;
        wg_sync(wg);
        tc_fence_after();
    };

    // The accumulator of step S, tile t, this thread's lane, 16 columns (8
    // complex outputs o' = 8 ch .. 8 ch + 7) at a time: f(ch, values).
    auto for_acc = [&](int np, uint32_t ta, auto &&f) {
        for (int c0 = 0; c0 * 16 < np; c0 += 3) {
            uint32_t r[48];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if ((c0 + j) * 16 < np) tmem_ld16_nc(ta + 16u * (c0 + j), r + 16 * j);
                else
#pragma unroll
                    for (int u = 0; u < 16; ++u) r[16 * j + u] = 0u;
            }
            tmem_wait_regs<3>(r);
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if ((c0 + j) * 16 < np) f(c0 + j, r + 16 * j);
        }
    };

    // Accumulator of step i -> operand of step i + 1 in this warpgroup's buffer.
    auto to_next = [&](int i) {
        const LtcStep &S = A.st[i], &N = A.st[i + 1];
        const int kpad = N.ks * 4, tiles = S.tiles, rows = S.rows, np = S.np, o = S.o, Sk = S.k, Nk = N.k, Nm = N.m;
        const uint32_t n_rs = N.a_rs, dcol = tmem + ((uint32_t)(32 * q) << 16) + S.tcol;
        int nr[LTC_MAXD];
        for (int j = 0; j < LTC_MAXD; ++j) nr[j] = j < d ? N.rstr[j] : 0;
        const int step = N.rstr[Sk];
        for (int t = 0; t < tiles; ++t) {
            const int r = t * 128 + 32 * q + lane;
            const bool live = r < rows;
            I3 idx{0, 0, 0};
            const int v = row_idx(S, live ? r : 0, idx);
            int base = v;
#pragma unroll
            for (int j = 0; j < LTC_MAXD; ++j)
                if (j < d && j != Sk) base += idx.get(j) * nr[j];
            const int kp = idx.get(Nk);
            const uint32_t ab = woff + (uint32_t)(kp >> 2) * n_rs;
            const uint32_t kc = (uint32_t)(kp & 3);
            for_acc(np, dcol + (uint32_t)(t * np), [&](int ch, const uint32_t *c) {
                if (!live) return;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int oo = 8 * ch + u;
                    if (oo >= o) break;
                    st8(ab + sw32c((uint32_t)(base + oo * step), kc),
                        split_pair(__uint_as_float(c[2 * u]), __uint_as_float(c[2 * u + 1])));
                }
            });
            // the row owning K column m - 1 also clears the padded columns of its rows
            if (live && kp == Nm - 1) {
                for (int oo = 0; oo < o; ++oo) {
                    const uint32_t rr = (uint32_t)(base + oo * step);
                    for (int z = Nm; z < kpad; ++z)
                        st8(woff + (uint32_t)(z >> 2) * n_rs + sw32c(rr, (uint32_t)(z & 3)), make_uint2(0u, 0u));
                }
            }
        }
    };

    // Accumulator of the last step -> the chain's output (level tile or user tensor).
    auto to_out = [&](int c, int v0, int nvc) {
        const LtcStep &S = A.st[d - 1];
        for (int t = 0; t < S.tiles; ++t) {
            const int r = t * 128 + 32 * q + lane;
            I3 idx{0, 0, 0};
            const int v = row_idx(S, r < S.rows ? r : 0, idx);
            const bool live = r < S.rows && v < nvc;
            const int64_t col = (int64_t)v0 + v;
            float2 *dst;
            int64_t stp = 0;
            const int64_t *gk = gstr + goff.get(S.k);
            if (a.pass == 3) {
                int64_t ub = 0;
                for (int j = 0; j < d; ++j)
                    if (j != S.k) ub += gstr[goff.get(j) + idx.get(j)];
                dst = reinterpret_cast<float2 *>(a.user.p) + ub * a.nv + col;
            } else {
                int e = 0;
                for (int j = 0; j < d; ++j)
                    if (j != S.k) e += idx.get(j) * S.tstr[j];
                dst = s_out[c] + (int64_t)e * a.nv + col;
                stp = (int64_t)S.tstr[S.k] * a.nv;
            }
            for_acc(S.np, tmem + ((uint32_t)(32 * q) << 16) + S.tcol + (uint32_t)(t * S.np),
                    [&](int ch, const uint32_t *cc) {
                if (!live) return;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int oo = 8 * ch + u;
                    if (oo >= S.o) break;
                    const float2 y = make_float2(__uint_as_float(cc[2 * u]), __uint_as_float(cc[2 * u + 1]));
                    if (a.pass == 3) dst[gk[oo] * a.nv] = y;
                    else dst[oo * stp] = y;
                }
            });
        }
    };

    // Runs the chain of child c (step-0 operand in place at a0off).
    auto chain = [&](int c, int slot, uint32_t a0off, bool acc_last, int v0, int nvc) {
        stage_b(slot);
        for (int i = 0; i < d; ++i) {
            mma_step(i, i == 0 ? a0off : woff, i == d - 1 && acc_last);
            if (i + 1 < d) to_next(i);
            else if (a.pass != 2) to_out(c, v0, nvc);
            tc_fence_before();
        }
    };

    if (leaf) {
        // --------------------------------------------- leaf passes: per warpgroup
        for (int64_t item = (int64_t)blockIdx.x * 2 + wg; item < a.nitems; item += (int64_t)gridDim.x * 2) {
            const int64_t g = item / a.nq;
            const int qv = (int)(item - g * a.nq);
            const int v0 = qv * vc;
            const int nvc = (int)(a.nv - v0 < vc ? a.nv - v0 : vc);
            wg_sync(wg);   // the previous item's tables and pointers are no longer read
            if (wt < 64) decode(g, wg, wt);
            wg_sync(wg);
            stage_a0(wg, woff, wt, 128, v0, nvc);
            chain(wg, wg, woff, false, v0, nvc);
        }
    } else {
        // -------------------------------------------- group passes: per block
        const bool split = a.pass == 1;
        for (int64_t item = blockIdx.x; item < a.nitems; item += gridDim.x) {
            const int64_t g = item / a.nq;
            const int qv = (int)(item - g * a.nq);
            const int v0 = qv * vc;
            const int nvc = (int)(a.nv - v0 < vc ? a.nv - v0 : vc);
            __syncthreads();   // the previous item is finished
            if (tid < 64) decode(g, 0, tid);
            __syncthreads();
            if (split) {
                stage_a0(0, A.a0_off, tid, LT_THREADS, v0, nvc);
                fence_proxy_async();
                __syncthreads();
            }
            bool first = true;
            for (int c = wg; c < nchild; c += 2) {
                if (!split) stage_a0(c, woff, wt, 128, v0, nvc);
                chain(c, c, split ? A.a0_off : woff, !split && !first, v0, nvc);
                first = false;
            }
            if (!split) {
                // Gather: the two warpgroups' accumulators -> the 2^d parent tiles
                // (combined parent tile of dims 2 Rp, entry bit of mode k set
                // where its index is >= Rp_k)
                tc_fence_before();
                __syncthreads();
                tc_fence_after();
                const LtcStep &S = A.st[d - 1];
                for (int t = wg; t < S.tiles; t += 2) {
                    const int r = t * 128 + 32 * q + lane;
                    I3 idx{0, 0, 0};
                    const int v = row_idx(S, r < S.rows ? r : 0, idx);
                    const bool live = r < S.rows && v < nvc;
                    int bits = 0, er = 0, es = 1, ek = 0;
                    for (int j = d - 1; j >= 0; --j) {
                        if (j == S.k) {
                            ek = es;
                        } else {
                            const int ij = idx.get(j), bj = ij >= a.Rp[j];
                            bits |= bj << (d - 1 - j);
                            er += (ij - bj * a.Rp[j]) * es;
                        }
                        es *= a.Rp[j];
                    }
                    const int half = a.Rp[S.k], kb = 1 << (d - 1 - S.k);
                    const int64_t col = (int64_t)v0 + v;
                    const uint32_t ta = tmem_sh + ((uint32_t)(32 * q) << 16) + S.tcol + (uint32_t)(t * S.np);
                    for (int ch = 0; ch * 16 < S.np; ch += 2) {
                        uint32_t c0[32], c1[32];   // two chunks of each warpgroup's accumulator
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            if ((ch + j) * 16 < S.np) {
                                tmem_ld16_nc(ta + 16u * (ch + j), c0 + 16 * j);
                                tmem_ld16_nc(ta + LT_WG_COLS + 16u * (ch + j), c1 + 16 * j);
                            } else {
#pragma unroll
                                for (int u = 0; u < 16; ++u) c0[16 * j + u] = c1[16 * j + u] = 0u;
                            }
                        }
                        tmem_wait_regs<2>(c0);
#pragma unroll
                        for (int u = 0; u < 32; ++u) asm volatile("" : "+r"(c1[u]));
                        if (!live) continue;
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int oo = 8 * ch + u;
                            if (oo >= S.o) break;
                            const int hi = oo >= half;
                            float2 *dst = s_par[bits | (hi ? kb : 0)];
                            dst[((int64_t)er + (int64_t)(oo - hi * half) * ek) * a.nv + col] =
                                make_float2(__uint_as_float(c0[2 * u]) + __uint_as_float(c1[2 * u]),
                                            __uint_as_float(c0[2 * u + 1]) + __uint_as_float(c1[2 * u + 1]));
                        }
                    }
                }
                tc_fence_before();
            }
        }
    }

    // every MMA of this warpgroup has completed before tensor memory is freed
    if (wt == 0) {
        mma_commit(&dbar[wg]);
        mbar_wait(&dbar[wg], 0);
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_sh), "r"(LT_TMEM_COLS)
                     : "memory");
    }
}

cudaError_t launch_level_tc(const LevelTcArgs &a, int blocks, cudaStream_t st) {
    cudaError_t e = set_smem_once((const void *)k_level_tc, a.smem);
    if (e != cudaSuccess) return e;
    if (blocks <= 0 || a.L.nitems <= 0) return cudaSuccess;
    k_level_tc<<<blocks, LT_THREADS, a.smem, st>>>(a);
    return cudaGetLastError();
}

int level_tc_threads() { return LT_THREADS; }

}  // namespace tb

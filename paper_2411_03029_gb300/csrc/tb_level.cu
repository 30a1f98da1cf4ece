// Level passes of the apply (Alg. 2, steps 1 and 3) as ONE persistent launch
// per pass, complex64 data, FP32 arithmetic.
//
// A level pass applies to every unit a chain of d mode products with the
// unit's own factor blocks (V / W on the source side, U^T / P^T on the target
// side; see tb_mode.cu for the unit of each pass).  Here one launch covers the
// whole pass: a thread block takes work items (a unit or a group of 2^d
// children, and a chunk of VC right-hand sides), runs the d mode products of
// the item back to back and keeps the intermediates in shared memory (two
// ping-pong buffers), so only the pass's input and output cross HBM.
//
//  * Mode order.  The mode products of a chain commute (each acts on its own
//    index), so the host picks the order with the fewest multiply-adds (the
//    modes that shrink the tile most first on the source side, the ones that
//    grow it least first on the target side).
//  * Arithmetic.  Each product y = A x (A staged in shared memory, x a fiber of
//    the item's tensor) is accumulated with three real products per complex
//    product (Gauss): T1 = sum ar xr, T2 = sum ai xi, T3 = sum (ar + ai)(xr + xi),
//    y = (T1 - T2, T3 - T1 - T2), i.e. three FMAs instead of four, paired over
//    two consecutive output rows with fma.rn.f32x2.  The factor is staged in
//    planar form (ar, ai, ar + ai), so a warp's lanes read it as broadcasts.
//  * Tasks.  A step is split into tasks (column, chunk of OB output rows);
//    consecutive threads take consecutive columns of the same chunk.
//  * Groups.  A Split reads the combined parent tile (2^d parent tiles) in its
//    first product and writes each child; a Gather accumulates the children,
//    in a fixed order, into a shared-memory copy of the combined parent tile in
//    its last product (each thread owns the same output entries for every
//    child: deterministic, no atomics) and writes it out once.
#include "tb_kernels.cuh"

namespace tb {

constexpr int LV_THREADS = 256;
constexpr int LV_MAXCH = 8;   // children of a group (d <= 3)

namespace {

TB_DEV float2 f2(float a, float b) { return make_float2(a, b); }

TB_DEV float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Where a step reads its input / writes its output.
enum LvSrc : int { LS_SCRATCH = 0, LS_TILE = 1, LS_PARENTS = 2, LS_USER = 3, LS_ACC = 4 };

struct Step {
    int k, m, o;
    int pre, post;          // products of the current dims before / after mode k
    int curd[MAXD];         // current dims (output dims for processed modes)
};

}  // namespace

// One task: output rows [a0, a0 + OB) of column (p, qe, vl) of step s for child
// c.  The input is a shared-memory tensor (C order over the current dims, the
// vc RHS innermost).  Factor of the step, staged per input b and output pair
// e = a / 2: fRI[b][e] = (ar_a, ar_a+1, ai_a, ai_a+1), fS[b][e] = (ar_a + ai_a,
// ar_a+1 + ai_a+1).  All index arithmetic is 32-bit: an item's tensors are small.
template <int OB, int DST>
TB_DEV void lv_task(const LevelArgs &a, const Step &s, int c, int p, int qe, int vl, int a0, int v0,
                    const float4 *__restrict__ fRI, const float2 *__restrict__ fS, int ldp,
                    const float2 *__restrict__ sin_, float2 *__restrict__ sout, float2 *tout, const int *gt,
                    const int *goff) {
    const int vc = a.vc, m = s.m;
    const float2 *x0 = sin_ + ((p * m) * s.post + qe) * vc + vl;
    const int xs = s.post * vc;
    constexpr int NP = OB / 2;
    float2 T1[NP], T2[NP], T3[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) T1[i] = T2[i] = T3[i] = f2(0.f, 0.f);
    const int e0 = a0 >> 1;
#pragma unroll 2
    for (int b = 0; b < m; ++b) {
        const float2 x = x0[b * xs];
        const float2 xr = f2(x.x, x.x), xi = f2(x.y, x.y);
        const float xsum = x.x + x.y;
        const float2 xsv = f2(xsum, xsum);
        const float4 *ri = fRI + b * ldp + e0;
        const float2 *sp = fS + b * ldp + e0;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const float4 v = ri[i];
            const float2 w = sp[i];
            T1[i] = ffma2(f2(v.x, v.y), xr, T1[i]);
            T2[i] = ffma2(f2(v.z, v.w), xi, T2[i]);
            T3[i] = ffma2(w, xsv, T3[i]);
        }
    }
    const int o = s.o;
    auto result = [&](int i) -> float2 {
        const float t1 = (i & 1) ? T1[i >> 1].y : T1[i >> 1].x;
        const float t2 = (i & 1) ? T2[i >> 1].y : T2[i >> 1].x;
        const float t3 = (i & 1) ? T3[i >> 1].y : T3[i >> 1].x;
        return f2(t1 - t2, t3 - t1 - t2);
    };
    if (DST == LS_SCRATCH || DST == LS_ACC) {
        float2 *y = sout + ((p * o) * s.post + qe) * vc + vl;
        const int ys = s.post * vc;
#pragma unroll
        for (int i = 0; i < OB; ++i) {
            if (a0 + i >= o) continue;
            float2 v = result(i);
            if (DST == LS_ACC && c > 0) {
                const float2 old = y[(a0 + i) * ys];
                v.x += old.x;
                v.y += old.y;
            }
            y[(a0 + i) * ys] = v;
        }
    } else if (DST == LS_TILE) {
        float2 *y = tout + ((int64_t)((p * o) * s.post + qe)) * a.nv + v0 + vl;
        const int64_t ys = (int64_t)s.post * a.nv;
#pragma unroll
        for (int i = 0; i < OB; ++i)
            if (a0 + i < o) y[(a0 + i) * ys] = result(i);
    } else {   // LS_USER: grid positions through the leaf's tree ordering
        const int d = a.d, k = s.k;
        int64_t ub = 0;
        int pp = p, qq = qe;
        for (int j = d - 1; j > k; --j) {
            const int ij = qq % s.curd[j];
            qq /= s.curd[j];
            ub += (int64_t)gt[goff[j] + ij] * a.user.gstride[j];
        }
        for (int j = k - 1; j >= 0; --j) {
            const int ij = pp % s.curd[j];
            pp /= s.curd[j];
            ub += (int64_t)gt[goff[j] + ij] * a.user.gstride[j];
        }
        float2 *y = reinterpret_cast<float2 *>(a.user.p) + ub * a.nv + v0 + vl;
        const int64_t ys = a.user.gstride[k] * a.nv;
        const int *gk = gt + goff[k];
#pragma unroll
        for (int i = 0; i < OB; ++i)
            if (a0 + i < o) y[(int64_t)gk[a0 + i] * ys] = result(i);
    }
}

template <int OB, int DST>
TB_DEV void lv_step(const LevelArgs &a, const Step &s, int c, int v0, int nvc, const float *fbase, int ldp,
                    const float2 *sin_, float2 *sout, float2 *tout, const int *gt, const int *goff) {
    const float4 *fRI = reinterpret_cast<const float4 *>(fbase);
    const float2 *fS = reinterpret_cast<const float2 *>(fbase + 4 * s.m * ldp);
    const int lvc = a.lvc, vc = a.vc;
    const int colsr = s.pre * s.post;          // columns without the RHS index
    const int nch = (s.o + OB - 1) / OB;
    const int tasks = (colsr * nch) << lvc;
    for (int t = threadIdx.x; t < tasks; t += blockDim.x) {
        const int vl = t & (vc - 1);
        if (vl >= nvc) continue;
        const int r = t >> lvc;
        const int ch = r / colsr;
        const int col = r - ch * colsr;
        const int p = col / s.post, qe = col - p * s.post;
        lv_task<OB, DST>(a, s, c, p, qe, vl, ch * OB, v0, fRI, fS, ldp, sin_, sout, tout, gt, goff);
    }
}

template <int OB>
__global__ void __launch_bounds__(LV_THREADS, 2) k_level(const LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float *fsm = reinterpret_cast<float *>(smraw);             // staged factors of one child
    int *gt = reinterpret_cast<int *>(fsm + a.fac_floats);      // leaf tree-order -> grid tables
    int64_t *gstr = reinterpret_cast<int64_t *>(smraw + a.off_gstr);   // the same x the axis stride
    __shared__ const cx<float> *s_fac[LV_MAXCH][MAXD];
    __shared__ const float2 *s_in[LV_MAXCH];
    __shared__ float2 *s_out[LV_MAXCH];
    __shared__ const float2 *s_par[LV_MAXCH];
    const int d = a.d, tid = threadIdx.x;
    const bool leaf = a.pass == 0 || a.pass == 3;
    const bool group = !leaf;
    const int nchild = group ? (1 << d) : 1;
    int goff[MAXD];
    {
        int off = 0;
        for (int i = 0; i < d; ++i) {
            goff[i] = off;
            off += a.cb[i];
        }
    }
    // shared-memory tensors: the step-0 input, two ping-pong intermediates and
    // (Gather) the combined parent tile
    float2 *inb = reinterpret_cast<float2 *>(smraw + a.off_in);
    float2 *scr0 = reinterpret_cast<float2 *>(smraw + a.off_s0);
    float2 *scr1 = reinterpret_cast<float2 *>(smraw + a.off_s1);
    float2 *acc = reinterpret_cast<float2 *>(smraw + a.off_acc);
    int64_t in_entries = 1;   // entries of the step-0 input per RHS
    for (int k = 0; k < d; ++k) in_entries *= a.m[k];
    for (int64_t item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const int64_t g = item / a.nq;
        const int q = (int)(item - g * a.nq);
        const int v0 = q * a.vc;
        const int nvc = (int)(a.nv - v0 < a.vc ? a.nv - v0 : a.vc);
        __syncthreads();   // the previous item's tables and factors are no longer read
        if (tid < 64) {
            const int Lc = a.Lc, lgs = a.lgs, lvl = a.lvl;
            const int64_t sflat = g & (((int64_t)1 << (lgs * d)) - 1);
            const int64_t rest = g >> (lgs * d);
            int sig[MAXD], pMk[MAXD];
            for (int i = 0; i < d; ++i) sig[i] = (int)((sflat >> (lgs * (d - 1 - i))) & ((1 << lgs) - 1));
            int64_t F = rest, pM = 0;
            if (!leaf) {
                const int64_t nMp = (int64_t)1 << (d * (lvl - 1));
                pM = rest & (nMp - 1);
                F = rest >> (d * (lvl - 1));
                for (int i = 0; i < d; ++i)
                    pMk[i] = (int)((pM >> ((lvl - 1) * (d - 1 - i))) & ((1 << (lvl - 1)) - 1));
            }
            const int j = tid;
            if (j < nchild) {
                int64_t M = 0;
                if (!leaf)
                    for (int i = 0; i < d; ++i) M = (M << lvl) | (2 * pMk[i] + ((j >> (d - 1 - i)) & 1));
                for (int k = 0; k < d; ++k) s_fac[j][k] = fac_block<float>(a.fac, k, F, M, sig[k], d, Lc);
                if (a.pass == 0 || a.pass == 1) {   // LeafIn: level-0 tile; Split: child tile j
                    s_out[j] = reinterpret_cast<float2 *>(a.lout.p + tile_index<float>(a.lout, F, M, sflat, a.nF, d) *
                                                                         a.lout.tsize * a.nv);
                } else {                            // LeafOut: level-0 tile; Gather: child tile j
                    s_in[j] = reinterpret_cast<const float2 *>(a.lin.p + tile_index<float>(a.lin, F, M, sflat, a.nF, d) *
                                                                             a.lin.tsize * a.nv);
                }
            }
            if (group && j < (1 << d)) {
                int64_t sp = 0;
                for (int i = 0; i < d; ++i) sp = (sp << (lgs + 1)) | (2 * sig[i] + ((j >> (d - 1 - i)) & 1));
                const TileBuf<float> &tb = a.pass == 1 ? a.lin : a.lout;
                s_par[j] = reinterpret_cast<const float2 *>(tb.p + tile_index<float>(tb, F, pM, sp, a.nF, d) * tb.tsize *
                                                                       a.nv);
            }
            if (leaf) {
                for (int i = 0; i < d; ++i) {
                    const int64_t Fi = (F >> (Lc * (d - 1 - i))) & ((1 << Lc) - 1);
                    for (int b = j; b < a.cb[i]; b += 64) {
                        const int gi = a.perm[i][Fi * a.nmid[i] + (int64_t)sig[i] * a.cb[i] + b];
                        gt[goff[i] + b] = gi;
                        gstr[goff[i] + b] = (int64_t)gi * a.user.gstride[i];
                    }
                }
            }
        }
        __syncthreads();
        // stage the step-0 input of the item (Gather: of each child, below) in
        // shared memory, C order over the input dims with the vc RHS innermost:
        // independent loads, many in flight per thread
        auto stage_input = [&](int c) {
            const int tot = (int)in_entries << a.lvc;
            for (int e0 = tid; e0 < tot; e0 += 4 * blockDim.x) {
                float2 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * blockDim.x;
                    v[u] = f2(0.f, 0.f);
                    if (e >= tot) continue;
                    const int vl = e & (a.vc - 1);
                    if (vl >= nvc) continue;
                    int rest = e >> a.lvc;
                    if (a.pass == 2 || a.pass == 3) {          // a level tile, C order over its dims
                        v[u] = s_in[c][(int64_t)rest * a.nv + v0 + vl];
                    } else if (a.pass == 1) {                  // combined parent tile of dims 2 Rp
                        int erest = 0, stride = 1, bits = 0;
                        for (int k = d - 1; k >= 0; --k) {
                            const int ik = rest % (2 * a.Rp[k]);
                            rest /= 2 * a.Rp[k];
                            const int bk = ik >= a.Rp[k];
                            bits |= bk << (d - 1 - k);
                            erest += (ik - bk * a.Rp[k]) * stride;
                            stride *= a.Rp[k];
                        }
                        v[u] = s_par[bits][(int64_t)erest * a.nv + v0 + vl];
                    } else {                                   // leaf of the user tensor, tree order
                        int64_t ub = 0;
                        for (int k = d - 1; k >= 0; --k) {
                            const int ik = rest & (a.cb[k] - 1);   // C_b is a power of two
                            rest >>= a.lcb[k];
                            ub += gstr[goff[k] + ik];
                        }
                        v[u] = reinterpret_cast<const float2 *>(a.user.p)[ub * a.nv + v0 + vl];
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * blockDim.x;
                    if (e < tot) inb[e] = v[u];
                }
            }
        };
        if (a.pass != 2) stage_input(0);
        for (int c = 0; c < nchild; ++c) {
            if (c > 0) __syncthreads();   // the previous child's last step is done with the factors
            if (a.pass == 2) stage_input(c);
            // stage the child's factors of every mode, [input b][output pair e]:
            // (ar_a, ar_a+1, ai_a, ai_a+1) and (ar + ai) pairs; rows a >= o_k are zero
            for (int k = 0; k < d; ++k) {
                const int mk = a.m[k], ok = a.o[k], ldp = a.lda[k] / 2;
                const int cols = a.fac.cols[k];
                const cx<float> *src = s_fac[c][k];
                float4 *dRI = reinterpret_cast<float4 *>(fsm + a.fac_off[k]);
                float2 *dS = reinterpret_cast<float2 *>(fsm + a.fac_off[k] + 4 * mk * ldp);
                for (int e = tid; e < mk * ldp; e += blockDim.x) {
                    const int b = e / ldp, pr = e - b * ldp;
                    cx<float> v[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int aa = 2 * pr + h;
                        v[h] = cx<float>{0.f, 0.f};
                        if (aa < ok) {
                            v[h] = a.trans ? src[b * cols + aa] : src[aa * cols + b];
                            if (a.conj) v[h].y = -v[h].y;
                        }
                    }
                    dRI[e] = make_float4(v[0].x, v[1].x, v[0].y, v[1].y);
                    dS[e] = f2(v[0].x + v[0].y, v[1].x + v[1].y);
                }
            }
            __syncthreads();
            for (int i = 0; i < d; ++i) {
                Step s;
                s.k = a.order[i];
                s.m = a.m[s.k];
                s.o = a.o[s.k];
                for (int j = 0; j < d; ++j) s.curd[j] = a.m[j];
                for (int ii = 0; ii < i; ++ii) s.curd[a.order[ii]] = a.o[a.order[ii]];
                s.pre = 1;
                s.post = 1;   // 32-bit: an item's tensors are far below 2^31 entries
                for (int j = 0; j < s.k; ++j) s.pre *= s.curd[j];
                for (int j = s.k + 1; j < d; ++j) s.post *= s.curd[j];
                const float2 *sin_ = (i & 1) ? scr0 : scr1;   // step i reads what step i - 1 wrote
                float2 *sout = (i & 1) ? scr1 : scr0;
                const float *fb = fsm + a.fac_off[s.k];
                const int ldp = a.lda[s.k] / 2;
                float2 *tout = s_out[c];
                if (i == 0) sin_ = inb;   // every step reads shared memory
                if (i + 1 < d) {
                    lv_step<OB, LS_SCRATCH>(a, s, c, v0, nvc, fb, ldp, sin_, sout, tout, gt, goff);
                } else {
                    if (a.pass == 3) lv_step<OB, LS_USER>(a, s, c, v0, nvc, fb, ldp, sin_, sout, tout, gt, goff);
                    else if (a.pass == 2) lv_step<OB, LS_ACC>(a, s, c, v0, nvc, fb, ldp, sin_, acc, tout, gt, goff);
                    else lv_step<OB, LS_TILE>(a, s, c, v0, nvc, fb, ldp, sin_, sout, tout, gt, goff);
                }
                if (i + 1 < d) __syncthreads();
            }
        }
        if (a.pass == 2) {
            // write the accumulated combined parent tile: entry (i_0..i_{d-1}) of dims
            // 2 Rp goes to parent tile (bits of i_k >= Rp_k) at its offset there
            __syncthreads();
            int64_t tot = a.vc;
            for (int k = 0; k < d; ++k) tot *= 2 * a.Rp[k];
            for (int64_t e = tid; e < tot; e += blockDim.x) {
                const int vl = (int)(e % a.vc);
                if (vl >= nvc) continue;
                int64_t rest = e / a.vc, erest = 0, stride = 1;
                int bits = 0;
                for (int k = d - 1; k >= 0; --k) {
                    const int ik = (int)(rest % (2 * a.Rp[k]));
                    rest /= 2 * a.Rp[k];
                    const int bk = ik >= a.Rp[k];
                    bits |= bk << (d - 1 - k);
                    erest += (int64_t)(ik - bk * a.Rp[k]) * stride;
                    stride *= a.Rp[k];
                }
                const_cast<float2 *>(s_par[bits])[erest * a.nv + v0 + vl] = acc[e];
            }
        }
    }
}

cudaError_t launch_level(const LevelArgs &a, int ob, int blocks, cudaStream_t st) {
    void (*fn)(const LevelArgs) = nullptr;
    switch (ob) {
        case 4: fn = k_level<4>; break;
        case 6: fn = k_level<6>; break;
        case 8: fn = k_level<8>; break;
        case 10: fn = k_level<10>; break;
        case 12: fn = k_level<12>; break;
        case 14: fn = k_level<14>; break;
        case 16: fn = k_level<16>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = set_smem_once((const void *)fn, a.smem);
    if (e != cudaSuccess) return e;
    if (blocks <= 0 || a.nitems <= 0) return cudaSuccess;
    fn<<<blocks, LV_THREADS, a.smem, st>>>(a);
    return cudaGetLastError();
}

bool level_ob_valid(int ob) { return ob >= 4 && ob <= 16 && (ob & 1) == 0; }

int level_threads() { return LV_THREADS; }
int level_max_children() { return LV_MAXCH; }

}  // namespace tb

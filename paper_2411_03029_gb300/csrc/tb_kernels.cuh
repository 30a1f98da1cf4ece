// Argument blocks and launchers of the construction and apply kernels.
#pragma once

#include <string>

#include "tb_common.cuh"

namespace tb {

// Record `msg` as the calling thread's tb_last_error() and return s.
tb_status fail_status(tb_status s, const std::string &msg);

// ------------------------------------------------------------- construction
struct IdArgs {
    int side;        // 0: source side (V, W; columns are source points of mode k)
                     // 1: target side (U, P; columns are target points of mode k)
    int d, l, Lc, separable;
    int n[MAXD], cb[MAXD];
    const int *perm[MAXD];        // tree position -> grid index (both sides)
    const double *own[MAXD];      // coordinates of the column side
    const double *oth[MAXD];      // coordinates of the other side
    KernelSpec ks;
    const int *pskel[MAXD];       // level l-1 skeletons (l > 0)
    const int *prank[MAXD];
    int pcap[MAXD], pR[MAXD];
    int *skel[MAXD];              // outputs
    int *rank[MAXD];
    c128 *fac[MAXD];
    int cap[MAXD], cin[MAXD];
    int rows_cap, rows_bits;
    double tol;
    int rank_max;
    uint32_t seed;
    int *err;
    int64_t nids;
    int ncmax;
};

struct CoreArgs {
    int d;
    int64_t P, nF;
    const int *dims;
    const int64_t *off;
    const int *tskel[MAXD];
    const int *sskel[MAXD];
    int tcap[MAXD], scap[MAXD];
    const double *xs[MAXD], *ys[MAXD];
    KernelSpec ks;
    c128 *out64;
    c64 *out32;
};

struct KronArgs {
    int Lc, Rt, Rs, tcap, scap;
    const int *trank, *srank, *tskel, *sskel;
    const double *xk, *yk;
    KernelSpec ks;
    c128 *out64;
    c64 *out32;
};

cudaError_t launch_interp_decomp(const IdArgs &a, cudaStream_t st);
cudaError_t launch_core_eval(const CoreArgs &a, cudaStream_t st);
cudaError_t launch_kron_eval(const KronArgs &a, cudaStream_t st);
cudaError_t launch_to_c64(const c128 *in, c64 *out, int64_t n, cudaStream_t st);
int id_max_columns();

// -------------------------------------------------------------------- apply
// A level tensor: P tiles of prod_k R[k] entries, each entry nv contiguous RHS.
// Tile index = (block << (lgseg * d)) + segment-tuple, block = M * nF + F
// (source layout, multiset M of the target tree, mid-level source multiset F)
// or F * nM + M (target layout).  Both give block = t * nF + s at level Lc.
template <class T>
struct TileBuf {
    cx<T> *p;
    int R[MAXD];
    int tsize;
    int lgseg;      // log2 of segments per mode at this level (Lc - l)
    int64_t nM;     // multisets at this level, 2^(d l)
    int layout;     // 0 source, 1 target
};

template <class R>
struct FacRef {
    const cx<R> *A[MAXD];
    const int *rank[MAXD];   // rank of each block (its rows past the rank are zero); may be null
    int rows[MAXD], cols[MAXD];
    int l, lgseg;
    int64_t nM;
    int separable;
};

// Tile index of (mid-level multiset F, multiset M, segment tuple sflat).
template <class R>
TB_DEV int64_t tile_index(const TileBuf<R> &b, int64_t F, int64_t M, int64_t sflat, int64_t nF, int d) {
    const int64_t blk = b.layout == 0 ? M * nF + F : F * b.nM + M;
    return (blk << (b.lgseg * d)) + sflat;
}

// Index of the factor block of mode k for (F, M, segment sig) at the factor's level.
template <class R>
TB_DEV int64_t fac_index(const FacRef<R> &f, int k, int64_t F, int64_t M, int sig, int d, int Lc) {
    if (!f.separable) return ((F * f.nM + M) << f.lgseg) + sig;
    const int64_t Fk = (F >> (Lc * (d - 1 - k))) & ((1 << Lc) - 1);
    const int64_t Mk = (M >> (f.l * (d - 1 - k))) & ((1 << f.l) - 1);
    return (((Fk << f.l) + Mk) << f.lgseg) + sig;
}
// Factor block of mode k for (F, M, segment sig) at the factor's level.
template <class R>
TB_DEV const cx<R> *fac_block(const FacRef<R> &f, int k, int64_t F, int64_t M, int sig, int d, int Lc) {
    return f.A[k] + fac_index<R>(f, k, F, M, sig, d, Lc) * (int64_t)f.rows[k] * f.cols[k];
}

template <class R>
struct UserArr {      // user tensor (n_1..n_d, nv) C order
    cx<R> *p;
    int64_t gstride[MAXD];   // element stride (in points) of axis k
};

// One mode product of a level pass applied to every unit (k_mode in tb_mode.cu).
// A unit is a tile (leaf passes) or one child chain of a split / gather group;
// its mode-k intermediate has dims (o_0..o_{k-1}, m_k..m_{d-1}) x nv with the
// RHS innermost.  Columns of a unit: pre = prod_{i<k} o_i times post =
// prod_{i>k} m_i * nv.
enum ModeKind : int { MK_UNIT = 0, MK_PARENTS = 1, MK_USER = 2 };

template <class R>
struct ModeArgs {
    int d, k, Lc, pass;        // pass: 0 LeafIn, 1 Split, 2 Gather, 3 LeafOut
    int m, o, lda, fsz;        // staged factor: m x lda (zero columns a >= o), fsz elements apart
    int trans, conj;           // the factor block is applied as op(A) = A or A^T, conjugated or not
    int64_t pre, post, cols;   // columns of one unit
    int64_t nblk, ncb;         // units (or groups) of the launch, column chunks per unit
    int64_t gsplit;            // thread blocks per unit; each walks every gsplit-th chunk
    int bt;                    // threads per block (32, 64 or 128; at least 2^d for a group launch)
    int sub;                   // slices of bt / sub threads (a multiple of 32) sharing each column slot
    int64_t nv, nF;
    int lvl, lgs;              // factor level and segment bits per mode of the pass's tiles
    int in_tile, out_tile;     // MK_UNIT input / output is the level tile instead of a unit buffer
    int cb[MAXD];
    int64_t nmid[MAXD];
    const int *perm[MAXD];
    int Rp[MAXD];              // parent tile dims (split input, gather output)
    FacRef<R> fac;
    TileBuf<R> lin, lout;      // level tensors read / written by the pass
    UserArr<R> user;
    const cx<R> *tin;          // unit buffers of the previous / this mode
    cx<R> *tout;
    int64_t in_usize, out_usize;
    int64_t f0, f1;            // units whose mid-level multiset F lies outside [f0, f1) are skipped
    size_t smem;
};

template <class R>
cudaError_t launch_mode(int in_kind, int out_kind, int ob, int rank, const ModeArgs<R> &a, cudaStream_t st);
int mode_cols_per_thread();

// A whole level pass (all d mode products) in one persistent launch
// (k_level in tb_level.cu), complex64.  Work item = (unit or group, chunk of
// vc right-hand sides); the intermediates stay in shared memory.
struct LevelArgs {
    int d, Lc, pass, lvl, lgs;     // pass: 0 LeafIn, 1 Split, 2 Gather, 3 LeafOut
    int conj, trans;               // factors applied as op(A) = A or A^T, conjugated or not
    int order[MAXD];               // mode of step i
    int ob[MAXD];                  // output rows per register chunk of step i (even, 4 .. 16)
    int m[MAXD], o[MAXD];          // input / output length of each mode for one unit
    int lda[MAXD];                 // staged factor row length of mode k (o_k padded to its chunks)
    int fac_off[MAXD];             // float offset of mode k's staged factor (3 planes of m_k x lda_k)
    int fac_floats;                // floats of all staged factors
    int vc, lvc, nq;               // RHS per item (a power of two, lvc = log2), chunks per unit
    int lcb[MAXD];                 // log2 C_b per mode (leaf passes)
    int64_t nv, nF, nitems;
    int cb[MAXD];
    int64_t nmid[MAXD];
    const int *perm[MAXD];
    int Rp[MAXD];                  // parent tile dims (Split input, Gather output)
    FacRef<float> fac;
    TileBuf<float> lin, lout;
    UserArr<float> user;
    size_t off_gstr;               // byte offset of the leaf tables of grid offsets (int64)
    size_t off_in, off_s0, off_s1, off_acc;   // byte offsets in shared memory of the staged
                                      // step-0 input, the two intermediate buffers and
                                      // (Gather) the combined parent tile
    size_t smem;
};
cudaError_t launch_level(const LevelArgs &a, int ob, int blocks, cudaStream_t st);
bool level_ob_valid(int ob);
int level_threads();
int level_max_children();

// A level pass as one persistent launch on the tcgen05 tensor cores
// (k_level_tc, split-BF16 mode products, FP32 accumulation; d <= 3).  Step i
// of a chain is the mode product of mode k = st[i].k, a tensor-core product
// D = X B^T with X the step's operand (rows = the entries of the other modes
// times the item's vc RHS, K = the m complex inputs of mode k, each as
// (hi re, hi im, lo re, lo im)) and B1, B2 the split real forms of the op(A)
// block (rows 2 o', 2 o' + 1).
constexpr int LTC_MAXD = 3;
struct LtcStep {
    int k, m, o;                   // mode, input / output length
    int rows, tiles, ks, np;       // operand rows, 128-row tiles, K-steps of 4 complex, MMA N (>= 2 o)
    int nod, om[LTC_MAXD], od[LTC_MAXD];   // the other modes, slowest first, and their current lengths
    int rstr[LTC_MAXD];            // row stride of each mode in this step's operand (0 for mode k)
    int tstr[LTC_MAXD];            // last step: entry stride of each mode in the output tile
    uint32_t a_rs;                 // operand: K-step region stride (tiles x 4 KB)
    uint32_t b_off, b_rs, b_half;  // B1 at b_off in the warpgroup's factor area, B2 b_half later
    uint32_t tcol;                 // accumulator column of tile 0
    uint32_t idesc;
};
struct LevelTcArgs {
    LevelArgs L;                   // pass, dims, item decomposition, tiles, factors, user tensor
    LtcStep st[LTC_MAXD];
    uint32_t a0_off;               // Split: the step-0 operand shared by the block
    uint32_t wg_off[2];            // per warpgroup: operand buffer, then factors, then leaf tables
    uint32_t fac_off, tab_off;     // offsets within a warpgroup's area
    uint32_t smem;
    int *err;                      // device error word (TB_ETIMEOUT)
};
cudaError_t launch_level_tc(const LevelTcArgs &a, int blocks, cudaStream_t st);
int level_tc_threads();

// Regeneration of the mid-level cores K(t-bar, s-bar) from the skeleton points
// inside the one-RHS forward core (k_core_regen), for the kernels whose
// distances or phases are exact integers on uniform grids:
//   HELMHOLTZ on x_k = x0_k + i h, y_k = x0_k + (j + off_k) h (one spacing h and
//     integer offsets): |x - y|^2 + hperp^2 = h^2 D with the integer
//     D = sum_k (i_k - j_k - off_k)^2 + hp2 < 2^24, phase (cycles) = cyc sqrt(D);
//   RADON on x_k = i / n, xi_k = j + xi0_k (integers): x.xi = (sum i_k xi_k) / n,
//     phase = x.xi + c(x) |xi|, c(x) = a + b prod_k sin(2 pi x_k) per target row.
struct CoreRegen {
    int kind;                       // 0: cores are read; TB_KERNEL_HELMHOLTZ or TB_KERNEL_RADON
    int off[MAXD], hp2;             // Helmholtz integer offsets and perpendicular offset^2 (grid units)
    float cyc_hi, cyc_lo;           // kappa h / (2 pi) as a double-float
    float inv_h;
    int n;                          // Radon: target grid denominator
    int xi0[MAXD];                  // Radon: integer source offsets
    double ra, rb;                  // Radon: c(x) = ra + rb prod sin(2 pi x_k)
    const double *xs[MAXD];         // target coordinates (Radon c(x) in FP64)
    const int *tskel[MAXD], *sskel[MAXD];   // level-Lc skeleton grid indices
    int tcap[MAXD], scap[MAXD];
    int64_t nF;
};

template <class R>
struct CoreApplyArgs {
    int d;
    int64_t P, nv, nvc;
    const int *dims;
    const int64_t *off;
    const cx<R> *core;
    TileBuf<R> in, out;    // forward: in = source Lc, out = target Lc
    const cx<R> *kron[MAXD];
    int Rt[MAXD], Rs[MAXD];
    int Lc;
    int offX, offB0, offB1, offY, offA;
    size_t smem;
    CoreRegen rg;
    int64_t pf0, pf1;      // pairs whose input-side mid-level multiset (forward: s, adjoint: t)
                           // lies outside [pf0, pf1) are skipped
};

// Split-BF16 tensor-core core contraction (tb_core_tc.cu).  A work item is one
// tile of up to 128 core rows of one pair; its K-chunks of 32 complex columns
// are stored as consecutive blocks of rows x 256 bytes (hi then lo BF16).
struct CoreItem {
    int pair, tile, rows, nkc;
    int64_t boff;      // byte offset of the item's first block
    int64_t xpos;      // offset of the pair's input-position table (nkc x 32 entries)
    int rout[MAXD];    // compact ranks of the pair on the output side (rows of this operator)
};

struct CoreTileArgs {
    int d, adjoint;
    int64_t nitems;
    const CoreItem *items;
    const int *dims;
    const int64_t *core_off;
    const c128 *c128;
    const c64 *c64;
    unsigned char *out;
};

struct CoreTcArgs {
    int d, adjoint;
    int64_t nitems;
    const CoreItem *items;
    const unsigned char *tiles;
    const int *dims;
    const int *xpos;   // per pair: padded tile position of each compact input index, -1 past the end
    const cx<float> *in;
    cx<float> *out;
    int in_tsize, out_tsize;
    int in_R[MAXD], out_R[MAXD];
    int nv;         // RHS stride of the tiles
    int v0, nvc;    // RHS chunk [v0, v0 + nvc) handled by this launch, nvc <= 16
    int zero_pad;   // 1: write zeros to the padded output entries; 0: they already hold zeros
    int *err;
};

cudaError_t launch_core_tile(const CoreTileArgs &a, cudaStream_t st);
cudaError_t launch_core_tc(const CoreTcArgs &a, cudaStream_t st);
int core_tc_rows_per_item();
int core_tc_cols_per_chunk();

// Separable kernels (a product over modes): every factor depends on one mode,
// so the butterfly is a tensor product of per-mode 1-D butterflies.  Each
// mode's chain (leaf V, transfers W, core K_k, transfers P, leaf U) is stored
// as a list of sparse step matrices (CSR, explicit zeros dropped) acting on
// the 1-D index of that mode.
// One nonzero of a step in row order, for the fiber kernel: its value, its
// column and whether it closes its row (rows without nonzeros carry one zero
// entry, so every row closes exactly once).
template <class R>
struct alignas(16) SepNz {
    cx<R> v;
    int col;
    int last;
};

template <class R>
struct SepStep {
    int n_out, n_in;
    const int *rowptr;   // n_out + 1
    const int *col;
    const cx<R> *val;
    const SepNz<R> *nz;  // the same step as a packed row-ordered stream
    int npk;             // entries of nz
};

template <class R>
struct SepPassArgs {
    int d, k0, k1;            // modes k0..k1 (contiguous) are transformed by this pass
    int n[MAXD];
    int64_t outer;            // prod_{k < k0} n_k
    int64_t inner;            // nv * prod_{k > k1} n_k (contiguous in memory)
    int ic;                   // inner elements per block
    int64_t nchunks;          // ceil(inner / ic)
    const cx<R> *in;
    cx<R> *out;
    const SepStep<R> *steps;  // device array
    int step0[MAXD], nsteps[MAXD];
    int buf;                  // elements of each of the two shared buffers
    size_t smem;
};

template <class R>
cudaError_t launch_sep_pass(const SepPassArgs<R> &a, cudaStream_t st);

// One mode's chain applied fiber by fiber: thread = (fiber, RHS), the fiber
// held in a shared-memory column of that thread.
template <class R>
struct SepFiberArgs {
    int k, nk;
    int64_t outer;            // prod_{j < k} n_j
    int64_t inner;            // nv * prod_{j > k} n_j
    const cx<R> *in;
    cx<R> *out;
    const SepStep<R> *steps;  // this mode's steps, in order
    int nsteps, maxext;
    int npk;                  // packed entries of all the steps
    int threads;
    size_t smem;
};

template <class R>
cudaError_t launch_sep_fiber(const SepFiberArgs<R> &a, cudaStream_t st);

// Register-resident chains.  When every rank of mode k equals its leaf size
// C_b (the bit-reversed uniform Fourier kernel, whose DFT blocks have exact
// rank C_b), every level of the mode's 1-D chain has N = C_b 4^Lc entries, the
// leaf interpolation V and the leaf U^T are permutation matrices (an ID that
// keeps every column), and each remaining step is a fixed pattern of dense
// blocks: W_l and P_l rows read 2 C_b inputs, core rows read C_b inputs.  The
// pattern is a compile-time function of (Lc, C_b), so a thread keeps its whole
// fiber in registers; V and U^T become the load and store positions.
//   step st = 0 .. Lc-1 : W_{st+1}      (source transfers)
//   step st = Lc        : core K_k
//   step st = Lc+1 .. 2Lc: P_{2Lc+1-st} (target transfers)
// Source level-l entry ((s 2^l + tau) 2^(Lc-l) + nu) C_b + a and target
// level-l entry ((t 2^l + nu) 2^(Lc-l) + tau) C_b + a, as in the CSR steps.
TB_HD constexpr int sepr_width(int lc, int rk, int st) { return st == lc ? rk : 2 * rk; }
// input column j of output row e of forward step st
TB_HD constexpr int sepr_col(int lc, int rk, int st, int e, int j) {
    const int a = e % rk, r1 = e / rk;
    if (st < lc) {   // W_l, l = st + 1: children 2 nu, 2 nu + 1 of source level l - 1, contiguous
        const int l = st + 1;
        const int nu = r1 & ((1 << (lc - l)) - 1), r2 = r1 >> (lc - l);
        const int tau = r2 & ((1 << l) - 1), s = r2 >> l;
        (void)a;
        return ((((s << (l - 1)) + (tau >> 1)) << (lc - l + 1)) + 2 * nu) * rk + j;
    }
    if (st == lc) {  // core: output (t nb + s) C_b + a reads source mid-level entry (s nb + t) C_b + q
        const int nb = 1 << lc, t = r1 / nb, s = r1 % nb;
        return (s * nb + t) * rk + j;
    }
    // P_l, l = 2 Lc + 1 - st: output target level l - 1, inputs nu = 2 pn + c at level l
    const int l = 2 * lc + 1 - st;
    const int tp = r1 & ((1 << (lc - l + 1)) - 1), r2 = r1 >> (lc - l + 1);
    const int pn = r2 & ((1 << (l - 1)) - 1), t = r2 >> (l - 1);
    const int c = j / rk, q = j % rk;
    return ((((t << l) + 2 * pn + c) << (lc - l)) + (tp >> 1)) * rk + q;
}
// offset of forward step st in the dense coefficient array (rows in order,
// sepr_width entries per row, in the order of sepr_col's j)
TB_HD constexpr int sepr_off(int lc, int rk, int st) {
    const int n = rk << (2 * lc);
    int o = 0;
    for (int i = 0; i < st; ++i) o += n * sepr_width(lc, rk, i);
    return o;
}
TB_HD constexpr int sepr_ncoef(int lc, int rk) { return sepr_off(lc, rk, 2 * lc + 1); }
constexpr int SEPR_MAXN = 32;   // longest fiber kept in registers

template <class R>
struct SepRegArgs {
    int lc, rk;                  // selects the instantiation
    int64_t outer, inner;        // fiber (o, q): entry p at (o N + p) inner + q
    const cx<R> *in;
    cx<R> *out;
    const cx<R> *coef;           // sepr_ncoef entries
    // complex64 paired-FMA form: per coefficient (re, re, im, im) for the
    // forward apply, (re, re, im, -im) for the adjoint (the host passes the
    // direction's array)
    const float4 *cf4;
    // element offsets (grid position x inner) of level-0 entry p within a fiber:
    // ldo for the source side (V and tree order), sto for the target side (U^T
    // and tree order); N inner < 2^31
    int ldo[SEPR_MAXN];
    int sto[SEPR_MAXN];
    int blocks;                  // grid size (0 = one thread per fiber)
};

// variant (complex64): 0 = paired FP32 FMAs, two fibers per thread;
// 1 = scalar FMAs, one fiber per thread with the next fiber's loads in flight.
// Complex128 has the scalar form only.
template <class R>
cudaError_t launch_sep_reg(bool adjoint, int variant, const SepRegArgs<R> &a, cudaStream_t st);

// Two consecutive exact-rank modes ka = kb - 1 and kb with the same N, fused
// in one pass: a block takes a tile (o, all i_ka, all i_kb, q chunk of Q),
// applies mode kb to its fibers with the result written to shared memory in
// grid order, then mode ka to the tile's other fibers.  Element
// (o, i_ka, i_kb, q) sits at ((o N + i_ka) N + i_kb) inner + q.
template <class R>
struct SepReg2Args {
    int lc, rk;
    int q, lq;                   // tile width Q = 2^lq along the inner index; blockDim = N Q
    int64_t outer, inner, nchunks;
    const cx<R> *in;
    cx<R> *out;
    const cx<R> *coef_a, *coef_b;
    const float4 *cf4_a, *cf4_b;   // complex64 paired-FMA coefficients (see SepRegArgs)
    int ld_a[SEPR_MAXN], st_a[SEPR_MAXN];   // grid positions of mode ka's level-0 entries
    int ld_b[SEPR_MAXN], st_b[SEPR_MAXN];   // and of mode kb's
};

template <class R>
cudaError_t launch_sep_reg2(bool adjoint, const SepReg2Args<R> &a, cudaStream_t st);
template <class R>
bool sep_reg_supported(int lc, int rk);

// Least-squares solver (tb_cgls, tb_cgls.cu): per-column scalars of the CGLS
// iteration, kept in device memory.
struct CglsScalars {
    double gamma, delta, alpha, beta;
};
enum CglsMode : int { CG_GAMMA0 = 0, CG_ALPHA = 1, CG_BETA = 2, CG_RESID = 3 };
int cgls_blocks();   // rows of the partial-sum arrays (blocks of the vector kernels)
int cgls_max_nv();
template <class R>
cudaError_t launch_cgls_sqnorm(const cx<R> *a, int64_t rows, int nv, double *partial, cudaStream_t st);
template <class R>
cudaError_t launch_cgls_xr(cx<R> *x, cx<R> *r, const cx<R> *p, const cx<R> *q, const CglsScalars *sc, int64_t rows,
                           int nv, double *partial, cudaStream_t st);
template <class R>
cudaError_t launch_cgls_sub(cx<R> *r, const cx<R> *b, const cx<R> *q, int64_t rows, int nv, double *partial,
                            cudaStream_t st);
template <class R>
cudaError_t launch_cgls_p(cx<R> *p, const cx<R> *s, const CglsScalars *sc, int64_t rows, int nv, cudaStream_t st);
cudaError_t launch_cgls_finalize(const double *partial, int nv, int mode, CglsScalars *sc, double *hist, int *count,
                                 int cap, cudaStream_t st);

enum class Pass { LeafIn, Split, Gather, LeafOut };

template <class R>
cudaError_t launch_core_dense(bool adjoint, const CoreApplyArgs<R> &a, cudaStream_t st);
template <class R>
cudaError_t launch_core_kron(bool adjoint, const CoreApplyArgs<R> &a, cudaStream_t st);
// Forward core for one RHS, complex64, 16 rows per warp (k_core_rows); the
// same with the core entries regenerated from the skeleton points (k_core_regen).
template <class R>
cudaError_t launch_core_rows(const CoreApplyArgs<R> &a, cudaStream_t st);
cudaError_t launch_core_regen(const CoreApplyArgs<float> &a, cudaStream_t st);

// Shared-memory plan of a mode-product chain: input dims m, output dims o.
struct ChainSmem {
    int64_t x, b0, b1, y, a;   // element counts
};
ChainSmem chain_smem(int d, const int *m, const int *o, int64_t nvc);
cudaError_t set_smem_once(const void *fn, size_t smem);

}  // namespace tb

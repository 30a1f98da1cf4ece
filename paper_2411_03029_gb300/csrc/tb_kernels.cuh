// Argument blocks and launchers of the construction and apply kernels.
#pragma once

#include "tb_common.cuh"

namespace tb {

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
    int rows[MAXD], cols[MAXD];
    int l, lgseg;
    int64_t nM;
    int separable;
};

template <class R>
struct UserArr {      // user tensor (n_1..n_d, nv) C order
    cx<R> *p;
    int64_t gstride[MAXD];   // element stride (in points) of axis k
};

template <class R>
struct LevelArgs {
    int d, Lc;
    int64_t nF;           // mid-level multisets per side, 2^(d Lc)
    int64_t nv, nvc;      // RHS total and per-block chunk
    int64_t nblocks;
    int cb[MAXD];
    int64_t nmid[MAXD];   // n_k >> Lc
    const int *perm[MAXD];
    TileBuf<R> in, out;
    FacRef<R> fac;
    UserArr<R> user;
    // smem layout (elements of cx<R>)
    int offX, offB0, offB1, offY, offA;
    size_t smem;
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
};

// Split-BF16 tensor-core core contraction (tb_core_tc.cu).  A work item is one
// tile of up to 128 core rows of one pair; its K-chunks of 32 complex columns
// are stored as consecutive blocks of rows x 256 bytes (hi then lo BF16).
struct CoreItem {
    int pair, tile, rows, nkc;
    int64_t boff;   // byte offset of the item's first block
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
    const cx<float> *in;
    cx<float> *out;
    int in_tsize, out_tsize;
    int in_R[MAXD], out_R[MAXD];
    int nv;         // RHS stride of the tiles
    int v0, nvc;    // RHS chunk [v0, v0 + nvc) handled by this launch, nvc <= 16
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
template <class R>
struct SepStep {
    int n_out, n_in;
    const int *rowptr;   // n_out + 1
    const int *col;
    const cx<R> *val;
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
    int nnz, nidx;            // total nonzeros / row-pointer entries of the steps
    int threads;
    size_t smem;
};

template <class R>
cudaError_t launch_sep_fiber(const SepFiberArgs<R> &a, cudaStream_t st);

enum class Pass { LeafIn, Split, Gather, LeafOut };

template <class R>
cudaError_t launch_level(Pass pass, bool conj, const LevelArgs<R> &a, cudaStream_t st);
template <class R>
cudaError_t launch_core_dense(bool adjoint, const CoreApplyArgs<R> &a, cudaStream_t st);
template <class R>
cudaError_t launch_core_kron(bool adjoint, const CoreApplyArgs<R> &a, cudaStream_t st);

// Shared-memory plan of a mode-product chain: input dims m, output dims o.
struct ChainSmem {
    int64_t x, b0, b1, y, a;   // element counts
};
ChainSmem chain_smem(int d, const int *m, const int *o, int64_t nvc);
cudaError_t set_smem_once(const void *fn, size_t smem);

}  // namespace tb

// Host-side plan of a built tensor butterfly and the device-side views that the
// construction and apply kernels receive by value.
#pragma once

#include <string>
#include <vector>

#include "tb_common.cuh"
#include "tb_kernels.cuh"

namespace tb {

// Interpolation / transfer factors of one side at one level (Alg. 1 output):
// for each mode k, `count[k]` blocks of R[k] x cin[k] entries, row-major.
// Rows are the skeleton entries of the block in pivot order (zero rows pad up
// to R[k]); columns are the candidate entries: the C_b leaf points at level 0,
// or the two child skeletons (child 1 in [0, R_{l-1,k}), child 2 in
// [R_{l-1,k}, 2 R_{l-1,k})) at level l > 0, zero-padded.
struct SideLevel {
    int R[MAXD] = {0};
    int cin[MAXD] = {0};
    int cap[MAXD] = {0};       // skeleton slots per block during construction
    int64_t count[MAXD] = {0};
    c128 *fac64[MAXD] = {nullptr};
    c64 *fac32[MAXD] = {nullptr};
    int *skel[MAXD] = {nullptr};   // count x cap grid indices (-1 = none)
    int *rank[MAXD] = {nullptr};   // count
    int rmin = 0, rmax = 0;
};

struct Workspace {
    void *buf[2] = {nullptr, nullptr};
    size_t bytes = 0;          // per buffer
    void *mbuf[2] = {nullptr, nullptr};   // mode intermediates of the level passes
    size_t mbytes[2] = {0, 0};
    // output of the split-BF16 core per direction ([0] forward: target side,
    // [1] adjoint: source side), laid out for cout_nv RHS; its padded entries
    // hold zeros (set at allocation and when nv changes; the core writes only
    // the compact entries)
    void *cout[2] = {nullptr, nullptr};
    size_t cout_bytes[2] = {0, 0};
    int64_t cout_nv[2] = {0, 0};
    void *host_in = nullptr;   // device staging for tb_apply_host
    void *host_out = nullptr;
    size_t host_bytes = 0;
};

// Streams, events and device buffers of the pipelined host-data apply
// (tb_apply_host_batch): [0] host-to-device, [1] apply, [2] device-to-host.
struct HostPipe {
    cudaStream_t s[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t in_ready[2] = {nullptr, nullptr}, in_free[2] = {nullptr, nullptr};
    cudaEvent_t out_ready[2] = {nullptr, nullptr}, out_free[2] = {nullptr, nullptr};
    void *din[2] = {nullptr, nullptr};
    void *dout[2] = {nullptr, nullptr};
    size_t bytes = 0;
};

struct ProfRec {
    const char *name;
    int level, adjoint;
    cudaEvent_t e0, e1;
    int64_t bytes;
    double flops;
    int kernels = 1;   // kernel launches between the two events
};

// Launch shape of one fused level pass picked by tb_autotune (0 = the
// built-in rule).
struct LevelTune {
    int mode = 0;    // 1 = the per-mode launches won the tuning, 2 = the fused launch,
                     // 3 = the tensor-core launch (split-BF16 applies)
    int vc = 0;      // right-hand sides per work item
    int cps = 0;     // resident thread blocks per SM the grid is sized for
    int obmax = 0;   // largest register chunk of output rows (4 .. 16)
    int tc_vc = 0;   // right-hand sides per work item of the tensor-core launch
};

// Launch shape of one mode-product launch picked by tb_autotune (0 = the
// built-in rule).
struct ModeTune {
    int ob = 0;      // output rows per register tile
    int waves = 0;   // thread blocks per SM the grid is sized for
    int rank = -1;   // rank-bounded products (1) or not (0); -1: the built-in rule
    int bt = 0;      // threads per column slice (32, 64, 128); 0: the built-in rule
    int sub = 0;     // column slices sharing each column (1, 2, 4); 0: one
};

struct GraphEntry {
    const void *in;
    void *out;
    int64_t nv;
    int prec;
    int adjoint;
    cudaStream_t stream;
    cudaGraphExec_t exec;
};

}  // namespace tb

struct tb_plan {
    int d = 0, L = 0, Lc = 0, order = 0, separable = 0, device = 0;
    int64_t n[TB_MAX_D] = {0}, cb[TB_MAX_D] = {0};
    double tol = 0;
    unsigned precisions = 0;
    int use_graphs = 0;
    tb::KernelSpec ks{};
    int proxy_rows = 1024, rank_max = 32;
    uint64_t seed = 0;

    // grids and per-axis tree orderings (tree position -> grid index), device
    double *xs[TB_MAX_D] = {nullptr}, *ys[TB_MAX_D] = {nullptr};
    int *perm[TB_MAX_D] = {nullptr};

    tb::SideLevel src[TB_MAX_LEVELS], tgt[TB_MAX_LEVELS];

    // mid-level cores K(t-bar, s-bar): P pairs, compact storage
    int64_t P = 0;
    int64_t *core_off = nullptr;   // P + 1 offsets into the core arrays (device)
    int *core_dims = nullptr;      // P x 2d: target ranks then source ranks (device)
    tb::c128 *core64 = nullptr;
    tb::c64 *core32 = nullptr;
    // split-BF16 tiles of the core for the tensor-core contraction: [0] forward
    // K(t-bar, s-bar), [1] adjoint K(t-bar, s-bar)^H (see tb_core_tc.cu)
    unsigned char *tc_tiles[2] = {nullptr, nullptr};
    tb::CoreItem *tc_items[2] = {nullptr, nullptr};
    int *tc_xpos[2] = {nullptr, nullptr};   // input-position tables of the tensor-core contraction
    int64_t tc_nitems[2] = {0, 0};
    int64_t tc_bytes[2] = {0, 0};
    int64_t core_entries = 0;
    int64_t core_in_entries = 0;   // sum over pairs of prod_k |s-bar_k| (compact core columns)
    int64_t core_out_entries = 0;  // sum over pairs of prod_k |t-bar_k|
    int profiling = 0;
    std::vector<tb::ProfRec> prof;
    // separable (Kronecker) cores: per mode k, (2^Lc x 2^Lc) blocks of Rt x Rs
    tb::c128 *kron64[TB_MAX_D] = {nullptr};
    tb::c64 *kron32[TB_MAX_D] = {nullptr};

    // separable chains: per direction (0 forward, 1 adjoint) the step
    // descriptors of every mode, FP64 and FP32 values
    tb::SepStep<double> *sep64[2] = {nullptr, nullptr};
    tb::SepStep<float> *sep32[2] = {nullptr, nullptr};
    int sep_step0[2][TB_MAX_D] = {{0}}, sep_nsteps[2][TB_MAX_D] = {{0}};
    int sep_maxext[TB_MAX_D] = {0};   // largest 1-D index along a mode's chain
    int64_t sep_nnz[2][TB_MAX_D] = {{0}};
    int64_t sep_nidx[2][TB_MAX_D] = {{0}};   // row-pointer entries of a mode's steps
    int64_t sep_npk[2][TB_MAX_D] = {{0}};    // packed nonzero-stream entries of a mode's steps
    // register-resident chains (see sepr_col): per mode, whether the chain has
    // the exact-rank form, its rank, dense step coefficients and the grid
    // positions of the level-0 source / target entries
    int sepr_ok[TB_MAX_D] = {0};
    int sepr_rk[TB_MAX_D] = {0};
    tb::c128 *sepr_coef64[TB_MAX_D] = {nullptr};
    tb::c64 *sepr_coef32[TB_MAX_D] = {nullptr};
    float4 *sepr_cf4[2][TB_MAX_D] = {{nullptr}};   // paired-FMA form: [0] forward, [1] adjoint
    int sepr_ld[TB_MAX_D][tb::SEPR_MAXN] = {{0}};
    int sepr_st[TB_MAX_D][tb::SEPR_MAXN] = {{0}};

    // launch shapes chosen by tb_autotune: [complex64 / complex128][side][pass][level][mode]
    tb::ModeTune tune[2][2][4][TB_MAX_LEVELS][TB_MAX_D];
    tb::LevelTune ltune[2][4][TB_MAX_LEVELS];   // fused level passes: [side][pass][level]
    int level_choice = 0;          // tb_options.level_schedule
    int core_rows = 1;             // forward complex64 core with one RHS: row batches per warp (k_core_rows)
    int core_mode = 0;             // tb_options.core_mode
    int mode_slices = 0;           // tb_options.mode_slices
    int core_regen_tuned = 0;      // tb_autotune found the regenerated core faster
    tb::CoreRegen rg{};            // regeneration parameters (rg.kind = 0: not possible)
    int sep_choice = 0;            // separable apply: tb_options.sep_schedule
    int autotune = 0;              // tune at the first apply of each (nv, precision)
    std::vector<std::pair<int64_t, int>> tuned;   // (nv, precision) pairs tuned so far
    int64_t level_max = 0;         // largest level tensor, entries per RHS
    int64_t mode_max[2] = {0, 0};  // largest even / odd mode intermediate, entries per RHS
    tb::Workspace ws;
    tb::HostPipe pipe;
    std::vector<tb::GraphEntry> graphs;
    std::vector<void *> allocations;
    int64_t device_bytes = 0;
    int64_t num_ids = 0;
    int rank_min = 0, rank_max_seen = 0;
    double build_seconds = 0;
    int *d_err = nullptr;          // device error word of the construction kernels
};

/*
 * tb.h -- C ABI of the GB300 tensor butterfly library.
 *
 * The library compresses a d-dimensional oscillatory integral operator
 *     u(x^i) = sum_j K(x^i, y^j) f(y^j)
 * discretized on tensor grids (a 2d-mode kernel tensor with n^{2d} entries, never
 * formed) into a tensor butterfly, then applies it in O(n^d) work per right-hand
 * side.  Reference: Kielstra, Shi, Luo, Qian, Liu, "A Linear-complexity Tensor
 * Butterfly Algorithm for Compressing High-dimensional Oscillatory Integral
 * Operators" (arXiv 2411.03029):
 *   - construction: Alg. 1 (Sec. 3.2), built on the Tucker-type ID of Sec. 3.1;
 *   - contraction (apply): Alg. 2 (Sec. 3.2), G = K x_{d+1..2d} F;
 *   - adjoint: the conjugate transpose of the factorization of Eq. (butterfly_tensor).
 *
 * Conventions shared by every entry point
 *   - Every call returns a tb_status and never aborts or exits.  On failure,
 *     tb_last_error() returns a message for the calling thread.
 *   - Complex arrays are interleaved (re, im) pairs: complex128 for
 *     TB_PREC_C128, complex64 for TB_PREC_C64 and TB_PREC_C64_SPLITBF16.
 *   - Data layout of the input F and output G: C order over (n_1, ..., n_d, nv),
 *     i.e. the right-hand-side index is innermost and axis 1 is slowest.  This
 *     is the paper's F in C^{n_1 x ... x n_d x n_v} (Alg. 2 input) read in C order.
 *   - Grid point i = (i_1..i_d) has coordinates (x_1[i_1], ..., x_d[i_d]).
 *   - Ownership: a handle owns all device memory it allocates (factors, cores,
 *     workspaces, CUDA graphs).  The caller owns f / u / g / v.
 *   - Threading: a handle may be used from one host thread at a time.
 *     Distinct handles are independent.
 */
#ifndef TB_H
#define TB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TB_MAX_D 6       /* largest supported dimension d */
#define TB_MAX_LEVELS 16 /* largest supported tree depth L */

typedef enum {
    TB_OK = 0,
    TB_EINVAL = 1,        /* invalid argument (sizes, pointers, aliasing, grid) */
    TB_ENOMEM = 2,        /* device or host allocation failed */
    TB_ECUDA = 3,         /* a CUDA runtime call failed */
    TB_ERANK = 4,         /* an ID needed more than the rank cap */
    TB_ETIMEOUT = 5,      /* a bounded device wait expired */
    TB_EUNSUPPORTED = 6   /* the request is valid but not built (precision, size) */
} tb_status;

/* Kernel families of the paper's numerical examples (Sec. 4). */
typedef enum {
    TB_KERNEL_FOURIER = 1,   /* K = exp(-2 pi i x.y)                        (Sec. 4.3); any
                                per-axis grids, e.g. random targets for the type-2
                                non-uniform DFT of Sec. 4.3 */
    TB_KERNEL_HELMHOLTZ = 2, /* K = exp(i kappa rho)/rho, rho = sqrt(|x-y|^2 + h^2),
                                params[0] = kappa, params[1] = h >= 0: the offset of the
                                source grid along an axis outside the d grid axes
                                (h = 0: the cubes of Sec. 4.1; d = 2, h = 1: the
                                parallel plates of Sec. 4.1) */
    TB_KERNEL_RADON = 3,     /* K = exp(2 pi i (x.xi + c(x)|xi|)),
                                c(x) = params[0] + params[1] prod_k sin(2 pi x_k) (Sec. 4.2;
                                (3/100, 1/100) with d = 3 is Eq. randon3d) */
    TB_KERNEL_RADON_ANISO = 4 /* d = 2 only: K = exp(2 pi i (x.xi + sqrt(c1^2 xi_1^2 + c2^2 xi_2^2))),
                                c1 = params[0] + params[1] sin(2 pi x_1) sin(2 pi x_2),
                                c2 = params[2] + params[3] cos(2 pi x_1) cos(2 pi x_2)
                                (Sec. 4.2, Eq. randon2d: (2, 1, 2, 1) / 16) */
} tb_kernel_kind;

typedef enum {
    TB_PREC_C128 = 0,          /* complex128 data, FP64 arithmetic ("plain FP64") */
    TB_PREC_C64 = 1,           /* complex64 data, FP32 arithmetic */
    TB_PREC_C64_SPLITBF16 = 2  /* complex64 data; the contractions on the tcgen05 tensor
                                  cores in two-term split BF16 (hi = rn(v), lo = rn(v - hi))
                                  with FP32 accumulation: the mid-level cores and, where
                                  the level passes run on the tensor cores
                                  (tb_options.level_schedule), the mode products */
} tb_precision;

typedef enum {
    TB_ORDER_AUTO = -1,    /* bit-reversed for FOURIER, natural otherwise */
    TB_ORDER_NATURAL = 0,  /* tree nodes are contiguous index ranges (Sec. 3.2) */
    TB_ORDER_BITREV = 1    /* bit-reversal ordering of each axis (Sec. 4.3) */
} tb_order;

typedef struct {
    int kind;          /* tb_kernel_kind */
    double params[4];  /* see tb_kernel_kind; unused entries ignored */
} tb_kernel;

/* Host pointers to per-axis coordinates: x[k] has n[k] target coordinates and
   y[k] has n[k] source coordinates (the paper's m_k = n_k, Sec. 3.2).  Copied
   during tb_build; the caller keeps ownership. */
typedef struct {
    const double *x[TB_MAX_D];
    const double *y[TB_MAX_D];
} tb_grids;

typedef struct {
    int L;                 /* tree levels per axis: even, n_k = C_b,k 2^L; -1 = planner's choice */
    int order;             /* tb_order */
    int proxy_rows;        /* row cap of each proxy matrix (power of two); 0 = 1024 */
    int rank_max;          /* rank cap of each ID (<= 32); 0 = 32; exceeded -> TB_ERANK */
    unsigned precisions;   /* bit mask of (1 << tb_precision) to prepare; 0 = all */
    int separable;         /* -1 = by kernel (FOURIER), 0 = off, 1 = on */
    int use_graphs;        /* 1 = replay each (f, u, nv, precision) apply as a CUDA graph */
    int device;            /* CUDA device ordinal; -1 = the current device */
    uint64_t seed;         /* seed of the proxy-row design (Sec. 2.1 proxy strategy) */
    int autotune;          /* 1 = run tb_autotune before the first apply of each (nv, precision) */
    int sep_schedule;      /* separable handles (tb_autotune may replace it):
                              0 = built-in rule (= 3),
                              1 = per-mode passes, each thread's fiber in shared memory,
                              2 = multi-mode tile passes in shared memory,
                              3 = per-mode passes with the fibers in registers for every
                                  mode whose ranks equal its leaf size (exact-rank chains,
                                  e.g. the bit-reversed Fourier kernel), 1 for the others;
                                  complex64 uses paired FP32 FMAs, two fibers per thread,
                              4 = as 3, with consecutive exact-rank modes fused in pairs
                                  through a shared-memory tile (half the HBM passes),
                              5 = as 3 with scalar FMAs, one fiber per thread and the
                                  next fiber's loads in flight,
                              6 = as 3 with one fiber per thread (4 resident blocks per SM) */
    int level_schedule;    /* non-separable level passes (Alg. 2 steps 1 and 3), complex64 data:
                              0 = built-in rule: 1; tb_autotune may pick another form per pass
                                  (3 only for split-BF16 applies),
                              1 = d launches per pass, one per mode product (FP32 FMAs),
                              2 = one fused persistent launch per pass on the CUDA cores (the
                                  mode products of a unit back to back, intermediates in
                                  shared memory),
                              3 = one persistent launch per pass on the tcgen05 tensor cores:
                                  each mode product in two-term split BF16 with FP32
                                  accumulation (split-BF16 applies; the others use 1);
                              complex128 always uses 1 */
    int core_mode;         /* the forward complex64 mid-level core with one RHS (Alg. 2 step 2):
                              0 = built-in rule (stored cores; tb_autotune may pick 2),
                              1 = read the stored cores K(t-bar, s-bar),
                              2 = evaluate K(t-bar, s-bar) at the skeleton points inside
                                  the contraction (Helmholtz and Radon kernels on uniform
                                  grids, where |x - y|^2 and x.xi are exact integers in
                                  grid units; else 1).  The cores stay stored: the adjoint
                                  and several-RHS contractions read them */
    int mode_slices;       /* complex64 per-mode level launches: groups of threads that share
                              each output column (each takes every n-th child / row chunk of
                              it), for units with few columns; 0 = built-in rule (1;
                              tb_autotune may pick 2 or 4 per launch), 1, 2 or 4 = that many
                              for every launch (at most 128 threads per block; complex128
                              always uses 1).  Results do not depend on it. */
} tb_options;

typedef struct tb_plan *tb_handle;

typedef struct {
    int d;
    int L;                         /* levels per tree */
    int Lc;                        /* middle level L/2 */
    int order;                     /* tb_order used */
    int separable;                 /* 1 if per-mode (Kronecker) factors are used */
    int64_t n[TB_MAX_D];           /* points per axis */
    int64_t cb[TB_MAX_D];          /* leaf size per axis (C_b) */
    int rank_src[TB_MAX_LEVELS][TB_MAX_D]; /* padded rank R_{l,k} of V/W, l = 0..Lc */
    int rank_tgt[TB_MAX_LEVELS][TB_MAX_D]; /* padded rank of U/P, l = 0..Lc */
    int rank_min;                  /* smallest rank over all IDs (Tables 2/3 r_min) */
    int rank_max;                  /* largest rank over all IDs (Tables 2/3 r) */
    int64_t num_ids;               /* IDs computed during construction */
    int64_t core_entries;          /* entries of all mid-level cores K(t-bar, s-bar) */
    int64_t factor_entries;        /* entries of all V, W, U, P blocks (padded) */
    int64_t level_entries_max;     /* largest intermediate (per RHS, padded) */
    int64_t device_bytes;          /* device memory held by the handle */
    double build_seconds;          /* wall time of tb_build */
    int64_t mid_src_entries;       /* entries of the source-side mid-level tensor F_{t,s} per RHS
                                      (compact: prod_k |s-bar_k| summed over the pairs) */
    int64_t mid_tgt_entries;       /* entries of the target-side mid-level tensor G_{t,s} per RHS */
} tb_info;

/* Fill *opt with the defaults described in tb_options. */
tb_status tb_options_default(tb_options *opt);

/*
 * Construct the tensor butterfly of K on the given grids (Alg. 1, Sec. 3.2).
 *   kernel  kernel family and parameters (host pointer, read during the call)
 *   d       dimension, 1 <= d <= TB_MAX_D (the paper's d > 1; d = 1 is the
 *           matrix butterfly, Sec. 3.2)
 *   n       n[k] points per axis on each side; n[k] = C_b,k 2^L, power of two
 *   grids   host coordinate arrays (copied)
 *   tol     relative ID tolerance epsilon of Sec. 2.1, 0 < tol < 1
 *   out     receives the handle (NULL on failure)
 * Factors are computed on the current CUDA device in FP64 (kernel phases,
 * column-pivoted QR, triangular solves) and stored in the precisions requested.
 * Errors: TB_EINVAL for bad sizes/pointers, coincident Helmholtz points, a
 * negative Helmholtz offset h or an anisotropic Radon kernel with d != 2,
 * TB_ERANK if an ID needs more than the rank cap, TB_ENOMEM, TB_ECUDA.
 */
tb_status tb_build(const tb_kernel *kernel, int d, const int64_t *n,
                   const tb_grids *grids, double tol, tb_handle *out);

/* tb_build with explicit options (NULL = defaults). */
tb_status tb_build_ex(const tb_kernel *kernel, int d, const int64_t *n,
                      const tb_grids *grids, double tol, const tb_options *opt,
                      tb_handle *out);

/*
 * u = K f (Alg. 2): device pointers f (input, prod n x nv) and u (output),
 * element type per `precision`, layout C order (n_1..n_d, nv).  Stream-ordered
 * on `cuda_stream` (a cudaStream_t; NULL = legacy default stream); returns
 * after the launches are enqueued.  f and u must not overlap (TB_EINVAL).
 * TB_EUNSUPPORTED if the handle was built without `precision`.
 */
tb_status tb_apply(tb_handle h, const void *f, void *u, int64_t nv, int precision,
                   void *cuda_stream);

/*
 * v = K^H g: the adjoint apply (conjugate transpose of Eq. butterfly_tensor,
 * factors traversed in reverse).  Same conventions as tb_apply; g has the
 * target-grid shape, v the source-grid shape.
 */
tb_status tb_apply_adjoint(tb_handle h, const void *g, void *v, int64_t nv, int precision,
                           void *cuda_stream);

/*
 * u = K f with HOST buffers: copies f to the device, applies, and copies u back
 * before returning (synchronous).  f and u are host pointers of the tb_apply
 * layout; pinned memory gives the best transfer rate.  Device staging buffers
 * are owned by the handle.
 */
tb_status tb_apply_host(tb_handle h, const void *f, void *u, int64_t nv, int precision);

/*
 * u_i = K f_i for count inputs with HOST buffers, pipelined: the copy of input
 * i + 1 to the device and the copy of result i - 1 to the host run while input
 * i is applied, on three streams owned by the handle (host-to-device, apply,
 * device-to-host) with two device buffer pairs.  Every input is copied in and
 * every result copied out inside the call; it returns when all results are in
 * host memory (synchronous).  f[i] and u[i] are host pointers of the tb_apply
 * layout, all of the same nv; the copies overlap only when they are pinned
 * (page-locked) memory.  The paper has no counterpart: this is the library's
 * host-data path.
 * Errors: TB_EINVAL for NULL arrays or pointers, count < 1 or nv < 1; as
 * tb_apply otherwise (on an error the streams are synchronized before return).
 */
tb_status tb_apply_host_batch(tb_handle h, const void *const *f, void *const *u, int64_t count, int64_t nv,
                              int precision);

/*
 * u = K f without allocating any device memory.  (The paper has no
 * counterpart: this is an interface of this library.)
 *
 * Same arguments, layout, result and stream ordering as tb_apply, but the
 * level intermediates live in one fixed scratch area compiled into the
 * library, instead of buffers the handle allocates on its first apply or when
 * nv grows.  It is meant for callers that cannot call cudaMalloc while they
 * apply the operator: processes whose device memory is owned by another
 * allocator (a framework's caching allocator, a fixed arena, a hard memory
 * cap), and latency-critical loops that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree imply.  The handle itself is
 * still built (and its factors allocated) by tb_build beforehand.
 *
 *   - Scratch: TB_NOALLOC_SCRATCH_BYTES per device, held by every GPU that
 *     loads the library until the process exits.  A request needing more
 *     (two level tensors of the handle's largest size x nv x element size)
 *     fails with TB_EUNSUPPORTED.
 *   - The first call on a device looks up the scratch address on the host
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call shares the one scratch area, and it keeps the last call's
 *     contents.  Nothing in it has to start at zero: each pass writes every
 *     entry that a later pass of the same call reads (the tests check this by
 *     calling first with an all-NaN input, then with clean ones).  Calls that overlap on the GPU (on different
 *     streams, or from several host threads) race on it and corrupt each
 *     other's results: serialise them.
 *   - No CUDA-graph replay and no per-pass profiling on this path.
 * Errors: as tb_apply, plus TB_EUNSUPPORTED for requests beyond the scratch.
 */
#define TB_NOALLOC_SCRATCH_BYTES (64ull << 20)
tb_status tb_apply_noalloc(tb_handle h, const void *f, void *u, int64_t nv, int precision,
                           void *cuda_stream);

/*
 * Least-squares solve on the device: for each right-hand-side column,
 * min_x ||K x - b||_2 by CGLS (conjugate gradients on the normal equations
 * K^H K x = K^H b), with the forward (tb_apply) and adjoint (tb_apply_adjoint)
 * butterflies as the operator.  This is the inversion of Radon-type data that
 * the paper motivates its generalized Radon kernels with (Sec. 4.2); the
 * paper itself gives no solver.
 *   b       device pointer, target-grid tensor (m_1..m_d, nv), apply layout
 *   x       device pointer, source-grid tensor (n_1..n_d, nv): the starting
 *           point on entry (zero it for x0 = 0), the iterate after `iters`
 *           iterations on return
 *   iters   CGLS iterations (>= 0)
 *   use_graph  1 = capture one iteration (two applies, the vector updates and
 *           the norms) as a CUDA graph once and replay it `iters` times; every
 *           scalar of the iteration stays in device memory, so no iteration
 *           waits on the host.  Needs a stream other than the legacy default
 *           stream (NULL runs eagerly)
 *   resid   NULL or host array of (iters + 1) x nv doubles: ||b - K x_k||_2 of
 *           each column after k iterations (row k), row 0 the start
 * Synchronous: returns when x and resid are final.  Allocates four N x nv
 * work tensors and small scalar arrays for the call and frees them on return;
 * the applies use the handle's workspaces (as tb_apply).  Columns whose
 * residual or search direction becomes exactly zero stop moving (alpha = 0,
 * beta = 0).  Reductions are deterministic (fixed summation order).
 * Errors: TB_EINVAL (NULL or overlapping b / x, nv < 1, iters < 0, called
 * inside a stream capture), TB_EUNSUPPORTED (precision not built, nv > 1024),
 * TB_ENOMEM, TB_ECUDA.
 */
tb_status tb_cgls(tb_handle h, const void *b, void *x, int64_t nv, int iters, int precision, int use_graph,
                  double *resid, void *cuda_stream);

/*
 * Partitioned apply, for running one operator over several devices (one
 * handle per device, each built with the same arguments).  Steps 1 and 3 of
 * Alg. 2 are independent per mid-level source multi-set s and per mid-level
 * target multi-set t (Sec. 3.2); the only coupling is the mid-level tensor of
 * the (t, s) pairs, so rank g takes a range S_g of the s and a range T_g of the
 * t, and one exchange of mid-level tiles connects the halves:
 *   tb_apply_src_part  steps 1 and 2 for s in [s_begin, s_end): reads the source
 *                      points of those s from f (the tb_apply layout), writes the
 *                      tiles G_{t,s} of every t and those s into g_mid;
 *   exchange           tile (t, s) goes from the owner of s to the owner of t;
 *   tb_apply_tgt_part  step 3 for t in [t_begin, t_end): reads the tiles (t, s)
 *                      of those t and every s from g_mid, writes the target points
 *                      of those t into u (other entries of u are left as they are).
 * g_mid is a device array of nF x nF tiles (nF = 2^(d Lc), tb_info.Lc) of
 * prod_k tb_info.rank_tgt[Lc][k] entries x nv each (element type of the
 * precision), tile (t, s) at position t nF + s, t and s the flat mid-level
 * multi-set indices (mode 0 most significant), entries in C order over the
 * padded ranks with the RHS innermost: for fixed t, the tiles of a range of s
 * are contiguous.  Complex128 and complex64 (TB_PREC_C64) only; the handle's
 * workspaces are used as in tb_apply (calls on one handle are stream-ordered).
 * Errors: TB_EINVAL (bad handle, range, pointers), TB_EUNSUPPORTED (separable
 * handle, split-BF16 or a precision not built), TB_ECUDA.
 */
tb_status tb_apply_src_part(tb_handle h, const void *f, void *g_mid, int64_t nv, int64_t s_begin, int64_t s_end,
                            int precision, void *cuda_stream);
tb_status tb_apply_tgt_part(tb_handle h, const void *g_mid, void *u, int64_t nv, int64_t t_begin, int64_t t_end,
                            int precision, void *cuda_stream);

/*
 * The partition of the nmid mid-level multi-sets over nranks ranks: contiguous
 * ranges [begin[g], end[g]) of near-equal size (the same plan serves the s and
 * the t ranges).  Host only.  TB_EINVAL for nmid < 1, nranks < 1 or NULL arrays.
 */
tb_status tb_shard_plan(int64_t nmid, int nranks, int64_t *begin, int64_t *end);

/*
 * Empirical tuning of the apply's launch shapes for nv right-hand sides at
 * `precision`, on the handle's own factors and workspaces (the paper fixes no
 * launch layout; this is the library's own schedule search):
 *  - non-separable handles: for every level pass, side and mode, the output
 *    rows per register tile (even values up to 24), the number of thread
 *    blocks per unit, the rank bounds (on or off) and the threads per block
 *    (the fewest covering a unit's columns, or 128); per pass, the fused,
 *    tensor-core (split-BF16 applies) or per-mode form; for the one-RHS
 *    forward core, stored or regenerated cores;
 *  - separable handles: per-mode passes with shared-memory fibers, with
 *    register-resident fibers (where the chain has the exact-rank form; see
 *    tb_options.sep_schedule) and multi-mode tile passes.
 * Each candidate runs a few times on `cuda_stream` (CUDA-event timed); the
 * fastest is kept in the handle and used by every later apply (results are
 * identical up to the summation order of separable passes).  Allocates two
 * temporary N x nv device buffers and frees them before returning.  Not for
 * use while the stream is being captured.  Status: TB_EINVAL on a bad handle,
 * nv or precision, TB_ECUDA on a CUDA error.
 */
tb_status tb_autotune(tb_handle h, int64_t nv, int precision, void *cuda_stream);

/*
 * Export of a built (non-separable) tensor butterfly, for checking the apply
 * step by step against an independent implementation of Alg. 2 (the paper has
 * no counterpart: a debugging interface).  All outputs are host memory;
 * calls with every array NULL only report the sizes; the copies are
 * synchronous.  TB_EUNSUPPORTED for separable handles.
 *
 * Index conventions (paper notation of Sec. 3.2 / Alg. 1):
 *   - A multi-set at level l has one node index per mode, i_k in [0, 2^l); its
 *     flat index is sum_k i_k 2^(l (d-1-k)) (mode 0 most significant).
 *     Node i at level l of mode k covers tree positions [i n_k / 2^l,
 *     (i+1) n_k / 2^l); tree position p is grid index perm_k[p]
 *     (tb_export_order).
 *   - tb_export_factors(side, level l, mode k): the blocks of
 *       side 0: V^{s,k}_{tau,nu} (l = 0) and W^{s,k}_{tau,nu} (l > 0),
 *       side 1: U^{t,k}_{tau,nu} (l = 0) and P^{t,k}_{tau,nu} (l > 0),
 *     block j = ((S 2^(d l) + T) 2^(Lc-l)) + q with S the flat mid-level
 *     multi-set of the side (s or t), T the flat level-l multi-set of the
 *     other tree (tau or nu) and q the node of mode k at depth Lc - l below
 *     S_k (nu for side 0, tau for side 1).  Each block is rows x cols complex128,
 *     row-major, rows = padded rank R_{l,k} (row a < ranks[j] is the a-th
 *     skeleton in pivot order, later rows are zero), cols = C_b,k (l = 0: the
 *     points of the leaf q in tree order) or 2 R_{l-1,k} (l > 0: the skeletons
 *     of the children 2q in [0, R_{l-1,k}) and 2q + 1 in [R_{l-1,k}, 2 R_{l-1,k}),
 *     each in its own pivot order, zero past the child's rank; the children's
 *     blocks are those of the parent multi-set p_T at level l - 1).
 *     skel[j * rows + a]: grid index along mode k of skeleton a (-1 past the rank).
 *     The source side applies a block as out = A in (contracting its columns),
 *     the target side as out = A^T in.
 *   - tb_export_cores: pair p = t nF + s (nF = 2^(d Lc)); dims[p * 2d + k] =
 *     |t-bar_k|, dims[p * 2d + d + k] = |s-bar_k| (the ranks of the level-Lc
 *     blocks of the pair); entries offsets[p] .. offsets[p+1] hold K(t-bar, s-bar)
 *     row-major, rows = target multi-index (C order over the modes), columns =
 *     source multi-index, complex128 (the complex64 cores widened when the
 *     handle was built without complex128).
 */
tb_status tb_export_factors(tb_handle h, int side, int level, int mode, int64_t *count, int *rows, int *cols,
                            int *ranks, int *skel, void *blocks);
tb_status tb_export_cores(tb_handle h, int64_t *pairs, int64_t *entries, int64_t *offsets, int *dims, void *core);
tb_status tb_export_order(tb_handle h, int axis, int *perm);

/* Describe a built handle (ranks, sizes, timings). */
tb_status tb_query(tb_handle h, tb_info *info);

/* Per-pass timing of eager applies (not of CUDA-graph replays). */
typedef struct {
    char name[24];          /* "leaf_in", "split", "core", "gather", "leaf_out" */
    int level;              /* tree level of the pass (core: Lc) */
    int adjoint;            /* 1 for passes of tb_apply_adjoint */
    int64_t launches;       /* executions of the pass recorded (one event pair each) */
    double ms_total;        /* summed device time of those executions (CUDA events) */
    int64_t bytes;          /* bytes one execution must move: its inputs, outputs
                               and factors at their stored sizes */
    double flops;           /* real floating-point operations of one execution */
    int64_t kernels;        /* kernel launches inside the recorded executions */
} tb_pass_stat;

/*
 * Enable (on = 1) or disable per-pass timing: while enabled, every eager
 * apply records a CUDA event pair around each pass (the kernel launches of one
 * step of Alg. 2) on the apply's stream.  Events add no work to the kernels
 * themselves.
 */
tb_status tb_profile_enable(tb_handle h, int on);

/*
 * Synchronize the recorded events, aggregate them by (name, level, adjoint)
 * into stats[0 .. *count) (at most `cap` entries, host memory) and clear the
 * record.
 */
tb_status tb_profile_stats(tb_handle h, tb_pass_stat *stats, int cap, int *count);

/*
 * Measured arithmetic throughput of the current CUDA device's FMA pipes, for
 * the ALU roofline of the apply's CUDA-core kernels (the paper has no
 * counterpart: this is a measurement utility of the library).  Runs a kernel
 * of independent fused multiply-add chains on every SM (FP32 scalar FFMA for
 * precision = TB_PREC_C64, FP64 DFMA for TB_PREC_C128), times it with CUDA
 * events on `cuda_stream` after one warm-up launch, and stores 2 x FMAs / s /
 * 1e12 in *tflops.  Allocates (and frees) a small device buffer; synchronous.
 * Errors: TB_EINVAL for a NULL tflops or another precision, TB_ECUDA.
 */
tb_status tb_alu_peak(int precision, void *cuda_stream, double *tflops);

/* Release everything the handle owns.  NULL is accepted (TB_OK). */
tb_status tb_free(tb_handle h);

/* Message of the last failing call on this host thread ("" if none). */
const char *tb_last_error(void);

/* Library version string. */
const char *tb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TB_H */

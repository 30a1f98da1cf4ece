// C ABI of the tensor butterfly library: argument checks, planning,
// construction orchestration (Alg. 1) and apply orchestration (Alg. 2).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <complex>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tb_kernels.cuh"
#include "tb_tc.cuh"
#include "tb_plan.cuh"

using namespace tb;

static thread_local std::string g_err;

// apply precisions this library implements (bit i = tb_precision i)
static const unsigned TB_PRECISIONS_BUILT =
    (1u << TB_PREC_C128) | (1u << TB_PREC_C64) | (1u << TB_PREC_C64_SPLITBF16);

static tb_status fail(tb_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

// The same for entry points defined in other translation units.
tb_status tb::fail_status(tb_status s, const std::string &msg) { return fail(s, msg); }

#define TB_CK(call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? TB_ENOMEM : TB_ECUDA,                  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                     \
        }                                                                                        \
    } while (0)

#define TB_TRY(expr)                      \
    do {                                  \
        tb_status s_ = (expr);            \
        if (s_ != TB_OK) return s_;       \
    } while (0)

namespace {

#ifndef TB_MODE_WAVES
#define TB_MODE_WAVES 32
#endif
size_t g_smem_optin = 0;
int64_t g_num_sms = 0;

bool pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2(int64_t x) {
    int r = 0;
    while ((int64_t(1) << r) < x) ++r;
    return r;
}

template <class T>
tb_status dalloc(tb_plan *h, T **p, int64_t count) {
    *p = nullptr;
    if (count <= 0) return TB_OK;
    cudaError_t e = cudaMalloc((void **)p, (size_t)count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TB_ENOMEM, "cudaMalloc of " + std::to_string((size_t)count * sizeof(T)) + " bytes failed");
    }
    h->allocations.push_back((void *)*p);
    h->device_bytes += (int64_t)count * sizeof(T);
    return TB_OK;
}

void dfree(tb_plan *h, void *p) {
    if (!p) return;
    auto it = std::find(h->allocations.begin(), h->allocations.end(), p);
    if (it != h->allocations.end()) h->allocations.erase(it);
    cudaFree(p);
}

int64_t prod_tile(const SideLevel &s, int d) {
    int64_t t = 1;
    for (int k = 0; k < d; ++k) t *= s.R[k];
    return t;
}

// Right-hand-side counts whose tensors (N x nv entries of es bytes) have a
// byte size representable in size_t and whose level tiles index with int
// (the kernels take nv as int; level_pass checks the tile sizes).
tb_status check_nv(int64_t N, int64_t nv, size_t es) {
    if (nv > (int64_t)INT32_MAX) return fail(TB_EUNSUPPORTED, "nv above 2^31 - 1 is not supported");
    if (N > 0 && (uint64_t)nv > (uint64_t)(SIZE_MAX / es) / (uint64_t)N)
        return fail(TB_EINVAL, "N x nv x element size overflows the address space");
    return TB_OK;
}

// Complex multiply-adds per RHS of a chain X (dims m) -> Y (dims o) applied
// in the mode order `ord`.
double chain_cmacs_order(int d, const int *m, const int *o, const int *ord) {
    int cur[TB_MAX_D];
    for (int k = 0; k < d; ++k) cur[k] = m[k];
    double f = 0.0;
    for (int i = 0; i < d; ++i) {
        const int k = ord[i];
        double t = (double)m[k] * o[k];
        for (int j = 0; j < d; ++j)
            if (j != k) t *= cur[j];
        f += t;
        cur[k] = o[k];
    }
    return f;
}

// The mode order with the fewest multiply-adds (ties: lexicographically first).
double best_order(int d, const int *m, const int *o, int *ord) {
    std::vector<int> p((size_t)d);
    for (int k = 0; k < d; ++k) p[(size_t)k] = k;
    double best = -1.0;
    do {
        const double f = chain_cmacs_order(d, m, o, p.data());
        if (best < 0.0 || f < best) {
            best = f;
            for (int k = 0; k < d; ++k) ord[k] = p[(size_t)k];
        }
    } while (std::next_permutation(p.begin(), p.end()));
    return best;
}

// Input / output lengths of each mode of one unit of a level pass.
void pass_dims(const tb_plan *h, Pass pass, int side, int l, int *m, int *o) {
    const SideLevel *S = side == 0 ? h->src : h->tgt;
    for (int k = 0; k < h->d; ++k) {
        switch (pass) {
            case Pass::LeafIn: m[k] = (int)h->cb[k]; o[k] = S[0].R[k]; break;
            case Pass::LeafOut: m[k] = S[0].R[k]; o[k] = (int)h->cb[k]; break;
            case Pass::Split: m[k] = 2 * S[l - 1].R[k]; o[k] = S[l].R[k]; break;
            case Pass::Gather: m[k] = S[l].R[k]; o[k] = 2 * S[l - 1].R[k]; break;
        }
    }
}

// Mode order of a pass as per-mode launches: the fewest multiply-adds among
// the orders the launch kinds allow (the user-tensor input of a LeafIn is
// read by mode 0 first, as are the parent tiles of a Split, the parent tiles of
// a Gather are written by mode d - 1 last; a LeafOut may end on any mode).
// Among orders of equal cost the lexicographically last is taken.
void mode_order_permode(const tb_plan *h, Pass pass, int side, int l, int *ord) {
    const int d = h->d;
    int m[TB_MAX_D], o[TB_MAX_D];
    pass_dims(h, pass, side, l, m, o);
    std::vector<int> p((size_t)d);
    for (int k = 0; k < d; ++k) p[(size_t)k] = k;
    double best = -1.0;
    do {
        if ((pass == Pass::LeafIn || pass == Pass::Split) && p[0] != 0) continue;
        if (pass == Pass::Gather && p[(size_t)d - 1] != d - 1) continue;
        const double f = chain_cmacs_order(d, m, o, p.data());
        if (best < 0.0 || f <= best) {   // ties: the last order
            best = f;
            for (int k = 0; k < d; ++k) ord[k] = p[(size_t)k];
        }
    } while (std::next_permutation(p.begin(), p.end()));
}


tb_status check_device_ptr(const void *p, const char *what) {
    if (!p) return fail(TB_EINVAL, std::string(what) + " is NULL");
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TB_EINVAL, std::string(what) + " is not a CUDA pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(TB_EINVAL, std::string(what) + " is not device memory");
    return TB_OK;
}

}  // namespace

extern "C" {

const char *tb_last_error(void) { return g_err.c_str(); }
const char *tb_version(void) { return "tb 0.1 (sm_103a)"; }

tb_status tb_options_default(tb_options *o) {
    if (!o) return fail(TB_EINVAL, "options pointer is NULL");
    o->L = -1;
    o->order = TB_ORDER_AUTO;
    o->proxy_rows = 1024;
    o->rank_max = 32;
    o->precisions = 0;
    o->separable = -1;
    o->use_graphs = 0;
    o->device = -1;
    o->seed = 0x5eed;
    o->autotune = 0;
    o->sep_schedule = 0;
    o->level_schedule = 0;
    o->core_mode = 0;
    o->mode_slices = 0;
    return TB_OK;
}

tb_status tb_free(tb_handle h) {
    if (!h) return TB_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    for (void *p : h->allocations) cudaFree(p);
    if (h->ws.buf[0]) cudaFree(h->ws.buf[0]);
    if (h->ws.buf[1]) cudaFree(h->ws.buf[1]);
    if (h->ws.mbuf[0]) cudaFree(h->ws.mbuf[0]);
    if (h->ws.mbuf[1]) cudaFree(h->ws.mbuf[1]);
    if (h->ws.cout[0]) cudaFree(h->ws.cout[0]);
    if (h->ws.cout[1]) cudaFree(h->ws.cout[1]);
    if (h->ws.host_in) cudaFree(h->ws.host_in);
    if (h->ws.host_out) cudaFree(h->ws.host_out);
    for (int b = 0; b < 2; ++b) {
        if (h->pipe.din[b]) cudaFree(h->pipe.din[b]);
        if (h->pipe.dout[b]) cudaFree(h->pipe.dout[b]);
        for (cudaEvent_t e : {h->pipe.in_ready[b], h->pipe.in_free[b], h->pipe.out_ready[b], h->pipe.out_free[b]})
            if (e) cudaEventDestroy(e);
    }
    for (int i = 0; i < 3; ++i)
        if (h->pipe.s[i]) cudaStreamDestroy(h->pipe.s[i]);
    cudaSetDevice(cur);
    delete h;
    return TB_OK;
}

}  // extern "C"

// -------------------------------------------------------------- construction
static tb_status build_side(tb_plan *h, int side) {
    const int d = h->d, Lc = h->Lc;
    const int64_t nF = ipow2(d * Lc);
    SideLevel *lv = side == 0 ? h->src : h->tgt;
    for (int l = 0; l <= Lc; ++l) {
        SideLevel &S = lv[l];
        const int64_t nM = ipow2(d * l);
        const int nseg = 1 << (Lc - l);
        IdArgs a;
        std::memset(&a, 0, sizeof(a));
        a.side = side;
        a.d = d;
        a.l = l;
        a.Lc = Lc;
        a.separable = h->separable;
        a.ks = h->ks;
        a.rows_cap = h->proxy_rows;
        a.rows_bits = ilog2(h->proxy_rows);
        a.tol = h->tol;
        a.rank_max = h->rank_max;
        a.seed = (uint32_t)(h->seed ^ (h->seed >> 32));
        a.err = h->d_err;
        int ncmax = 0;
        for (int k = 0; k < d; ++k) {
            a.n[k] = (int)h->n[k];
            a.cb[k] = (int)h->cb[k];
            a.perm[k] = h->perm[k];
            a.own[k] = side == 0 ? h->ys[k] : h->xs[k];
            a.oth[k] = side == 0 ? h->xs[k] : h->ys[k];
            S.cin[k] = l == 0 ? (int)h->cb[k] : 2 * lv[l - 1].R[k];
            S.cap[k] = std::min(S.cin[k], h->rank_max);
            S.count[k] = h->separable ? ipow2(h->L) : nF * nM * nseg;
            ncmax = std::max(ncmax, S.cin[k]);
            if (l > 0) {
                a.pskel[k] = lv[l - 1].skel[k];
                a.prank[k] = lv[l - 1].rank[k];
                a.pcap[k] = lv[l - 1].cap[k];
                a.pR[k] = lv[l - 1].R[k];
            }
        }
        if (ncmax > id_max_columns())
            return fail(TB_ERANK, "level " + std::to_string(l) + " needs " + std::to_string(ncmax) +
                                      " candidate columns; the ID kernel holds at most " +
                                      std::to_string(id_max_columns()));
        a.ncmax = ncmax;
        for (int k = 0; k < d; ++k) {
            TB_TRY(dalloc(h, &S.fac64[k], S.count[k] * S.cap[k] * S.cin[k]));
            TB_TRY(dalloc(h, &S.skel[k], S.count[k] * S.cap[k]));
            TB_TRY(dalloc(h, &S.rank[k], S.count[k]));
            a.fac[k] = S.fac64[k];
            a.skel[k] = S.skel[k];
            a.rank[k] = S.rank[k];
            a.cap[k] = S.cap[k];
            a.cin[k] = S.cin[k];
        }
        a.nids = h->separable ? (int64_t)d * ipow2(h->L) : nF * nM * d * nseg;
        h->num_ids += a.nids;
        TB_CK(launch_interp_decomp(a, 0));
        TB_CK(cudaDeviceSynchronize());
        int err = 0;
        TB_CK(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (err == 2)
            return fail(TB_ERANK, "an ID at level " + std::to_string(l) + " needs more than rank cap " +
                                      std::to_string(h->rank_max) + " at tolerance " + std::to_string(h->tol));
        // padded ranks R_{l,k} and rank statistics
        S.rmin = 1 << 30;
        S.rmax = 0;
        for (int k = 0; k < d; ++k) {
            std::vector<int> rk((size_t)S.count[k]);
            TB_CK(cudaMemcpy(rk.data(), S.rank[k], rk.size() * sizeof(int), cudaMemcpyDeviceToHost));
            int mx = 1, mn = 1 << 30;
            for (int r : rk) { mx = std::max(mx, r); mn = std::min(mn, r); }
            S.R[k] = mx;
            S.rmin = std::min(S.rmin, mn);
            S.rmax = std::max(S.rmax, mx);
            if (S.R[k] < S.cap[k]) {   // drop the unused padding rows
                c128 *packed = nullptr;
                TB_TRY(dalloc(h, &packed, S.count[k] * S.R[k] * S.cin[k]));
                const size_t w = (size_t)S.R[k] * S.cin[k] * sizeof(c128);
                const size_t sp = (size_t)S.cap[k] * S.cin[k] * sizeof(c128);
                TB_CK(cudaMemcpy2D(packed, w, S.fac64[k], sp, w, (size_t)S.count[k], cudaMemcpyDeviceToDevice));
                dfree(h, S.fac64[k]);
                h->device_bytes -= S.count[k] * S.cap[k] * S.cin[k] * (int64_t)sizeof(c128);
                S.fac64[k] = packed;
            }
        }
        h->rank_min = std::min(h->rank_min, S.rmin);
        h->rank_max_seen = std::max(h->rank_max_seen, S.rmax);
    }
    return TB_OK;
}

static tb_status build_cores(tb_plan *h) {
    const int d = h->d, Lc = h->Lc;
    const int64_t nF = ipow2(d * Lc);
    h->P = nF * nF;
    const bool want64 = h->precisions & (1u << TB_PREC_C128);
    const bool want32 = h->precisions & ((1u << TB_PREC_C64) | (1u << TB_PREC_C64_SPLITBF16));
    SideLevel &T = h->tgt[Lc], &S = h->src[Lc];
    if (h->separable) {
        const int nb = 1 << Lc;
        for (int k = 0; k < d; ++k) {
            const int64_t cnt = (int64_t)nb * nb * T.R[k] * S.R[k];
            (void)want64;   // FP64 per-mode cores are always kept: they feed the separable chains
            TB_TRY(dalloc(h, &h->kron64[k], cnt));
            if (want32) TB_TRY(dalloc(h, &h->kron32[k], cnt));
            KronArgs a;
            a.Lc = Lc;
            a.Rt = T.R[k];
            a.Rs = S.R[k];
            a.tcap = T.cap[k];
            a.scap = S.cap[k];
            a.trank = T.rank[k];
            a.srank = S.rank[k];
            a.tskel = T.skel[k];
            a.sskel = S.skel[k];
            a.xk = h->xs[k];
            a.yk = h->ys[k];
            a.ks = h->ks;
            a.out64 = h->kron64[k];
            a.out32 = h->kron32[k];
            TB_CK(launch_kron_eval(a, 0));
            h->core_entries += cnt;
        }
        TB_CK(cudaDeviceSynchronize());
        return TB_OK;
    }
    std::vector<std::vector<int>> rt(d), rs(d);
    for (int k = 0; k < d; ++k) {
        rt[k].resize((size_t)T.count[k]);
        rs[k].resize((size_t)S.count[k]);
        TB_CK(cudaMemcpy(rt[k].data(), T.rank[k], rt[k].size() * sizeof(int), cudaMemcpyDeviceToHost));
        TB_CK(cudaMemcpy(rs[k].data(), S.rank[k], rs[k].size() * sizeof(int), cudaMemcpyDeviceToHost));
    }
    std::vector<int> dims((size_t)h->P * 2 * d);
    std::vector<int64_t> off((size_t)h->P + 1);
    int64_t acc = 0;
    for (int64_t p = 0; p < h->P; ++p) {
        const int64_t t = p / nF, s = p % nF;
        int64_t mt = 1, ms = 1;
        for (int k = 0; k < d; ++k) {
            const int a = rt[k][(size_t)(t * nF + s)], b = rs[k][(size_t)(s * nF + t)];
            dims[(size_t)p * 2 * d + k] = a;
            dims[(size_t)p * 2 * d + d + k] = b;
            mt *= a;
            ms *= b;
        }
        off[(size_t)p] = acc;
        acc += mt * ms;
        h->core_out_entries += mt;
        h->core_in_entries += ms;
    }
    off[(size_t)h->P] = acc;
    h->core_entries = acc;
    TB_TRY(dalloc(h, &h->core_dims, (int64_t)dims.size()));
    TB_TRY(dalloc(h, &h->core_off, (int64_t)off.size()));
    TB_CK(cudaMemcpy(h->core_dims, dims.data(), dims.size() * sizeof(int), cudaMemcpyHostToDevice));
    TB_CK(cudaMemcpy(h->core_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    if (want64) TB_TRY(dalloc(h, &h->core64, acc));
    if (want32) TB_TRY(dalloc(h, &h->core32, acc));
    CoreArgs a;
    std::memset(&a, 0, sizeof(a));
    a.d = d;
    a.P = h->P;
    a.nF = nF;
    a.dims = h->core_dims;
    a.off = h->core_off;
    for (int k = 0; k < d; ++k) {
        a.tskel[k] = T.skel[k];
        a.sskel[k] = S.skel[k];
        a.tcap[k] = T.cap[k];
        a.scap[k] = S.cap[k];
        a.xs[k] = h->xs[k];
        a.ys[k] = h->ys[k];
    }
    a.ks = h->ks;
    a.out64 = h->core64;
    a.out32 = h->core32;
    TB_CK(launch_core_eval(a, 0));
    TB_CK(cudaDeviceSynchronize());
    if (h->precisions & (1u << TB_PREC_C64_SPLITBF16)) {
        // split-BF16 tiles of K(t-bar, s-bar) and of its conjugate transpose
        const int NTc = core_tc_rows_per_item(), KCc = core_tc_cols_per_chunk();
        for (int dir = 0; dir < 2; ++dir) {
            std::vector<CoreItem> items;
            std::vector<int> xpos;   // per pair: padded position of each compact input index (-1 = none)
            const SideLevel &Sin = dir ? h->tgt[h->Lc] : h->src[h->Lc];
            int64_t boff = 0;
            for (int64_t p = 0; p < h->P; ++p) {
                int64_t mt = 1, ms = 1;
                int rin[TB_MAX_D], rout[TB_MAX_D];
                for (int k = 0; k < d; ++k) {
                    const int rt = dims[(size_t)p * 2 * d + k], rs = dims[(size_t)p * 2 * d + d + k];
                    mt *= rt;
                    ms *= rs;
                    rin[k] = dir ? rt : rs;
                    rout[k] = dir ? rs : rt;
                }
                const int64_t nrows = dir ? ms : mt, ncols = dir ? mt : ms;
                const int64_t np = (nrows + 15) / 16 * 16;
                const int nkc = (int)((ncols + KCc - 1) / KCc);
                const int64_t x0 = (int64_t)xpos.size();
                for (int64_t c = 0; c < (int64_t)nkc * KCc; ++c) {
                    int pos = -1;
                    if (c < ncols) {
                        int64_t idx = c;
                        int stride = 1;
                        pos = 0;
                        for (int k = d - 1; k >= 0; --k) {
                            pos += (int)(idx % rin[k]) * stride;
                            idx /= rin[k];
                            stride *= Sin.R[k];
                        }
                    }
                    xpos.push_back(pos);
                }
                for (int64_t j = 0; j * NTc < np; ++j) {
                    const int rows = (int)std::min<int64_t>(NTc, np - j * NTc);
                    CoreItem it;
                    std::memset(&it, 0, sizeof(it));
                    it.pair = (int)p;
                    it.tile = (int)j;
                    it.rows = rows;
                    it.nkc = nkc;
                    it.boff = boff;
                    it.xpos = x0;
                    for (int k = 0; k < d; ++k) it.rout[k] = rout[k];
                    items.push_back(it);
                    boff += (int64_t)nkc * rows * 256;
                }
            }
            TB_TRY(dalloc(h, &h->tc_xpos[dir], (int64_t)std::max<size_t>(xpos.size(), 1)));
            TB_CK(cudaMemcpy(h->tc_xpos[dir], xpos.data(), xpos.size() * sizeof(int), cudaMemcpyHostToDevice));
            h->tc_nitems[dir] = (int64_t)items.size();
            h->tc_bytes[dir] = boff;
            TB_TRY(dalloc(h, &h->tc_items[dir], (int64_t)items.size()));
            TB_CK(cudaMemcpy(h->tc_items[dir], items.data(), items.size() * sizeof(CoreItem), cudaMemcpyHostToDevice));
            TB_TRY(dalloc(h, &h->tc_tiles[dir], boff));
            CoreTileArgs ta;
            std::memset(&ta, 0, sizeof(ta));
            ta.d = d;
            ta.adjoint = dir;
            ta.nitems = h->tc_nitems[dir];
            ta.items = h->tc_items[dir];
            ta.dims = h->core_dims;
            ta.core_off = h->core_off;
            ta.c128 = h->core64;
            ta.c64 = h->core32;
            ta.out = h->tc_tiles[dir];
            TB_CK(launch_core_tile(ta, 0));
        }
        TB_CK(cudaDeviceSynchronize());
    }
    return TB_OK;
}

extern "C" tb_status tb_build(const tb_kernel *kernel, int d, const int64_t *n, const tb_grids *grids,
                              double tol, tb_handle *out) {
    return tb_build_ex(kernel, d, n, grids, tol, nullptr, out);
}

// --------------------------------------------------- separable (per-mode) chains
namespace {

struct HostStep {
    int n_out = 0, n_in = 0;
    std::vector<int> rowptr, col;
    std::vector<std::complex<double>> val;
};

// Sparse step built row by row: rows are appended in order, explicit zeros dropped.
struct StepBuilder {
    HostStep s;
    StepBuilder(int n_out, int n_in) {
        s.n_out = n_out;
        s.n_in = n_in;
        s.rowptr.push_back(0);
    }
    void add(int c, std::complex<double> v) {
        if (v != std::complex<double>(0.0, 0.0)) {
            s.col.push_back(c);
            s.val.push_back(v);
        }
    }
    void end_row() { s.rowptr.push_back((int)s.col.size()); }
};

HostStep conj_transpose(const HostStep &a) {
    HostStep t;
    t.n_out = a.n_in;
    t.n_in = a.n_out;
    std::vector<std::vector<std::pair<int, std::complex<double>>>> rows((size_t)a.n_in);
    for (int r = 0; r < a.n_out; ++r)
        for (int j = a.rowptr[(size_t)r]; j < a.rowptr[(size_t)r + 1]; ++j)
            rows[(size_t)a.col[(size_t)j]].push_back({r, std::conj(a.val[(size_t)j])});
    t.rowptr.push_back(0);
    for (auto &row : rows) {
        for (auto &e : row) {
            t.col.push_back(e.first);
            t.val.push_back(e.second);
        }
        t.rowptr.push_back((int)t.col.size());
    }
    return t;
}

}  // namespace

// Register-resident form of mode k's chain (sepr_col): eligible when the
// chain has N = C_b 4^Lc entries at every level, V and U^T are permutation
// matrices (every row a single exact 1) and every other step's nonzeros lie
// in the dense-block pattern.  Fills the load / store positions and the
// dense coefficients (zero where the CSR step dropped an exact zero).
static tb_status build_sep_reg(tb_plan *h, int k, const std::vector<HostStep> &st) {
    const int lc = h->Lc, rk = (int)h->cb[k], N = rk << (2 * lc), nk = (int)h->n[k];
    h->sepr_ok[k] = 0;
    if (N != nk || N > SEPR_MAXN || (int)st.size() != 2 * lc + 3) return TB_OK;
    if (!sep_reg_supported<float>(lc, rk) && !sep_reg_supported<double>(lc, rk)) return TB_OK;
    for (const HostStep &s : st)
        if (s.n_out != N || s.n_in != N) return TB_OK;
    const std::complex<double> one(1.0, 0.0);
    // V (first step): row e reads grid position ld[e]; U^T (last): row g reads entry e, so st[e] = g
    std::vector<int> ld(N, -1), sto(N, -1), seen(N, 0), seen2(N, 0);
    const HostStep &V = st.front(), &U = st.back();
    for (int e = 0; e < N; ++e) {
        if (V.rowptr[e + 1] - V.rowptr[e] != 1 || V.val[V.rowptr[e]] != one) return TB_OK;
        const int c = V.col[V.rowptr[e]];
        if (seen[c]++) return TB_OK;
        ld[e] = c;
        if (U.rowptr[e + 1] - U.rowptr[e] != 1 || U.val[U.rowptr[e]] != one) return TB_OK;
        const int c2 = U.col[U.rowptr[e]];
        if (seen2[c2]++) return TB_OK;
        sto[c2] = e;
    }
    std::vector<std::complex<double>> coef((size_t)sepr_ncoef(lc, rk), std::complex<double>(0.0, 0.0));
    for (int i = 0; i <= 2 * lc; ++i) {
        const HostStep &S = st[(size_t)i + 1];
        const int K = sepr_width(lc, rk, i), off = sepr_off(lc, rk, i);
        for (int e = 0; e < N; ++e)
            for (int j = S.rowptr[e]; j < S.rowptr[e + 1]; ++j) {
                int pos = -1;
                for (int q = 0; q < K && pos < 0; ++q)
                    if (sepr_col(lc, rk, i, e, q) == S.col[j]) pos = q;
                if (pos < 0) return TB_OK;   // a nonzero outside the dense-block pattern
                coef[(size_t)(off + e * K + pos)] = S.val[j];
            }
    }
    std::vector<c128> c64v(coef.size());
    std::vector<c64> c32v(coef.size());
    for (size_t i = 0; i < coef.size(); ++i) {
        c64v[i] = c128{coef[i].real(), coef[i].imag()};
        c32v[i] = c64{(float)coef[i].real(), (float)coef[i].imag()};
    }
    TB_TRY(dalloc(h, &h->sepr_coef64[k], (int64_t)coef.size()));
    TB_TRY(dalloc(h, &h->sepr_coef32[k], (int64_t)coef.size()));
    TB_CK(cudaMemcpy(h->sepr_coef64[k], c64v.data(), c64v.size() * sizeof(c128), cudaMemcpyHostToDevice));
    TB_CK(cudaMemcpy(h->sepr_coef32[k], c32v.data(), c32v.size() * sizeof(c64), cudaMemcpyHostToDevice));
    for (int dir = 0; dir < 2; ++dir) {
        std::vector<float4> f4(coef.size());
        for (size_t i = 0; i < coef.size(); ++i) {
            const float re = (float)coef[i].real(), im = (float)coef[i].imag();
            f4[i] = make_float4(re, re, im, dir ? -im : im);
        }
        TB_TRY(dalloc(h, &h->sepr_cf4[dir][k], (int64_t)f4.size()));
        TB_CK(cudaMemcpy(h->sepr_cf4[dir][k], f4.data(), f4.size() * sizeof(float4), cudaMemcpyHostToDevice));
    }
    for (int e = 0; e < N; ++e) {
        h->sepr_ld[k][e] = ld[(size_t)e];
        h->sepr_st[k][e] = sto[(size_t)e];
    }
    h->sepr_rk[k] = rk;
    h->sepr_ok[k] = 1;
    return TB_OK;
}

// The per-mode chains of a separable handle: step matrices on the 1-D index
// of mode k, assembled from the factor blocks (which depend on the mode-k
// nodes only).  Source level l index: ((s 2^l + tau) 2^(Lc-l) + nu) R_l + a;
// target level l index: ((t 2^l + nu) 2^(Lc-l) + tau) R_l + a.
static tb_status build_sep_steps(tb_plan *h) {
    const int d = h->d, Lc = h->Lc, L = h->L;
    using C = std::complex<double>;
    auto fetch = [&](const c128 *p, int64_t n, std::vector<C> &out) -> tb_status {
        std::vector<c128> tmp((size_t)n);
        TB_CK(cudaMemcpy(tmp.data(), p, (size_t)n * sizeof(c128), cudaMemcpyDeviceToHost));
        out.resize((size_t)n);
        for (int64_t i = 0; i < n; ++i) out[(size_t)i] = C(tmp[(size_t)i].x, tmp[(size_t)i].y);
        return TB_OK;
    };
    std::vector<HostStep> all[2];
    for (int k = 0; k < d; ++k) {
        const int nk = (int)h->n[k], cb = (int)h->cb[k], nmid = nk >> Lc, nb = 1 << Lc;
        std::vector<int> perm((size_t)nk);
        const int bits = ilog2(nk);
        for (int p = 0; p < nk; ++p) {
            int q = p;
            if (h->order == TB_ORDER_BITREV) {
                q = 0;
                for (int b = 0; b < bits; ++b) q |= ((p >> b) & 1) << (bits - 1 - b);
            }
            perm[(size_t)p] = q;
        }
        std::vector<std::vector<C>> fs(Lc + 1), ft(Lc + 1);
        for (int l = 0; l <= Lc; ++l) {
            TB_TRY(fetch(h->src[l].fac64[k], h->src[l].count[k] * h->src[l].R[k] * h->src[l].cin[k], fs[l]));
            TB_TRY(fetch(h->tgt[l].fac64[k], h->tgt[l].count[k] * h->tgt[l].R[k] * h->tgt[l].cin[k], ft[l]));
        }
        std::vector<C> kr;
        const int Rt = h->tgt[Lc].R[k], Rs = h->src[Lc].R[k];
        TB_TRY(fetch(h->kron64[k], (int64_t)nb * nb * Rt * Rs, kr));
        auto Rsrc = [&](int l) { return h->src[l].R[k]; };
        auto Rtgt = [&](int l) { return h->tgt[l].R[k]; };
        auto esrc = [&](int l, int s, int tau, int nu, int a) {
            return ((((s << l) + tau) << (Lc - l)) + nu) * Rsrc(l) + a;
        };
        auto etgt = [&](int l, int t, int nu, int tau, int a) {
            return ((((t << l) + nu) << (Lc - l)) + tau) * Rtgt(l) + a;
        };
        // factor block (F, M, sig) of side-level data, R x cin, row-major
        auto blk = [&](const std::vector<C> &f, const SideLevel &S, int l, int F, int M, int sig, int a, int c) {
            const int64_t j = ((((int64_t)F << l) + M) << (Lc - l)) + sig;
            return f[(size_t)((j * S.R[k] + a) * S.cin[k] + c)];
        };
        std::vector<HostStep> st;
        // source leaves: V
        {
            StepBuilder b(esrc(0, nb - 1, 0, nb - 1, Rsrc(0) - 1) + 1, nk);
            for (int s = 0; s < nb; ++s)
                for (int nu = 0; nu < nb; ++nu)
                    for (int a = 0; a < Rsrc(0); ++a) {
                        for (int c = 0; c < cb; ++c)
                            b.add(perm[(size_t)(s * nmid + nu * cb + c)], blk(fs[0], h->src[0], 0, s, 0, nu, a, c));
                        b.end_row();
                    }
            st.push_back(b.s);
        }
        // source transfers: W
        for (int l = 1; l <= Lc; ++l) {
            const int ns = 1 << (Lc - l);
            StepBuilder b(nb * (1 << l) * ns * Rsrc(l), nb * (1 << (l - 1)) * 2 * ns * Rsrc(l - 1));
            for (int s = 0; s < nb; ++s)
                for (int tau = 0; tau < (1 << l); ++tau)
                    for (int nu = 0; nu < ns; ++nu)
                        for (int a = 0; a < Rsrc(l); ++a) {
                            for (int c = 0; c < 2; ++c)
                                for (int q = 0; q < Rsrc(l - 1); ++q)
                                    b.add(esrc(l - 1, s, tau >> 1, 2 * nu + c, q),
                                          blk(fs[l], h->src[l], l, s, tau, nu, a, c * Rsrc(l - 1) + q));
                            b.end_row();
                        }
            st.push_back(b.s);
        }
        // core: K_k(t-bar_k, s-bar_k)
        {
            StepBuilder b(nb * nb * Rt, nb * nb * Rs);
            for (int t = 0; t < nb; ++t)
                for (int s = 0; s < nb; ++s)
                    for (int a = 0; a < Rt; ++a) {
                        for (int q = 0; q < Rs; ++q)
                            b.add(esrc(Lc, s, t, 0, q), kr[(size_t)(((int64_t)t * nb + s) * Rt * Rs + a * Rs + q)]);
                        b.end_row();
                    }
            st.push_back(b.s);
        }
        // target transfers: P (gather over the two children of each source node)
        for (int l = Lc; l >= 1; --l) {
            const int ns = 1 << (Lc - l);
            StepBuilder b(nb * (1 << (l - 1)) * 2 * ns * Rtgt(l - 1), nb * (1 << l) * ns * Rtgt(l));
            for (int t = 0; t < nb; ++t)
                for (int pn = 0; pn < (1 << (l - 1)); ++pn)
                    for (int tp = 0; tp < 2 * ns; ++tp)
                        for (int a = 0; a < Rtgt(l - 1); ++a) {
                            for (int c = 0; c < 2; ++c)
                                for (int q = 0; q < Rtgt(l); ++q)
                                    b.add(etgt(l, t, 2 * pn + c, tp >> 1, q),
                                          blk(ft[l], h->tgt[l], l, t, 2 * pn + c, tp >> 1, q,
                                              (tp & 1) * Rtgt(l - 1) + a));
                            b.end_row();
                        }
            st.push_back(b.s);
        }
        // target leaves: U^T, rows in grid order
        {
            StepBuilder b(nk, nb * nb * Rtgt(0));
            std::vector<int> owner((size_t)nk);
            for (int p = 0; p < nk; ++p) owner[(size_t)perm[(size_t)p]] = p;
            for (int g = 0; g < nk; ++g) {
                const int p = owner[(size_t)g];
                const int t = p / nmid, tau = (p % nmid) / cb, a = p % cb;
                for (int q = 0; q < Rtgt(0); ++q) b.add(etgt(0, t, 0, tau, q), blk(ft[0], h->tgt[0], 0, t, 0, tau, q, a));
                b.end_row();
            }
            st.push_back(b.s);
        }
        TB_TRY(build_sep_reg(h, k, st));
        int mx = nk;
        for (auto &s : st) mx = std::max({mx, s.n_out, s.n_in});
        h->sep_maxext[k] = mx;
        h->sep_step0[0][k] = (int)all[0].size();
        h->sep_nsteps[0][k] = (int)st.size();
        h->sep_step0[1][k] = (int)all[1].size();
        h->sep_nsteps[1][k] = (int)st.size();
        for (auto &s : st) {
            h->sep_nnz[0][k] += (int64_t)s.col.size();
            h->sep_nidx[0][k] += s.n_out + 1;
            all[0].push_back(s);
        }
        for (auto it = st.rbegin(); it != st.rend(); ++it) {   // adjoint: reversed, conjugate transposed
            all[1].push_back(conj_transpose(*it));
            h->sep_nnz[1][k] += (int64_t)it->col.size();
            h->sep_nidx[1][k] += it->n_in + 1;
        }
    }
    // upload: shared index arrays, FP64 and FP32 values, step descriptors
    for (int dir = 0; dir < 2; ++dir) {
        std::vector<int> idx;
        std::vector<c128> v64;
        std::vector<c64> v32;
        std::vector<std::pair<int64_t, int64_t>> off;   // (rowptr offset, col/val offset)
        for (auto &s : all[dir]) {
            off.push_back({(int64_t)idx.size(), (int64_t)v64.size()});
            idx.insert(idx.end(), s.rowptr.begin(), s.rowptr.end());
            for (size_t j = 0; j < s.col.size(); ++j) {
                v64.push_back(c128{s.val[j].real(), s.val[j].imag()});
                v32.push_back(c64{(float)s.val[j].real(), (float)s.val[j].imag()});
            }
        }
        std::vector<int> cols;
        for (auto &s : all[dir]) cols.insert(cols.end(), s.col.begin(), s.col.end());
        int *d_idx = nullptr, *d_col = nullptr;
        c128 *d_v64 = nullptr;
        c64 *d_v32 = nullptr;
        TB_TRY(dalloc(h, &d_idx, (int64_t)std::max<size_t>(idx.size(), 1)));
        TB_TRY(dalloc(h, &d_col, (int64_t)std::max<size_t>(cols.size(), 1)));
        TB_TRY(dalloc(h, &d_v64, (int64_t)std::max<size_t>(v64.size(), 1)));
        TB_TRY(dalloc(h, &d_v32, (int64_t)std::max<size_t>(v32.size(), 1)));
        TB_CK(cudaMemcpy(d_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
        TB_CK(cudaMemcpy(d_col, cols.data(), cols.size() * sizeof(int), cudaMemcpyHostToDevice));
        TB_CK(cudaMemcpy(d_v64, v64.data(), v64.size() * sizeof(c128), cudaMemcpyHostToDevice));
        TB_CK(cudaMemcpy(d_v32, v32.data(), v32.size() * sizeof(c64), cudaMemcpyHostToDevice));
        // packed row-ordered streams (one zero entry for an empty row)
        std::vector<SepNz<double>> p64;
        std::vector<SepNz<float>> p32;
        std::vector<std::pair<int64_t, int>> poff;   // (offset, count) per step
        for (auto &s : all[dir]) {
            const int64_t o0 = (int64_t)p64.size();
            for (int r = 0; r < s.n_out; ++r) {
                const int j0 = s.rowptr[(size_t)r], j1 = s.rowptr[(size_t)r + 1];
                if (j0 == j1) {
                    p64.push_back(SepNz<double>{c128{0.0, 0.0}, 0, 1});
                    p32.push_back(SepNz<float>{c64{0.f, 0.f}, 0, 1});
                }
                for (int j = j0; j < j1; ++j) {
                    const auto v = s.val[(size_t)j];
                    p64.push_back(SepNz<double>{c128{v.real(), v.imag()}, s.col[(size_t)j], j + 1 == j1 ? 1 : 0});
                    p32.push_back(SepNz<float>{c64{(float)v.real(), (float)v.imag()}, s.col[(size_t)j],
                                               j + 1 == j1 ? 1 : 0});
                }
            }
            poff.push_back({o0, (int)((int64_t)p64.size() - o0)});
        }
        SepNz<double> *d_p64 = nullptr;
        SepNz<float> *d_p32 = nullptr;
        TB_TRY(dalloc(h, &d_p64, (int64_t)std::max<size_t>(p64.size(), 1)));
        TB_TRY(dalloc(h, &d_p32, (int64_t)std::max<size_t>(p32.size(), 1)));
        TB_CK(cudaMemcpy(d_p64, p64.data(), p64.size() * sizeof(p64[0]), cudaMemcpyHostToDevice));
        TB_CK(cudaMemcpy(d_p32, p32.data(), p32.size() * sizeof(p32[0]), cudaMemcpyHostToDevice));
        for (int k = 0; k < d; ++k) {
            h->sep_npk[dir][k] = 0;
            for (int i = 0; i < h->sep_nsteps[dir][k]; ++i) h->sep_npk[dir][k] += poff[(size_t)(h->sep_step0[dir][k] + i)].second;
        }
        std::vector<SepStep<double>> s64;
        std::vector<SepStep<float>> s32;
        for (size_t i = 0; i < all[dir].size(); ++i) {
            const HostStep &s = all[dir][i];
            s64.push_back(SepStep<double>{s.n_out, s.n_in, d_idx + off[i].first, d_col + off[i].second,
                                          d_v64 + off[i].second, d_p64 + poff[i].first, poff[i].second});
            s32.push_back(SepStep<float>{s.n_out, s.n_in, d_idx + off[i].first, d_col + off[i].second,
                                         d_v32 + off[i].second, d_p32 + poff[i].first, poff[i].second});
        }
        TB_TRY(dalloc(h, &h->sep64[dir], (int64_t)s64.size()));
        TB_TRY(dalloc(h, &h->sep32[dir], (int64_t)s32.size()));
        TB_CK(cudaMemcpy(h->sep64[dir], s64.data(), s64.size() * sizeof(s64[0]), cudaMemcpyHostToDevice));
        TB_CK(cudaMemcpy(h->sep32[dir], s32.data(), s32.size() * sizeof(s32[0]), cudaMemcpyHostToDevice));
    }
    (void)L;
    return TB_OK;
}

// Largest mode intermediates (entries per RHS) of all level passes, for the
// intermediates after the even and the odd launches of a pass (the two
// ping-pong buffers), each pass in its per-mode launch order.
static void mode_sizes(const tb_plan *h, int64_t mm[2]) {
    const int d = h->d;
    mm[0] = mm[1] = 0;
    const Pass passes[4] = {Pass::LeafIn, Pass::Split, Pass::Gather, Pass::LeafOut};
    for (int side = 0; side < 2; ++side)
        for (Pass p : passes) {
            const bool leaf = p == Pass::LeafIn || p == Pass::LeafOut;
            for (int l = leaf ? 0 : 1; l <= (leaf ? 0 : h->Lc); ++l) {
                int m[TB_MAX_D], o[TB_MAX_D], ord[TB_MAX_D], cur[TB_MAX_D];
                pass_dims(h, p, side, l, m, o);
                mode_order_permode(h, p, side, l, ord);
                for (int k = 0; k < d; ++k) cur[k] = m[k];
                for (int st = 0; st + 1 < d; ++st) {
                    cur[ord[st]] = o[ord[st]];
                    int64_t sz = h->P;
                    for (int k = 0; k < d; ++k) sz *= cur[k];
                    mm[st & 1] = std::max(mm[st & 1], sz);
                }
            }
        }
}

// Whether the cores can be regenerated inside the contraction with exact
// integer distances / phases (tb_options.core_mode = 2, see CoreRegen), and
// the parameters.  Grids must be uniform: coordinate i = x0 + i h up to 1e-12.
static void detect_regen(tb_plan *h, const tb_grids *g) {
    CoreRegen r;
    std::memset(&r, 0, sizeof(r));
    h->rg = r;
    if (h->separable || h->d > TB_MAX_D) return;
    const int d = h->d;
    auto uniform = [](const double *v, int64_t n, double &x0, double &hh) {
        x0 = v[0];
        hh = n > 1 ? v[1] - v[0] : 1.0;
        if (!(hh > 0)) return false;
        for (int64_t i = 0; i < n; ++i)
            if (std::fabs(v[i] - (x0 + (double)i * hh)) > 1e-12 * std::max(1.0, std::fabs(v[i]))) return false;
        return true;
    };
    auto integer = [](double v, int &out) {
        const double q = std::nearbyint(v);
        if (std::fabs(v - q) > 1e-9 || std::fabs(q) > 1e6) return false;
        out = (int)q;
        return true;
    };
    if (h->ks.kind == TB_KERNEL_HELMHOLTZ) {
        double hh = -1.0, dmax = 0.0;
        for (int k = 0; k < d; ++k) {
            double x0, hx, y0, hy;
            if (!uniform(g->x[k], h->n[k], x0, hx) || !uniform(g->y[k], h->n[k], y0, hy)) return;
            if (std::fabs(hx - hy) > 1e-12 * hx) return;
            if (hh < 0) hh = hx;
            if (std::fabs(hx - hh) > 1e-12 * hh) return;
            if (!integer((y0 - x0) / hh, r.off[k])) return;
            const double ext = (double)(h->n[k] - 1) + std::fabs((double)r.off[k]);
            dmax += ext * ext;
        }
        int hp = 0;
        if (!integer(std::sqrt(h->ks.p[1]) / hh, hp)) return;
        r.hp2 = hp * hp;
        if (dmax + r.hp2 >= 16777216.0) return;   // D must be exact in FP32
        const double cyc = h->ks.p[2] * hh;         // cycles per unit of sqrt(D)
        r.cyc_hi = (float)cyc;
        r.cyc_lo = (float)(cyc - (double)r.cyc_hi);
        r.inv_h = (float)(1.0 / hh);
    } else if (h->ks.kind == TB_KERNEL_RADON) {
        int nn = 0;
        for (int k = 0; k < d; ++k) {
            double x0, hx, y0, hy;
            if (!uniform(g->x[k], h->n[k], x0, hx) || !uniform(g->y[k], h->n[k], y0, hy)) return;
            int nk = 0;
            if (x0 != 0.0 || !integer(1.0 / hx, nk) || std::fabs(hy - 1.0) > 1e-12) return;
            if (nn == 0) nn = nk;
            if (nk != nn || !integer(y0, r.xi0[k])) return;
            r.xs[k] = h->xs[k];
        }
        r.n = nn;
        r.ra = h->ks.p[0];
        r.rb = h->ks.p[1];
    } else {
        return;
    }
    const int Lc = h->Lc;
    for (int k = 0; k < d; ++k) {
        r.tskel[k] = h->tgt[Lc].skel[k];
        r.sskel[k] = h->src[Lc].skel[k];
        r.tcap[k] = h->tgt[Lc].cap[k];
        r.scap[k] = h->src[Lc].cap[k];
    }
    r.nF = ipow2(d * Lc);
    r.kind = h->ks.kind;
    h->rg = r;
}

static tb_status build_impl(tb_plan *h, const tb_grids *grids) {
    const int d = h->d;
    TB_TRY(dalloc(h, &h->d_err, 1));
    TB_CK(cudaMemset(h->d_err, 0, sizeof(int)));
    for (int k = 0; k < d; ++k) {
        const int64_t nk = h->n[k];
        TB_TRY(dalloc(h, &h->xs[k], nk));
        TB_TRY(dalloc(h, &h->ys[k], nk));
        TB_TRY(dalloc(h, &h->perm[k], nk));
        TB_CK(cudaMemcpy(h->xs[k], grids->x[k], nk * sizeof(double), cudaMemcpyHostToDevice));
        TB_CK(cudaMemcpy(h->ys[k], grids->y[k], nk * sizeof(double), cudaMemcpyHostToDevice));
        std::vector<int> pm((size_t)nk);
        const int bits = ilog2(nk);
        for (int64_t p = 0; p < nk; ++p) {
            int64_t q = p;
            if (h->order == TB_ORDER_BITREV) {
                q = 0;
                for (int b = 0; b < bits; ++b) q |= ((p >> b) & 1) << (bits - 1 - b);
            }
            pm[(size_t)p] = (int)q;
        }
        TB_CK(cudaMemcpy(h->perm[k], pm.data(), pm.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    TB_TRY(build_side(h, 0));
    TB_TRY(build_side(h, 1));
    TB_TRY(build_cores(h));
    detect_regen(h, grids);
    // apply precisions of the factors
    const bool want32 = h->precisions & ((1u << TB_PREC_C64) | (1u << TB_PREC_C64_SPLITBF16));
    for (int side = 0; side < 2; ++side) {
        SideLevel *lv = side == 0 ? h->src : h->tgt;
        for (int l = 0; l <= h->Lc; ++l)
            for (int k = 0; k < d; ++k) {
                const int64_t cnt = lv[l].count[k] * lv[l].R[k] * lv[l].cin[k];
                if (want32) {
                    TB_TRY(dalloc(h, &lv[l].fac32[k], cnt));
                    TB_CK(launch_to_c64(lv[l].fac64[k], lv[l].fac32[k], cnt, 0));
                }
            }
    }
    int64_t lm = 0;
    for (int l = 0; l <= h->Lc; ++l) {
        lm = std::max(lm, h->P * prod_tile(h->src[l], d));
        lm = std::max(lm, h->P * prod_tile(h->tgt[l], d));
    }
    h->level_max = lm;
    mode_sizes(h, h->mode_max);
    if (h->separable) {
        TB_TRY(build_sep_steps(h));
        int64_t N = 1;
        for (int k = 0; k < d; ++k) N *= h->n[k];
        h->level_max = std::max(h->level_max, N);   // the per-mode passes ping-pong full tensors
    }
    TB_CK(cudaDeviceSynchronize());
    return TB_OK;
}

extern "C" tb_status tb_build_ex(const tb_kernel *kernel, int d, const int64_t *n, const tb_grids *grids,
                                 double tol, const tb_options *opt_in, tb_handle *out) {
    if (!out) return fail(TB_EINVAL, "out handle pointer is NULL");
    *out = nullptr;
    if (!kernel || !n || !grids) return fail(TB_EINVAL, "kernel, n and grids must be non-NULL");
    if (kernel->kind < TB_KERNEL_FOURIER || kernel->kind > TB_KERNEL_RADON_ANISO)
        return fail(TB_EINVAL, "unknown kernel kind " + std::to_string(kernel->kind));
    if (d < 1 || d > TB_MAX_D) return fail(TB_EINVAL, "d must be in [1, " + std::to_string(TB_MAX_D) + "]");
    if (kernel->kind == TB_KERNEL_RADON_ANISO && d != 2)
        return fail(TB_EINVAL, "the anisotropic Radon kernel is defined for d = 2");
    if (kernel->kind == TB_KERNEL_HELMHOLTZ && !(kernel->params[1] >= 0.0))
        return fail(TB_EINVAL, "Helmholtz offset h = params[1] must be >= 0");
    if (!(tol > 0.0 && tol < 1.0)) return fail(TB_EINVAL, "tol must be in (0, 1)");
    tb_options opt;
    tb_options_default(&opt);
    if (opt_in) opt = *opt_in;
    for (int k = 0; k < d; ++k) {
        if (!pow2(n[k]) || n[k] < 2) return fail(TB_EINVAL, "n[k] must be a power of two >= 2");
        if (n[k] > (1 << 24)) return fail(TB_EINVAL, "n[k] too large");
        if (!grids->x[k] || !grids->y[k]) return fail(TB_EINVAL, "grid pointer is NULL");
    }
    if (opt.proxy_rows <= 0) opt.proxy_rows = 1024;
    if (!pow2(opt.proxy_rows) || opt.proxy_rows > (1 << 20)) return fail(TB_EINVAL, "proxy_rows must be a power of two");
    if (opt.rank_max <= 0) opt.rank_max = 32;
    if (opt.rank_max > id_max_columns() / 2) return fail(TB_EINVAL, "rank_max must be <= 32");
    // coincident source/target points make the Helmholtz kernel singular
    if (kernel->kind == TB_KERNEL_HELMHOLTZ && kernel->params[1] == 0.0) {
        bool all_axes_meet = true;
        for (int k = 0; k < d && all_axes_meet; ++k) {
            std::vector<double> xa(grids->x[k], grids->x[k] + n[k]), ya(grids->y[k], grids->y[k] + n[k]);
            std::sort(xa.begin(), xa.end());
            std::sort(ya.begin(), ya.end());
            std::vector<double> both;
            std::set_intersection(xa.begin(), xa.end(), ya.begin(), ya.end(), std::back_inserter(both));
            all_axes_meet = !both.empty();
        }
        if (all_axes_meet) return fail(TB_EINVAL, "Helmholtz kernel: a source point coincides with a target point");
    }
    // levels: n_k = C_b,k 2^L with L even
    int L = opt.L;
    int64_t nmin = n[0];
    for (int k = 1; k < d; ++k) nmin = std::min(nmin, n[k]);
    if (L < 0) {
        // leaves of 4 points, or 16 for large 3-D grids, where larger leaves
        // shrink the mid-level cores (their count grows as (n / C_b)^d)
        const int64_t cbmin = (d == 3 && nmin >= 256) ? 16 : 4;
        L = 0;
        while ((nmin >> (L + 2)) >= cbmin) L += 2;
    }
    if (L % 2 != 0 || L < 0 || L >= TB_MAX_LEVELS || (nmin >> L) < 1)
        return fail(TB_EINVAL, "L must be even with n_k / 2^L >= 1");
    if (opt.sep_schedule < 0 || opt.sep_schedule > 6) return fail(TB_EINVAL, "sep_schedule must be in [0, 6]");
    if (opt.level_schedule < 0 || opt.level_schedule > 3) return fail(TB_EINVAL, "level_schedule must be in [0, 3]");
    if (opt.core_mode < 0 || opt.core_mode > 2) return fail(TB_EINVAL, "core_mode must be in [0, 2]");
    if (opt.mode_slices != 0 && opt.mode_slices != 1 && opt.mode_slices != 2 && opt.mode_slices != 4)
        return fail(TB_EINVAL, "mode_slices must be 0, 1, 2 or 4");
    int dev = opt.device;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "no CUDA device"); }
    }
    if (cudaSetDevice(dev) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice failed"); }

    auto t0 = std::chrono::steady_clock::now();
    tb_plan *h = new tb_plan();
    h->d = d;
    h->L = L;
    h->Lc = L / 2;
    h->device = dev;
    h->tol = tol;
    h->order = opt.order == TB_ORDER_AUTO ? (kernel->kind == TB_KERNEL_FOURIER ? TB_ORDER_BITREV : TB_ORDER_NATURAL)
                                          : opt.order;
    h->separable = opt.separable < 0 ? (kernel->kind == TB_KERNEL_FOURIER) : opt.separable;
    if (h->separable && kernel->kind != TB_KERNEL_FOURIER) {
        delete h;
        return fail(TB_EINVAL, "separable factors need a kernel that is a product over modes (FOURIER)");
    }
    h->precisions = opt.precisions ? opt.precisions : TB_PRECISIONS_BUILT;
    if (h->precisions & ~TB_PRECISIONS_BUILT) {
        delete h;
        return fail(TB_EUNSUPPORTED, "requested apply precision is not built into this library");
    }
    h->use_graphs = opt.use_graphs;
    h->autotune = opt.autotune;
    h->sep_choice = opt.sep_schedule;
    h->level_choice = opt.level_schedule;
    h->core_mode = opt.core_mode;
    h->mode_slices = opt.mode_slices;
    h->proxy_rows = opt.proxy_rows;
    h->rank_max = opt.rank_max;
    h->seed = opt.seed;
    h->rank_min = 1 << 30;
    h->ks.kind = kernel->kind;
    for (int i = 0; i < 4; ++i) h->ks.p[i] = kernel->params[i];
    if (kernel->kind == TB_KERNEL_HELMHOLTZ) {
        h->ks.p[1] = kernel->params[1] * kernel->params[1];
        h->ks.p[2] = kernel->params[0] / (2.0 * M_PI);
    }
    for (int k = 0; k < d; ++k) {
        h->n[k] = n[k];
        h->cb[k] = n[k] >> L;
    }
    tb_status st = build_impl(h, grids);
    if (st != TB_OK) {
        std::string msg = g_err;
        tb_free(h);
        g_err = msg;
        return st;
    }
    h->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return TB_OK;
}

extern "C" tb_status tb_query(tb_handle h, tb_info *info) {
    if (!h || !info) return fail(TB_EINVAL, "handle and info must be non-NULL");
    std::memset(info, 0, sizeof(*info));
    info->d = h->d;
    info->L = h->L;
    info->Lc = h->Lc;
    info->order = h->order;
    info->separable = h->separable;
    for (int k = 0; k < h->d; ++k) {
        info->n[k] = h->n[k];
        info->cb[k] = h->cb[k];
    }
    int64_t fe = 0;
    for (int l = 0; l <= h->Lc; ++l)
        for (int k = 0; k < h->d; ++k) {
            info->rank_src[l][k] = h->src[l].R[k];
            info->rank_tgt[l][k] = h->tgt[l].R[k];
            fe += h->src[l].count[k] * h->src[l].R[k] * h->src[l].cin[k];
            fe += h->tgt[l].count[k] * h->tgt[l].R[k] * h->tgt[l].cin[k];
        }
    info->rank_min = h->rank_min;
    info->rank_max = h->rank_max_seen;
    info->num_ids = h->num_ids;
    info->core_entries = h->core_entries;
    info->factor_entries = fe;
    info->level_entries_max = h->level_max;
    info->device_bytes = h->device_bytes + (int64_t)h->ws.bytes * 2 + (int64_t)(h->ws.mbytes[0] + h->ws.mbytes[1]) +
                         (int64_t)(h->ws.cout_bytes[0] + h->ws.cout_bytes[1]);
    info->build_seconds = h->build_seconds;
    if (h->separable) {
        int64_t ms = h->P, mt = h->P;
        for (int k = 0; k < h->d; ++k) {
            ms *= h->src[h->Lc].R[k];
            mt *= h->tgt[h->Lc].R[k];
        }
        info->mid_src_entries = ms;
        info->mid_tgt_entries = mt;
    } else {
        info->mid_src_entries = h->core_in_entries;
        info->mid_tgt_entries = h->core_out_entries;
    }
    return TB_OK;
}

// --------------------------------------------------------------------- apply
namespace {

template <class R>
TileBuf<R> tilebuf(const tb_plan *h, int side, int l, void *p) {
    const SideLevel &S = side == 0 ? h->src[l] : h->tgt[l];
    TileBuf<R> t;
    t.p = static_cast<cx<R> *>(p);
    t.tsize = 1;
    for (int k = 0; k < TB_MAX_D; ++k) t.R[k] = k < h->d ? S.R[k] : 1;
    for (int k = 0; k < h->d; ++k) t.tsize *= S.R[k];
    t.lgseg = h->Lc - l;
    t.nM = ipow2(h->d * l);
    t.layout = side;
    return t;
}

template <class R>
const cx<R> *facptr(const SideLevel &S, int k);
template <>
const cx<double> *facptr<double>(const SideLevel &S, int k) { return S.fac64[k]; }
template <>
const cx<float> *facptr<float>(const SideLevel &S, int k) { return S.fac32[k]; }

template <class R>
FacRef<R> facref(const tb_plan *h, int side, int l) {
    const SideLevel &S = side == 0 ? h->src[l] : h->tgt[l];
    FacRef<R> f;
    std::memset(&f, 0, sizeof(f));
    for (int k = 0; k < h->d; ++k) {
        f.A[k] = facptr<R>(S, k);
        f.rank[k] = S.rank[k];
        f.rows[k] = S.R[k];
        f.cols[k] = S.cin[k];
    }
    f.l = l;
    f.lgseg = h->Lc - l;
    f.nM = ipow2(h->d * l);
    f.separable = h->separable;
    return f;
}

// Largest RHS chunk whose shared-memory plan fits `limit` bytes (at least 1).
template <class R>
tb_status pick_chunk(int d, const int *m, const int *o, int64_t nv, int64_t &nvc, size_t &smem, int &offX,
                     int &offB0, int &offB1, int &offY, int &offA, bool no_x = false, bool no_y = false) {
    auto plan = [&](int64_t c) {
        ChainSmem s = chain_smem(d, m, o, c);
        if (no_x) s.x = 0;   // the first pass reads global memory directly
        if (no_y) s.y = 0;   // the last pass writes global memory directly
        return s;
    };
    ChainSmem s1 = plan(1);
    const int64_t per = s1.x + s1.b0 + s1.b1 + s1.y;
    const int64_t es = sizeof(cx<R>);
    const int64_t limit = 100 * 1024;
    int64_t c = (limit / es - s1.a) / std::max<int64_t>(per, 1);
    if (c < 1) c = 1;
    if (c > nv) c = nv;
    nvc = c;
    ChainSmem s = plan(nvc);
    // buffers start on 32-byte boundaries (vector loads in the mode products)
    auto up4 = [](int64_t v) { return (v + 3) & ~(int64_t)3; };
    s.x = up4(s.x);
    s.b0 = up4(s.b0);
    s.b1 = up4(s.b1);
    s.y = up4(s.y);
    offX = 0;
    offB0 = (int)s.x;
    offB1 = (int)(s.x + s.b0);
    offY = (int)(s.x + s.b0 + s.b1);
    offA = (int)(s.x + s.b0 + s.b1 + s.y);
    smem = (size_t)(s.x + s.b0 + s.b1 + s.y + s.a) * es;
    if (smem > g_smem_optin)
        return fail(TB_EUNSUPPORTED, "tile of " + std::to_string(smem) + " bytes exceeds shared memory (" +
                                         std::to_string(g_smem_optin) + ")");
    return TB_OK;
}

// Output rows per register tile of a mode launch: the instantiated values
// (even, up to 16, and 18, 20, 24), and the built-in rule: the fewest chunks
// of at most 24 rows, split evenly.
bool mode_ob_valid(int ob) { return ob >= 2 && !(ob & 1) && (ob <= 20 || ob == 24); }

// Threads per block of a mode launch: `want` if valid (32, 64 or 128, and at
// least `minbt`), else the fewest that cover `cols` columns (at least minbt).
int mode_bt(int want, int64_t cols, int minbt) {
    const int lo = minbt <= 32 ? 32 : 64;
    if ((want == 32 || want == 64 || want == 128) && want >= lo) return want;
    const int64_t per = (int64_t)mode_cols_per_thread();
    int bt = 128;
    if (cols <= 32 * per) bt = 32;
    else if (cols <= 64 * per) bt = 64;
    return bt < lo ? lo : bt;
}
int mode_ob_rule(int o) {
    const int nch = (o + 23) / 24;
    int ob = (o + nch - 1) / nch;
    ob += ob & 1;
    if (ob == 22) ob = 24;
    return ob;
}


// One level pass as d mode-product launches (tb_mode.cu).  T holds the two
// ping-pong buffers of the mode intermediates.
template <class R>
tb_status level_pass(const tb_plan *h, Pass pass, bool conj, int side, int l, const void *in, void *out, int64_t nv,
                     cudaStream_t st, void *const *T, int only_k = -1, int ob_set = 0, int waves_set = 0,
                     int64_t f0 = 0, int64_t f1 = -1, int rank_set = -1, int bt_set = 0, int *bt_used = nullptr,
                     int sub_set = 0) {
    const int d = h->d, Lc = h->Lc;
    const bool leaf = pass == Pass::LeafIn || pass == Pass::LeafOut;
    ModeArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.f0 = f0;
    a.f1 = f1 < 0 ? ipow2(d * Lc) : f1;
    a.d = d;
    a.Lc = Lc;
    a.pass = (int)pass;
    a.nv = nv;
    a.nF = ipow2(d * Lc);
    a.trans = (pass == Pass::LeafOut || pass == Pass::Gather) ? 1 : 0;
    a.conj = conj ? 1 : 0;
    int m[TB_MAX_D], o[TB_MAX_D];
    const SideLevel *S = side == 0 ? h->src : h->tgt;
    for (int k = 0; k < d; ++k) {
        a.cb[k] = (int)h->cb[k];
        a.nmid[k] = h->n[k] >> Lc;
        a.perm[k] = h->perm[k];
    }
    int64_t gs = 1;
    for (int k = d - 1; k >= 0; --k) {
        a.user.gstride[k] = gs;
        gs *= h->n[k];
    }
    switch (pass) {
        case Pass::LeafIn:
            a.user.p = (cx<R> *)in;
            a.lout = tilebuf<R>(h, side, 0, out);
            a.fac = facref<R>(h, side, 0);
            for (int k = 0; k < d; ++k) { m[k] = (int)h->cb[k]; o[k] = S[0].R[k]; }
            break;
        case Pass::LeafOut:
            a.user.p = (cx<R> *)out;
            a.lin = tilebuf<R>(h, side, 0, (void *)in);
            a.fac = facref<R>(h, side, 0);
            for (int k = 0; k < d; ++k) { m[k] = S[0].R[k]; o[k] = (int)h->cb[k]; }
            break;
        case Pass::Split:
            a.lin = tilebuf<R>(h, side, l - 1, (void *)in);
            a.lout = tilebuf<R>(h, side, l, out);
            a.fac = facref<R>(h, side, l);
            for (int k = 0; k < d; ++k) { m[k] = 2 * S[l - 1].R[k]; o[k] = S[l].R[k]; a.Rp[k] = S[l - 1].R[k]; }
            break;
        case Pass::Gather:
            a.lin = tilebuf<R>(h, side, l, (void *)in);
            a.lout = tilebuf<R>(h, side, l - 1, out);
            a.fac = facref<R>(h, side, l);
            for (int k = 0; k < d; ++k) { m[k] = S[l].R[k]; o[k] = 2 * S[l - 1].R[k]; a.Rp[k] = S[l - 1].R[k]; }
            break;
    }
    a.lvl = leaf ? 0 : l;
    a.lgs = Lc - a.lvl;
    const size_t es = sizeof(cx<R>);
    int64_t gtab = 0;
    for (int k = 0; k < d; ++k) gtab += h->cb[k];
    const tb::ModeTune *tune = h->tune[std::is_same<R, double>::value ? 1 : 0][side][(int)pass][leaf ? 0 : l];
    int ord[TB_MAX_D];
    mode_order_permode(h, pass, side, l, ord);
    int cur[TB_MAX_D];
    for (int i = 0; i < d; ++i) cur[i] = m[i];
    for (int step = 0; step < d; ++step) {
        const int k = ord[step];
        if (only_k >= 0 && k != only_k) {
            cur[k] = o[k];
            continue;
        }
        a.k = k;
        a.m = m[k];
        a.o = o[k];
        int64_t pre = 1, post = nv, usz_in = nv, usz_out = nv;
        for (int i = 0; i < k; ++i) pre *= cur[i];
        for (int i = k + 1; i < d; ++i) post *= cur[i];
        for (int i = 0; i < d; ++i) {
            usz_in *= cur[i];
            usz_out *= i == k ? o[i] : cur[i];
        }
        cur[k] = o[k];
        a.pre = pre;
        a.post = post;
        a.cols = pre * post;
        int ink = MK_UNIT, outk = MK_UNIT;
        a.in_tile = 0;
        a.out_tile = 0;
        a.tin = nullptr;
        a.tout = nullptr;
        if (step == 0) {
            if (pass == Pass::LeafIn) ink = MK_USER;
            else if (pass == Pass::Split) ink = MK_PARENTS;
            else a.in_tile = 1;
        } else {
            a.tin = (const cx<R> *)T[(step - 1) & 1];
            a.in_usize = usz_in;
        }
        if (step == d - 1) {
            if (pass == Pass::LeafOut) outk = MK_USER;
            else if (pass == Pass::Gather) outk = MK_PARENTS;
            else a.out_tile = 1;
        } else {
            a.tout = (cx<R> *)T[step & 1];
            a.out_usize = usz_out;
        }
        const bool group = ink == MK_PARENTS || outk == MK_PARENTS;
        a.nblk = (!leaf && group) ? (h->P >> d) : h->P;
        if (a.cols >= ((int64_t)1 << 31) || usz_in >= ((int64_t)1 << 31) || usz_out >= ((int64_t)1 << 31))
            return fail(TB_EUNSUPPORTED, "a level tile with its RHS exceeds 2^31 entries (reduce nv)");
        // threads per column slice: the tuner's choice, else the fewest (32, 64
        // or 128) that give one thread to each of a unit's columns; a group
        // launch sets up its 2^d children with one thread each.  sub slices
        // (1, 2 or 4; at most 128 threads) share each column's work.
        const int cw = mode_bt(bt_set ? bt_set : tune[k].bt, a.cols, group ? (1 << d) : 1);
        if (bt_used) *bt_used = cw;
        int sub = sub_set ? sub_set : (h->mode_slices ? h->mode_slices : (tune[k].sub > 0 ? tune[k].sub : 1));
        if ((sub != 1 && sub != 2 && sub != 4) || sizeof(R) != 4) sub = 1;   // slices: complex64 only
        while (sub > 1 && sub * cw > 128) sub >>= 1;
        a.sub = sub;
        a.bt = sub * cw;
        const int cpb = cw * mode_cols_per_thread();
        a.ncb = (a.cols + cpb - 1) / cpb;
        // enough blocks for a few waves of four resident blocks per SM
        const int waves = waves_set ? waves_set : (tune[k].waves > 0 ? tune[k].waves : TB_MODE_WAVES);
        const int64_t target = waves * (int64_t)g_num_sms;
        a.gsplit = std::min<int64_t>(a.ncb, std::max<int64_t>(1, (target + a.nblk - 1) / a.nblk));
        int ob = ob_set ? ob_set : tune[k].ob;
        if (!mode_ob_valid(ob)) ob = mode_ob_rule(o[k]);
        a.lda = (o[k] + ob - 1) / ob * ob;
        a.fsz = m[k] * a.lda;
        const int nfac = group ? (1 << d) : 1;
        a.smem = (size_t)nfac * a.fsz * es +
                 ((ink == MK_USER || outk == MK_USER) ? (size_t)gtab * sizeof(int) : 0);
        if (a.smem > g_smem_optin)
            return fail(TB_EUNSUPPORTED, "factor blocks of " + std::to_string(a.smem) +
                                             " bytes exceed shared memory");
        // rank-bounded products: the tuner's choice, else on for Split / Gather
        // (their blocks' ranks spread below the padded length), off for the leaves
        const int rk = rank_set >= 0 ? rank_set : (tune[k].rank >= 0 ? tune[k].rank : (leaf ? 0 : 1));
        TB_CK(launch_mode<R>(ink, outk, ob, rk, a, st));
    }
    return TB_OK;
}




// Whether a level pass runs fused: tb_options.level_schedule, then the tuner's
// per-pass choice (the faster of the two forms), then the built-in rule
// (per-mode launches).
bool level_fused_wanted(const tb_plan *h, Pass pass, int side, int l) {
    if (h->level_choice == 1 || h->level_choice == 3) return false;
    if (h->level_choice == 2) return true;
    const bool leaf = pass == Pass::LeafIn || pass == Pass::LeafOut;
    return h->ltune[side][(int)pass][leaf ? 0 : l].mode == 2;
}

// Whether a level pass runs on the tensor cores (split-BF16 applies only):
// tb_options.level_schedule = 3, else the tuner's per-pass choice (the
// built-in rule keeps the per-mode launches, measured faster at the
// benchmark ranks).
bool level_tc_wanted(const tb_plan *h, Pass pass, int side, int l, int precision) {
    if (precision != TB_PREC_C64_SPLITBF16) return false;
    if (h->level_choice == 3) return true;
    if (h->level_choice != 0) return false;
    const bool leaf = pass == Pass::LeafIn || pass == Pass::LeafOut;
    return h->ltune[side][(int)pass][leaf ? 0 : l].mode == 3;
}

// One level pass as a single fused persistent launch (k_level, complex64),
// its intermediates in `scratch` (scratch_bytes long).  done = false (and
// nothing launched) when the pass does not fit the fused kernel: d > 3, too
// little scratch or shared memory.  dry = true only plans.
// The pass-generic part of a fused level launch's arguments: dims, item
// decomposition, tiles, factors and the user tensor.
void level_args_common(const tb_plan *h, Pass pass, bool conj, int side, int l, const void *in, void *out,
                       int64_t nv, LevelArgs &a) {
    const int d = h->d, Lc = h->Lc;
    const bool leaf = pass == Pass::LeafIn || pass == Pass::LeafOut;
    std::memset(&a, 0, sizeof(a));
    a.d = d;
    a.Lc = Lc;
    a.pass = (int)pass;
    a.nv = nv;
    a.nF = ipow2(d * Lc);
    a.trans = (pass == Pass::LeafOut || pass == Pass::Gather) ? 1 : 0;
    a.conj = conj ? 1 : 0;
    int m[TB_MAX_D], o[TB_MAX_D];
    pass_dims(h, pass, side, l, m, o);
    const SideLevel *S = side == 0 ? h->src : h->tgt;
    for (int k = 0; k < d; ++k) {
        a.m[k] = m[k];
        a.o[k] = o[k];
        a.cb[k] = (int)h->cb[k];
        a.nmid[k] = h->n[k] >> Lc;
        a.perm[k] = h->perm[k];
        if (!leaf) a.Rp[k] = S[l - 1].R[k];
    }
    int64_t gs = 1;
    for (int k = d - 1; k >= 0; --k) {
        a.user.gstride[k] = gs;
        gs *= h->n[k];
    }
    switch (pass) {
        case Pass::LeafIn:
            a.user.p = (cx<float> *)in;
            a.lout = tilebuf<float>(h, side, 0, out);
            a.fac = facref<float>(h, side, 0);
            break;
        case Pass::LeafOut:
            a.user.p = (cx<float> *)out;
            a.lin = tilebuf<float>(h, side, 0, (void *)in);
            a.fac = facref<float>(h, side, 0);
            break;
        case Pass::Split:
            a.lin = tilebuf<float>(h, side, l - 1, (void *)in);
            a.lout = tilebuf<float>(h, side, l, out);
            a.fac = facref<float>(h, side, l);
            break;
        case Pass::Gather:
            a.lin = tilebuf<float>(h, side, l, (void *)in);
            a.lout = tilebuf<float>(h, side, l - 1, out);
            a.fac = facref<float>(h, side, l);
            break;
    }
    a.lvl = leaf ? 0 : l;
    a.lgs = Lc - a.lvl;
    for (int k = 0; k < d; ++k) a.lcb[k] = ilog2(h->cb[k]);
}

tb_status level_pass_fused(const tb_plan *h, Pass pass, bool conj, int side, int l, const void *in, void *out,
                           int64_t nv, cudaStream_t st, void *scratch, size_t scratch_bytes, bool &done,
                           bool dry = false, int vc_set = 0, int cps_set = 0, int obmax_set = 0) {
    done = false;
    const int d = h->d;
    if (d > 3 || (1 << d) > level_max_children()) return TB_OK;
    const bool leaf = pass == Pass::LeafIn || pass == Pass::LeafOut;
    LevelArgs a;
    level_args_common(h, pass, conj, side, l, in, out, nv, a);
    int m[TB_MAX_D], o[TB_MAX_D];
    pass_dims(h, pass, side, l, m, o);
    best_order(d, m, o, a.order);
    const tb::LevelTune &tn = h->ltune[side][(int)pass][leaf ? 0 : l];
    // output rows per register chunk, one value for the launch: the even value
    // in [4, 16] with the fewest padded multiply-adds (ties: fewer chunks)
    int OB = obmax_set ? obmax_set : tn.obmax;
    if (!level_ob_valid(OB)) {
        double best = -1.0;
        int cur[TB_MAX_D];
        double stepc[TB_MAX_D];
        for (int k = 0; k < d; ++k) cur[k] = m[k];
        for (int i = 0; i < d; ++i) {
            const int k = a.order[i];
            double t = (double)m[k];
            for (int j = 0; j < d; ++j)
                if (j != k) t *= cur[j];
            stepc[k] = t;   // multiply-adds per output row of mode k
            cur[k] = o[k];
        }
        for (int ob = 12; ob >= 4; ob -= 2) {   // 14 and 16 spill registers: tuner only
            double c = 0.0;
            for (int k = 0; k < d; ++k) c += stepc[k] * ((o[k] + ob - 1) / ob * ob);
            if (best < 0.0 || c < best * (1.0 - 1e-9)) {
                best = c;
                OB = ob;
            }
        }
    }
    for (int k = 0; k < d; ++k) a.lda[k] = (o[k] + OB - 1) / OB * OB;
    int off = 0;
    for (int k = 0; k < d; ++k) {
        a.fac_off[k] = off;
        off += (3 * m[k] * a.lda[k] + 3) / 4 * 4;   // planes start on 16-byte boundaries
    }
    a.fac_floats = off;
    for (int i = 0; i < d; ++i) a.ob[i] = OB;
    int64_t gtab = 0;
    for (int k = 0; k < d; ++k) gtab += h->cb[k];
    // shared memory: factors, tree-order tables, two intermediate buffers and
    // (Gather) the combined parent tile, for vc right-hand sides per item
    int64_t inter[2] = {0, 0};   // entries per RHS of the even / odd step outputs
    {
        int cur[TB_MAX_D];
        for (int k = 0; k < d; ++k) cur[k] = m[k];
        for (int i = 0; i + 1 < d; ++i) {
            cur[a.order[i]] = o[a.order[i]];
            int64_t t = 1;
            for (int k = 0; k < d; ++k) t *= cur[k];
            inter[i & 1] = std::max(inter[i & 1], t);
        }
    }
    int64_t accn = 0;
    if (pass == Pass::Gather) {
        accn = 1;
        for (int k = 0; k < d; ++k) accn *= o[k];
    }
    auto up16 = [](size_t b) { return (b + 15) / 16 * 16; };
    const size_t gstr_off = up16((size_t)a.fac_floats * sizeof(float) + (leaf ? (size_t)gtab * sizeof(int) : 0));
    const size_t fixed = up16(gstr_off + (leaf ? (size_t)gtab * sizeof(int64_t) : 0));
    a.off_gstr = gstr_off;
    for (int k = 0; k < d; ++k) a.lcb[k] = ilog2(h->cb[k]);
    int64_t inn = 1;
    for (int k = 0; k < d; ++k) inn *= m[k];
    auto smem_for = [&](int v) {
        return fixed + up16((size_t)inn * v * sizeof(float2)) + up16((size_t)inter[0] * v * sizeof(float2)) +
               up16((size_t)inter[1] * v * sizeof(float2)) + up16((size_t)accn * v * sizeof(float2));
    };
    // two resident blocks per SM by default (the static shared arrays take ~1 KB each)
    const size_t budget = std::min<size_t>(g_smem_optin, 110 * 1024);
    int vc = vc_set ? vc_set : tn.vc;
    if (vc <= 0) {
        vc = 4;
        while (vc > 1 && smem_for(vc) > budget) vc /= 2;
    }
    vc = (int)std::max<int64_t>(1, std::min<int64_t>(vc, nv));
    while (vc & (vc - 1)) --vc;   // a power of two
    a.smem = smem_for(vc);
    if (a.smem > g_smem_optin) return TB_OK;
    a.off_in = fixed;
    a.off_s0 = a.off_in + up16((size_t)inn * vc * sizeof(float2));
    a.off_s1 = a.off_s0 + up16((size_t)inter[0] * vc * sizeof(float2));
    a.off_acc = a.off_s1 + up16((size_t)inter[1] * vc * sizeof(float2));
    a.vc = vc;
    a.lvc = ilog2(vc);
    a.nq = (int)((nv + vc - 1) / vc);
    const int64_t nunits = leaf ? h->P : (h->P >> d);
    a.nitems = nunits * a.nq;
    const int cps = cps_set ? cps_set : (tn.cps ? tn.cps : 2);
    const int64_t blocks = std::min<int64_t>(a.nitems, (int64_t)cps * g_num_sms);
    (void)scratch;
    (void)scratch_bytes;
    done = true;
    if (dry) return TB_OK;
    TB_CK(launch_level(a, OB, (int)blocks, st));
    return TB_OK;
}

// ------------------------------------------- level passes on the tensor cores
// Plan of a level pass for k_level_tc with vc RHS per work item and mode order
// ord: per-step operand shapes, shared-memory layout and accumulator columns.
// Bit i of rowbits swaps the order of step i's two other modes (d = 3) in its
// operand rows; the cost counts the shared-memory wavefronts of one warp's
// accumulator stores into the next operand (simulated here).
// false when it does not fit (shared memory, tensor memory, MMA N <= 256).
bool plan_level_tc(const tb_plan *h, Pass pass, int vc, const int *ord, int rowbits, LevelTcArgs &A,
                   double *cost) {
    const int d = h->d;
    LevelArgs &a = A.L;
    const bool leaf = pass == Pass::LeafIn || pass == Pass::LeafOut;
    const bool split = pass == Pass::Split, gather = pass == Pass::Gather;
    std::memset(A.st, 0, sizeof(A.st));
    int cur[LTC_MAXD];
    for (int k = 0; k < d; ++k) cur[k] = a.m[k];
    double c = 0.0;
    uint32_t abytes_max = 0, a0_bytes = 0, bbytes = 0, cols_max = 0;
    auto up = [](uint32_t x, uint32_t al) { return (x + al - 1) / al * al; };
    for (int i = 0; i < d; ++i) {
        LtcStep &S = A.st[i];
        const int k = ord[i];
        S.k = k;
        S.m = cur[k];
        S.o = a.o[k];
        if (2 * S.o > 256 || S.m > 128) return false;   // MMA N <= 256
        if (i == 0 && S.m > 32) return false;             // the staging holds a fiber of <= 32
        // the other modes in C order, the two swapped where rowbits says so
        S.nod = 0;
        int64_t rows = vc;
        for (int j = 0; j < d; ++j)
            if (j != k) {
                S.om[S.nod] = j;
                S.od[S.nod] = cur[j];
                ++S.nod;
            }
        if (S.nod == 2 && ((rowbits >> i) & 1)) {
            std::swap(S.om[0], S.om[1]);
            std::swap(S.od[0], S.od[1]);
        }
        for (int jj = 0; jj < S.nod; ++jj) rows *= S.od[jj];
        int st = vc;
        for (int jj = S.nod - 1; jj >= 0; --jj) {
            S.rstr[S.om[jj]] = st;
            st *= S.od[jj];
        }
        S.rstr[k] = 0;
        if (rows > (1 << 20)) return false;
        S.rows = (int)rows;
        S.tiles = (S.rows + 127) / 128;
        S.ks = (S.m + 3) / 4;                  // 4 complex (hi, lo interleaved) per K-step
        S.np = (2 * S.o + 15) / 16 * 16;
        S.a_rs = (uint32_t)S.tiles * 4096u;
        S.b_rs = (uint32_t)S.np * 32u;
        S.b_half = (uint32_t)S.ks * S.b_rs;    // B1, then B2
        S.b_off = bbytes;
        bbytes += up(2 * S.b_half, 1024);
        S.idesc = tc::idesc_bf16(S.np);
        const uint32_t ab = (uint32_t)S.ks * S.a_rs;
        if (i == 0 && split) a0_bytes = ab;
        else abytes_max = std::max(abytes_max, ab);
        const uint32_t cols = (uint32_t)S.tiles * S.np;
        if (!(gather && i == d - 1)) cols_max = std::max(cols_max, cols);
        // tensor-pipe cycles (2 MMAs of N / 2 cycles per tile and K-step) plus
        // the conversion of the accumulator (about 10 instructions per output)
        c += 1.0 * S.tiles * S.ks * S.np + 0.08 * (double)S.rows * S.o;
        cur[k] = a.o[k];
    }
    {
        LtcStep &S = A.st[d - 1];
        int st = 1;
        for (int j = d - 1; j >= 0; --j) {
            S.tstr[j] = st;
            st *= a.o[j];
        }
        if (gather) {
            S.tcol = (cols_max + 31) / 32 * 32;
            if (S.tcol + (uint32_t)S.tiles * S.np > 256) return false;
        }
    }
    if (cols_max > 256) return false;
    // shared memory: [split: step-0 operand] [warpgroup 0] [warpgroup 1] [slack]
    int64_t gtab = 0;
    for (int k = 0; k < d; ++k) gtab += h->cb[k];
    const uint32_t tab = leaf ? up((uint32_t)gtab * 12u, 16) : 0;
    A.fac_off = up(abytes_max, 1024);
    A.tab_off = A.fac_off + bbytes;
    const uint32_t wg_bytes = up(A.tab_off + tab, 1024);
    uint32_t off = 0;
    A.a0_off = 0;
    if (split) off = up(a0_bytes, 1024);
    A.wg_off[0] = off;
    A.wg_off[1] = off + wg_bytes;
    // 1 KB for the base alignment and 2 KB of slack past the last operand
    uint32_t smem = off + 2 * wg_bytes + 1024 + 2048;
    const uint32_t budget = (uint32_t)g_smem_optin - 2048;   // static shared arrays
    if (smem > budget) return false;
    // one block per SM (it holds all 512 tensor-memory columns)
    smem = std::max<uint32_t>(smem, (uint32_t)g_smem_optin / 2 + 4096);
    A.smem = std::min(smem, budget);
    // shared-memory wavefronts of the accumulator stores of warp 0, tile 0
    // (output 0) into the next operand: 8-byte stores, 16 slots per wavefront
    for (int i = 0; i + 1 < d; ++i) {
        const LtcStep &S = A.st[i], &N = A.st[i + 1];
        int cnt[16] = {0};
        for (int r = 0; r < 32 && r < S.rows; ++r) {
            int idx[LTC_MAXD] = {0, 0, 0};
            int rest = r / vc;
            for (int jj = S.nod - 1; jj >= 0; --jj) {
                idx[S.om[jj]] = rest % S.od[jj];
                rest /= S.od[jj];
            }
            int rr = r % vc;
            for (int j = 0; j < d; ++j)
                if (j != S.k) rr += idx[j] * N.rstr[j];
            const int kp = idx[N.k];
            const uint32_t off = (uint32_t)(kp >> 2) * N.a_rs + tc::sw32c((uint32_t)rr, (uint32_t)(kp & 3));
            ++cnt[(off >> 3) & 15];
        }
        int deg = 1;
        for (int u = 0; u < 16; ++u) deg = std::max(deg, cnt[u]);
        c += 0.04 * (double)S.rows * S.o * deg;
    }
    if (cost) *cost = c;
    return true;
}

// One level pass as a single persistent launch on the tensor cores
// (k_level_tc, complex64 data, split-BF16 products).  done = false (nothing
// launched) when the pass does not fit the kernel.  dry = true only plans.
tb_status level_pass_tc(const tb_plan *h, Pass pass, bool conj, int side, int l, const void *in, void *out,
                        int64_t nv, cudaStream_t st, bool &done, bool dry = false, int vc_set = 0) {
    done = false;
    const int d = h->d;
    if (d > LTC_MAXD || d < 1) return TB_OK;
    const bool leaf = pass == Pass::LeafIn || pass == Pass::LeafOut;
    LevelTcArgs A;
    std::memset(&A, 0, sizeof(A));
    level_args_common(h, pass, conj, side, l, in, out, nv, A.L);
    LevelArgs &a = A.L;
    A.err = h->d_err;
    const tb::LevelTune &tn = h->ltune[side][(int)pass][leaf ? 0 : l];
    int vc = vc_set ? vc_set : tn.tc_vc;
    int cands[3] = {4, 2, 1}, nc = 3;
    if (vc > 0) {
        cands[0] = vc;
        nc = 1;
    }
    bool found = false;
    for (int ci = 0; ci < nc && !found; ++ci) {
        int v = (int)std::min<int64_t>(cands[ci], nv);
        while (v & (v - 1)) --v;
        // the mode order with the lowest planned cost among those that fit
        std::vector<int> p((size_t)d);
        for (int k = 0; k < d; ++k) p[(size_t)k] = k;
        double best = -1.0;
        int bord[LTC_MAXD] = {0, 1, 2};
        int brow = 0;
        do {
            for (int rb = 0; rb < (1 << d); ++rb) {
                double c = 0.0;
                if (!plan_level_tc(h, pass, v, p.data(), rb, A, &c)) continue;
                if (best < 0.0 || c < best) {
                    best = c;
                    brow = rb;
                    for (int k = 0; k < d; ++k) bord[k] = p[(size_t)k];
                }
            }
        } while (std::next_permutation(p.begin(), p.end()));
        if (best < 0.0) continue;
        a.vc = v;
        plan_level_tc(h, pass, v, bord, brow, A, nullptr);
        for (int k = 0; k < d; ++k) a.order[k] = bord[k];
        found = true;
    }
    if (!found) return TB_OK;
    a.lvc = ilog2(a.vc);
    a.nq = (int)((nv + a.vc - 1) / a.vc);
    const int64_t nunits = leaf ? h->P : (h->P >> d);
    a.nitems = nunits * a.nq;
    const int64_t per = leaf ? 2 : 1;   // work items per block at a time
    const int64_t blocks = std::min<int64_t>((a.nitems + per - 1) / per, (int64_t)g_num_sms);
    done = true;
    if (dry) return TB_OK;
    TB_CK(launch_level_tc(A, (int)blocks, st));
    return TB_OK;
}


template <class R>
const cx<R> *coreptr(const tb_plan *h);
template <>
const cx<double> *coreptr<double>(const tb_plan *h) { return h->core64; }
template <>
const cx<float> *coreptr<float>(const tb_plan *h) { return h->core32; }

// Split-BF16 tensor-core core contraction (complex64 tiles), 16 RHS per launch.
tb_status core_pass_tc(const tb_plan *h, bool adjoint, const void *in, void *out, int64_t nv, cudaStream_t st,
                       bool zero_pad = true) {
    const int d = h->d, Lc = h->Lc;
    const int dir = adjoint ? 1 : 0;
    const TileBuf<float> tin = tilebuf<float>(h, adjoint ? 1 : 0, Lc, (void *)in);
    const TileBuf<float> tout = tilebuf<float>(h, adjoint ? 0 : 1, Lc, out);
    CoreTcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.d = d;
    a.adjoint = dir;
    a.nitems = h->tc_nitems[dir];
    a.items = h->tc_items[dir];
    a.xpos = h->tc_xpos[dir];
    a.tiles = h->tc_tiles[dir];
    a.dims = h->core_dims;
    a.in = tin.p;
    a.out = tout.p;
    a.in_tsize = tin.tsize;
    a.out_tsize = tout.tsize;
    for (int k = 0; k < d; ++k) {
        a.in_R[k] = tin.R[k];
        a.out_R[k] = tout.R[k];
    }
    a.nv = (int)nv;
    a.zero_pad = zero_pad ? 1 : 0;
    a.err = h->d_err;
    for (int64_t v0 = 0; v0 < nv; v0 += 16) {
        a.v0 = (int)v0;
        a.nvc = (int)std::min<int64_t>(16, nv - v0);
        TB_CK(launch_core_tc(a, st));
    }
    return TB_OK;
}

template <class R>
tb_status core_pass(const tb_plan *h, bool adjoint, const void *in, void *out, int64_t nv, cudaStream_t st,
                    int precision, int64_t pf0 = 0, int64_t pf1 = -1) {
    const int d = h->d, Lc = h->Lc;
    if (precision == TB_PREC_C64_SPLITBF16 && !h->separable) return core_pass_tc(h, adjoint, in, out, nv, st);
    CoreApplyArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.pf0 = pf0;
    a.pf1 = pf1 < 0 ? ipow2(d * Lc) : pf1;
    a.d = d;
    a.P = h->P;
    a.nv = nv;
    a.Lc = Lc;
    a.in = tilebuf<R>(h, adjoint ? 1 : 0, Lc, (void *)in);
    a.out = tilebuf<R>(h, adjoint ? 0 : 1, Lc, out);
    const int64_t es = sizeof(cx<R>);
    if (h->separable) {
        int m[TB_MAX_D], o[TB_MAX_D];
        for (int k = 0; k < d; ++k) {
            a.Rt[k] = h->tgt[Lc].R[k];
            a.Rs[k] = h->src[Lc].R[k];
            a.kron[k] = std::is_same<R, double>::value ? (const cx<R> *)h->kron64[k] : (const cx<R> *)h->kron32[k];
            m[k] = adjoint ? a.Rt[k] : a.Rs[k];
            o[k] = adjoint ? a.Rs[k] : a.Rt[k];
        }
        TB_TRY(pick_chunk<R>(d, m, o, nv, a.nvc, a.smem, a.offX, a.offB0, a.offB1, a.offY, a.offA));
        TB_CK(launch_core_kron<R>(adjoint, a, st));
        return TB_OK;
    }
    a.dims = h->core_dims;
    a.off = h->core_off;
    a.core = coreptr<R>(h);
    const int64_t tmax = std::max(prod_tile(h->src[Lc], d), prod_tile(h->tgt[Lc], d));
    int64_t c = (96 * 1024) / (tmax * es);
    c = std::max<int64_t>(1, std::min<int64_t>({c, nv, 16}));
    a.nvc = c;
    a.smem = (size_t)(tmax * c * es);
    if (a.smem > g_smem_optin) return fail(TB_EUNSUPPORTED, "core block exceeds shared memory");
    if constexpr (std::is_same<R, float>::value) {
        if (!adjoint && nv == 1 && h->rg.kind &&
            (h->core_mode == 2 || (h->core_mode == 0 && h->core_regen_tuned))) {
            CoreApplyArgs<float> b = a;
            b.rg = h->rg;
            b.offX = (int)tmax;     // table length (entries of the largest mid-level tile)
            b.offB0 = (int)tmax;
            b.smem = (size_t)tmax * (3 * sizeof(float2) + 2 * (size_t)d * sizeof(int));
            if (b.smem <= g_smem_optin) {
                TB_CK(launch_core_regen(b, st));
                return TB_OK;
            }
        }
        if (!adjoint && nv == 1 && h->core_rows) {
            TB_CK(launch_core_rows<float>(a, st));
            return TB_OK;
        }
    }
    TB_CK(launch_core_dense<R>(adjoint, a, st));
    return TB_OK;
}

// Real flops of one mode-product chain X (dims m) -> Y (dims o), per RHS.
double chain_flops(int d, const int *m, const int *o) {
    double f = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = (double)m[k] * o[k];
        for (int i = 0; i < k; ++i) t *= o[i];
        for (int i = k + 1; i < d; ++i) t *= m[i];
        f += 8.0 * t;
    }
    return f;
}

// Bytes and flops one launch of a pass must move / execute (stored sizes).
void pass_cost(const tb_plan *h, Pass pass, int side, int l, int64_t nv, size_t es, int64_t &bytes, double &flops) {
    const int d = h->d;
    const SideLevel *S = side == 0 ? h->src : h->tgt;
    int64_t N = 1;
    for (int k = 0; k < d; ++k) N *= h->n[k];
    auto tensor = [&](int lv) { return h->P * prod_tile(S[lv], d) * nv * (int64_t)es; };
    auto facb = [&](int lv) {
        int64_t b = 0;
        for (int k = 0; k < d; ++k) b += S[lv].count[k] * S[lv].R[k] * S[lv].cin[k];
        return b * (int64_t)es;
    };
    int m[TB_MAX_D], o[TB_MAX_D];
    switch (pass) {
        case Pass::LeafIn:
        case Pass::LeafOut:
            bytes = N * nv * (int64_t)es + tensor(0) + facb(0);
            break;
        case Pass::Split:
        case Pass::Gather:
            bytes = tensor(l - 1) + tensor(l) + facb(l);
            break;
    }
    // algorithmic flops: 8 per complex multiply-add of the chain in its
    // fewest-multiply mode order (the products of a chain commute)
    pass_dims(h, pass, side, l, m, o);
    int ord[TB_MAX_D];
    flops = 8.0 * (double)h->P * nv * best_order(d, m, o, ord);
}

template <class R>
const SepStep<R> *sepptr(const tb_plan *h, int dir);
template <>
const SepStep<double> *sepptr<double>(const tb_plan *h, int dir) { return h->sep64[dir]; }
template <>
const SepStep<float> *sepptr<float>(const tb_plan *h, int dir) { return h->sep32[dir]; }

template <class R>
const cx<R> *sepr_coef(const tb_plan *h, int k);
template <>
const cx<double> *sepr_coef<double>(const tb_plan *h, int k) { return h->sepr_coef64[k]; }
template <>
const cx<float> *sepr_coef<float>(const tb_plan *h, int k) { return h->sepr_coef32[k]; }

// Separable handle: per-mode chains applied in passes over up to three
// consecutive modes (from the last mode down), ping-ponging full tensors.
template <class R>
tb_status run_sep(tb_plan *h, bool adjoint, const void *in, void *out, int64_t nv, cudaStream_t st, bool prof,
                  void *const *B) {
    const int d = h->d, dir = adjoint ? 1 : 0;
    const int64_t es = sizeof(cx<R>);
    const int64_t limit = 96 * 1024;
    int64_t N = 1;
    for (int k = 0; k < d; ++k) N *= h->n[k];
    // per-mode passes: register-resident chains where the mode has the
    // exact-rank form, else thread-per-fiber passes when the chain fits a
    // shared-memory column of at least 32 threads per block
    {
        int threads[TB_MAX_D];
        size_t smem[TB_MAX_D];
        bool use_reg[TB_MAX_D];
        bool fits = true;
        for (int k = 0; k < d && fits; ++k) {
            int64_t inner = nv;
            for (int j = k + 1; j < d; ++j) inner *= h->n[j];
            use_reg[k] = h->sep_choice != 1 && h->sep_choice != 2 && h->sepr_ok[k] &&
                         sep_reg_supported<R>(h->Lc, h->sepr_rk[k]) && h->n[k] * inner < ((int64_t)1 << 31);
            const int64_t fixed = h->sep_npk[dir][k] * (int64_t)sizeof(SepNz<R>);
            int T = 256;
            while (T >= 32 && 2 * h->sep_maxext[k] * T * es + fixed > limit) T /= 2;
            threads[k] = T;
            smem[k] = (size_t)(2 * h->sep_maxext[k] * T * es + fixed + 16);
            fits = use_reg[k] || T >= 32;
        }
        if (fits && h->sep_choice != 2) {
            int i = 0;
            for (int k = d - 1; k >= 0; --k, ++i) {
                if (h->sep_choice == 4 && k > 0 && use_reg[k] && use_reg[k - 1] &&
                    h->sepr_rk[k] == h->sepr_rk[k - 1] && h->n[k] == h->n[k - 1]) {
                    // modes k - 1 and k fused in one pass
                    SepReg2Args<R> a;
                    std::memset(&a, 0, sizeof(a));
                    const int nk = (int)h->n[k];
                    a.lc = h->Lc;
                    a.rk = h->sepr_rk[k];
                    a.outer = 1;
                    for (int j = 0; j < k - 1; ++j) a.outer *= h->n[j];
                    a.inner = nv;
                    for (int j = k + 1; j < d; ++j) a.inner *= h->n[j];
                    int lq = 0;
                    while ((2 << lq) * nk <= 128 && ((int64_t)2 << lq) <= a.inner) ++lq;
                    a.lq = lq;
                    a.q = 1 << lq;
                    a.nchunks = (a.inner + a.q - 1) / a.q;
                    a.in = (const cx<R> *)(i == 0 ? in : B[(i - 1) & 1]);
                    a.out = (cx<R> *)(k - 1 == 0 ? out : B[i & 1]);
                    a.coef_a = sepr_coef<R>(h, k - 1);
                    a.coef_b = sepr_coef<R>(h, k);
                    a.cf4_a = h->sepr_cf4[dir][k - 1];
                    a.cf4_b = h->sepr_cf4[dir][k];
                    for (int p = 0; p < nk; ++p) {
                        a.ld_a[p] = h->sepr_ld[k - 1][p];
                        a.st_a[p] = h->sepr_st[k - 1][p];
                        a.ld_b[p] = h->sepr_ld[k][p];
                        a.st_b[p] = h->sepr_st[k][p];
                    }
                    ProfRec r{"sep_reg2", k - 1, (int)adjoint, nullptr, nullptr, 0, 0.0};
                    if (prof) {
                        r.bytes = 2 * N * nv * es;
                        for (int j = k - 1; j <= k; ++j) {
                            r.bytes += h->sep_nnz[dir][j] * (es + 4);
                            r.flops += 8.0 * (double)h->sep_nnz[dir][j] * (double)(N / h->n[j]) * (double)nv;
                        }
                        TB_CK(cudaEventCreate(&r.e0));
                        TB_CK(cudaEventCreate(&r.e1));
                        TB_CK(cudaEventRecord(r.e0, st));
                    }
                    TB_CK(launch_sep_reg2<R>(adjoint, a, st));
                    if (prof) {
                        TB_CK(cudaEventRecord(r.e1, st));
                        h->prof.push_back(r);
                    }
                    --k;
                    continue;
                }
                if (use_reg[k]) {
                    SepRegArgs<R> a;
                    std::memset(&a, 0, sizeof(a));
                    a.lc = h->Lc;
                    a.rk = h->sepr_rk[k];
                    a.outer = 1;
                    for (int j = 0; j < k; ++j) a.outer *= h->n[j];
                    a.inner = nv;
                    for (int j = k + 1; j < d; ++j) a.inner *= h->n[j];
                    a.in = (const cx<R> *)(i == 0 ? in : B[(i - 1) & 1]);
                    a.out = (cx<R> *)(k == 0 ? out : B[i & 1]);
                    a.coef = sepr_coef<R>(h, k);
                    a.cf4 = h->sepr_cf4[dir][k];
                    for (int p = 0; p < h->n[k]; ++p) {
                        a.ldo[p] = (int)(h->sepr_ld[k][p] * a.inner);
                        a.sto[p] = (int)(h->sepr_st[k][p] * a.inner);
                    }
                    a.blocks = (int)g_num_sms * 3;   // grid of the persistent scalar form
                    ProfRec r{"sep_reg", k, (int)adjoint, nullptr, nullptr, 0, 0.0};
                    if (prof) {
                        r.bytes = 2 * N * nv * es + h->sep_nnz[dir][k] * (es + 4);
                        r.flops = 8.0 * (double)h->sep_nnz[dir][k] * (double)(N / h->n[k]) * (double)nv;
                        TB_CK(cudaEventCreate(&r.e0));
                        TB_CK(cudaEventCreate(&r.e1));
                        TB_CK(cudaEventRecord(r.e0, st));
                    }
                    const int variant = h->sep_choice == 5 ? 1 : h->sep_choice == 6 ? 2 : 0;
                    TB_CK(launch_sep_reg<R>(adjoint, variant, a, st));
                    if (prof) {
                        TB_CK(cudaEventRecord(r.e1, st));
                        h->prof.push_back(r);
                    }
                    continue;
                }
                SepFiberArgs<R> a;
                std::memset(&a, 0, sizeof(a));
                a.k = k;
                a.nk = (int)h->n[k];
                a.outer = 1;
                for (int j = 0; j < k; ++j) a.outer *= h->n[j];
                a.inner = nv;
                for (int j = k + 1; j < d; ++j) a.inner *= h->n[j];
                a.in = (const cx<R> *)(i == 0 ? in : B[(i - 1) & 1]);
                a.out = (cx<R> *)(k == 0 ? out : B[i & 1]);
                a.steps = sepptr<R>(h, dir) + h->sep_step0[dir][k];
                a.nsteps = h->sep_nsteps[dir][k];
                a.maxext = h->sep_maxext[k];
                a.npk = (int)h->sep_npk[dir][k];
                a.threads = threads[k];
                a.smem = smem[k];
                ProfRec r{"sep_mode", k, (int)adjoint, nullptr, nullptr, 0, 0.0};
                if (prof) {
                    r.bytes = 2 * N * nv * es + h->sep_nnz[dir][k] * (es + 4);
                    r.flops = 8.0 * (double)h->sep_nnz[dir][k] * (double)(N / h->n[k]) * (double)nv;
                    TB_CK(cudaEventCreate(&r.e0));
                    TB_CK(cudaEventCreate(&r.e1));
                    TB_CK(cudaEventRecord(r.e0, st));
                }
                TB_CK(launch_sep_fiber<R>(a, st));
                if (prof) {
                    TB_CK(cudaEventRecord(r.e1, st));
                    h->prof.push_back(r);
                }
            }
            return TB_OK;
        }
    }
    struct Plan {
        int k0, k1;
        int64_t ic, buf;
    };
    std::vector<Plan> plan;
    auto bufsz = [&](int k0, int k1) {
        int64_t b = 0;
        for (int k = k0; k <= k1; ++k) {
            int64_t t = h->sep_maxext[k];
            for (int j = k0; j <= k1; ++j)
                if (j != k) t *= h->n[j];
            b = std::max(b, t);
        }
        return b;
    };
    for (int k1 = d - 1; k1 >= 0;) {
        int64_t inner = nv;
        for (int k = k1 + 1; k < d; ++k) inner *= h->n[k];
        const int64_t icmin = std::min<int64_t>(inner, 8);   // keep >= 64 contiguous bytes per fiber
        int k0 = k1;
        while (k0 > 0 && k1 - k0 < 2 && 2 * bufsz(k0 - 1, k1) * icmin * es <= limit) --k0;
        const int64_t b = bufsz(k0, k1);
        const int64_t ic = std::max<int64_t>(1, std::min<int64_t>(inner, limit / (2 * b * es)));
        if ((size_t)(2 * b * ic * es) > g_smem_optin)
            return fail(TB_EUNSUPPORTED, "per-mode pass needs more shared memory than the device has");
        plan.push_back(Plan{k0, k1, ic, b * ic});
        k1 = k0 - 1;
    }
    for (size_t i = 0; i < plan.size(); ++i) {
        const Plan &pl = plan[i];
        SepPassArgs<R> a;
        std::memset(&a, 0, sizeof(a));
        a.d = d;
        a.k0 = pl.k0;
        a.k1 = pl.k1;
        for (int k = 0; k < d; ++k) a.n[k] = (int)h->n[k];
        a.outer = 1;
        for (int k = 0; k < pl.k0; ++k) a.outer *= h->n[k];
        a.inner = nv;
        for (int k = pl.k1 + 1; k < d; ++k) a.inner *= h->n[k];
        a.ic = (int)pl.ic;
        a.nchunks = (a.inner + a.ic - 1) / a.ic;
        // pass i reads the user input (i = 0) or buffer (i-1) % 2 and writes
        // buffer i % 2, the last pass writes the user output
        a.in = (const cx<R> *)(i == 0 ? in : B[(i - 1) & 1]);
        a.out = (cx<R> *)(i + 1 == plan.size() ? out : B[i & 1]);
        a.steps = sepptr<R>(h, dir);
        for (int k = 0; k < d; ++k) {
            a.step0[k] = h->sep_step0[dir][k];
            a.nsteps[k] = h->sep_nsteps[dir][k];
        }
        a.buf = (int)pl.buf;
        a.smem = (size_t)(2 * pl.buf * es);
        ProfRec r{"sep_pass", (int)i, (int)adjoint, nullptr, nullptr, 0, 0.0};
        if (prof) {
            r.bytes = 2 * N * nv * es;
            for (int k = pl.k0; k <= pl.k1; ++k) {
                r.bytes += h->sep_nnz[dir][k] * (es + 4);
                r.flops += 8.0 * (double)h->sep_nnz[dir][k] * (double)(N / h->n[k]) * (double)nv;
            }
            TB_CK(cudaEventCreate(&r.e0));
            TB_CK(cudaEventCreate(&r.e1));
            TB_CK(cudaEventRecord(r.e0, st));
        }
        TB_CK(launch_sep_pass<R>(a, st));
        if (prof) {
            TB_CK(cudaEventRecord(r.e1, st));
            h->prof.push_back(r);
        }
    }
    return TB_OK;
}

// `bufs` overrides the handle's workspace buffers (tb_apply_noalloc); NULL
// keeps them.
template <class R>
tb_status run_chain(tb_plan *h, bool adjoint, const void *in, void *out, int64_t nv, cudaStream_t st, bool prof,
                    int precision, void *const *bufs = nullptr, size_t t0_bytes = 0) {
    void *B[2] = {h->ws.buf[0], h->ws.buf[1]};
    void *T[2] = {h->ws.mbuf[0], h->ws.mbuf[1]};
    size_t T0bytes = h->ws.mbytes[0];
    if (bufs) {
        B[0] = bufs[0];
        B[1] = bufs[1];
        T[0] = bufs[2];
        T[1] = bufs[3];
        T0bytes = t0_bytes;
    }
    if (h->separable) return run_sep<R>(h, adjoint, in, out, nv, st, prof, B);
    const int Lc = h->Lc, d = h->d;
    const int first = adjoint ? 1 : 0, second = 1 - first;   // side traversed first / last
    const size_t es = sizeof(cx<R>);
    auto timed = [&](const char *name, int level, int64_t bytes, double flops, int kernels,
                     auto &&fn) -> tb_status {
        ProfRec r{name, level, (int)adjoint, nullptr, nullptr, bytes, flops, kernels};
        if (prof) {
            TB_CK(cudaEventCreate(&r.e0));
            TB_CK(cudaEventCreate(&r.e1));
            TB_CK(cudaEventRecord(r.e0, st));
        }
        tb_status s = fn();
        if (prof) {
            TB_CK(cudaEventRecord(r.e1, st));
            h->prof.push_back(r);
        }
        return s;
    };
    auto level = [&](Pass p, const char *name, int side, int l, const void *i, void *o) -> tb_status {
        int64_t bytes = 0;
        double flops = 0;
        if (prof) pass_cost(h, p, side, l, nv, es, bytes, flops);
        if (std::is_same<R, float>::value && level_tc_wanted(h, p, side, l, precision)) {
            bool ok = false;
            TB_TRY(level_pass_tc(h, p, adjoint, side, l, i, o, nv, st, ok, true));
            if (ok)
                return timed(name, l, bytes, flops, 1, [&] {
                    bool done = false;
                    return level_pass_tc(h, p, adjoint, side, l, i, o, nv, st, done);
                });
        }
        if (std::is_same<R, float>::value && h->level_choice != 1 && level_fused_wanted(h, p, side, l)) {
            bool ok = false;
            TB_TRY(level_pass_fused(h, p, adjoint, side, l, i, o, nv, st, T[0], T0bytes, ok, true));
            if (ok)
                return timed(name, l, bytes, flops, 1, [&] {
                    bool done = false;
                    return level_pass_fused(h, p, adjoint, side, l, i, o, nv, st, T[0], T0bytes, done);
                });
        }
        return timed(name, l, bytes, flops, d,
                     [&] { return level_pass<R>(h, p, adjoint, side, l, i, o, nv, st, T); });
    };
    int cur = 0;
    const void *gin = nullptr;   // input of the next target-side pass
    TB_TRY(level(Pass::LeafIn, "leaf_in", first, 0, in, B[cur]));
    for (int l = 1; l <= Lc; ++l) {
        TB_TRY(level(Pass::Split, "split", first, l, B[cur], B[cur ^ 1]));
        cur ^= 1;
    }
    {
        int64_t bytes = 0;
        double flops = 0;
        if (prof) {
            if (h->separable) {
                int m[TB_MAX_D], o[TB_MAX_D];
                int64_t kb = 0;
                for (int k = 0; k < d; ++k) {
                    m[k] = h->src[Lc].R[k];
                    o[k] = h->tgt[Lc].R[k];
                    kb += (int64_t)(1 << Lc) * (1 << Lc) * m[k] * o[k];
                }
                bytes = (h->P * (prod_tile(h->src[Lc], d) + prod_tile(h->tgt[Lc], d)) * nv + kb) * (int64_t)es;
                flops = (double)h->P * nv * chain_flops(d, m, o);
            } else {
                bytes = (h->core_entries + (h->core_in_entries + h->core_out_entries) * nv) * (int64_t)es;
                flops = 8.0 * (double)h->core_entries * nv;
            }
        }
        const bool tc_core = precision == TB_PREC_C64_SPLITBF16 && !h->separable;
        const int core_kernels = tc_core ? (int)((nv + 15) / 16) : 1;
        // the split-BF16 core writes its own buffer, whose padded entries keep
        // their zeros between applies (not with caller-provided buffers)
        const int dir = adjoint ? 1 : 0;
        void *cdst = (tc_core && !bufs && h->ws.cout[dir] && h->ws.cout_nv[dir] == nv) ? h->ws.cout[dir] : nullptr;
        TB_TRY(timed("core", Lc, bytes, flops, core_kernels, [&] {
            if (cdst) return core_pass_tc(h, adjoint, B[cur], cdst, nv, st, false);
            return core_pass<R>(h, adjoint, B[cur], B[cur ^ 1], nv, st, precision);
        }));
        if (!cdst) {
            cur ^= 1;
            gin = B[cur];
        } else {
            gin = cdst;   // B[cur], the core's input, is free again
        }
    }
    for (int l = Lc; l >= 1; --l) {
        TB_TRY(level(Pass::Gather, "gather", second, l, gin, B[cur ^ 1]));
        cur ^= 1;
        gin = B[cur];
    }
    TB_TRY(level(Pass::LeafOut, "leaf_out", second, 0, gin, out));
    return TB_OK;
}

// The split-BF16 core's output buffers (tb::Workspace::cout) for nv RHS: on
// handles that apply split BF16, one per direction, holding zeros in every
// padded entry.  They are (re)allocated when too small and cleared when nv
// changes (the padded positions depend on nv); both take a device-wide
// synchronisation, outside any stream capture.
tb_status ensure_core_out(tb_plan *h, int64_t nv) {
    if (h->separable || !(h->precisions & (1u << TB_PREC_C64_SPLITBF16))) return TB_OK;
    for (int dir = 0; dir < 2; ++dir) {
        const TileBuf<float> t = tilebuf<float>(h, dir == 0 ? 1 : 0, h->Lc, nullptr);
        const int64_t entries = h->P * (int64_t)t.tsize;
        if ((uint64_t)nv > (uint64_t)(SIZE_MAX / sizeof(c64)) / (uint64_t)std::max<int64_t>(entries, 1))
            return fail(TB_ENOMEM, "core output size for nv = " + std::to_string(nv) + " overflows");
        const size_t need = (size_t)entries * (size_t)nv * sizeof(c64);
        if (need > h->ws.cout_bytes[dir]) {
            TB_CK(cudaDeviceSynchronize());
            for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
            h->graphs.clear();
            if (h->ws.cout[dir]) cudaFree(h->ws.cout[dir]);
            h->ws.cout[dir] = nullptr;
            h->ws.cout_bytes[dir] = 0;
            h->ws.cout_nv[dir] = 0;
            TB_CK(cudaMalloc(&h->ws.cout[dir], need));
            h->ws.cout_bytes[dir] = need;
        }
        if (h->ws.cout_nv[dir] != nv) {
            TB_CK(cudaDeviceSynchronize());
            TB_CK(cudaMemset(h->ws.cout[dir], 0, need));
            TB_CK(cudaDeviceSynchronize());
            h->ws.cout_nv[dir] = nv;
        }
    }
    return TB_OK;
}

tb_status ensure_workspace(tb_plan *h, int64_t nv) {
    const int64_t lm = std::max<int64_t>({h->level_max, h->mode_max[0], h->mode_max[1], 1});
    if ((uint64_t)nv > (uint64_t)(SIZE_MAX / sizeof(c128)) / (uint64_t)lm)
        return fail(TB_ENOMEM, "workspace size for nv = " + std::to_string(nv) + " overflows");
    const size_t need = (size_t)h->level_max * (size_t)nv * sizeof(c128);
    const size_t mneed[2] = {(size_t)h->mode_max[0] * (size_t)nv * sizeof(c128),
                             (size_t)h->mode_max[1] * (size_t)nv * sizeof(c128)};
    TB_TRY(ensure_core_out(h, nv));
    if (need <= h->ws.bytes && mneed[0] <= h->ws.mbytes[0] && mneed[1] <= h->ws.mbytes[1]) return TB_OK;
    TB_CK(cudaDeviceSynchronize());
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    for (int i = 0; i < 2; ++i) {
        if (h->ws.buf[i]) cudaFree(h->ws.buf[i]);
        if (h->ws.mbuf[i]) cudaFree(h->ws.mbuf[i]);
        h->ws.buf[i] = h->ws.mbuf[i] = nullptr;
        h->ws.mbytes[i] = 0;
    }
    h->ws.bytes = 0;
    for (int i = 0; i < 2; ++i) TB_CK(cudaMalloc(&h->ws.buf[i], need));
    for (int i = 0; i < 2; ++i) TB_CK(cudaMemset(h->ws.buf[i], 0, need));
    h->ws.bytes = need;
    for (int i = 0; i < 2; ++i)
        if (mneed[i] > 0) {
            TB_CK(cudaMalloc(&h->ws.mbuf[i], mneed[i]));
            h->ws.mbytes[i] = mneed[i];
        }
    return TB_OK;
}

// Output lengths o_k of the modes of a level pass (see level_pass).
void pass_out_dims(const tb_plan *h, Pass pass, int side, int l, int *o) {
    const SideLevel *S = side == 0 ? h->src : h->tgt;
    for (int k = 0; k < h->d; ++k) {
        switch (pass) {
            case Pass::LeafIn: o[k] = S[0].R[k]; break;
            case Pass::LeafOut: o[k] = (int)h->cb[k]; break;
            case Pass::Split: o[k] = S[l].R[k]; break;
            case Pass::Gather: o[k] = 2 * S[l - 1].R[k]; break;
        }
    }
}

// Empirical launch-shape search (tb_autotune): each candidate runs once to
// warm up and three times under CUDA events on `st`; the fastest is kept.
// `uin` / `uout` stand in for the user tensors (N x nv).
template <class R>
tb_status tune_impl(tb_plan *h, int64_t nv, int precision, cudaStream_t st, const void *uin, void *uout) {
    cudaEvent_t e0, e1;
    TB_CK(cudaEventCreate(&e0));
    TB_CK(cudaEventCreate(&e1));
    tb_status status = TB_OK;
    auto time_it = [&](auto &&fn, float &best) -> tb_status {
        TB_TRY(fn());
        best = 3.0e38f;
        for (int r = 0; r < 3; ++r) {
            TB_CK(cudaEventRecord(e0, st));
            TB_TRY(fn());
            TB_CK(cudaEventRecord(e1, st));
            TB_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            TB_CK(cudaEventElapsedTime(&ms, e0, e1));
            best = std::min(best, ms);
        }
        return TB_OK;
    };
    if (h->separable) {
        float best = 3.0e38f;
        int choice = 0;
        bool any_reg = false;
        for (int k = 0; k < h->d; ++k) any_reg = any_reg || h->sepr_ok[k];
        for (int c = 1; c <= (any_reg ? 6 : 2) && status == TB_OK; ++c) {
            h->sep_choice = c;
            float t = 0.f;
            status = time_it([&] { return run_chain<R>(h, false, uin, uout, nv, st, false, precision); }, t);
            if (status == TB_OK && t < best) {
                best = t;
                choice = c;
            }
        }
        h->sep_choice = choice;
    } else {
        void *B[2] = {h->ws.buf[0], h->ws.buf[1]};
        void *T[2] = {h->ws.mbuf[0], h->ws.mbuf[1]};
        // the one-RHS forward core: stored cores against cores regenerated at the
        // skeleton points (tb_options.core_mode = 0 only)
        h->core_regen_tuned = 0;
        if (std::is_same<R, float>::value && nv == 1 && h->rg.kind && h->core_mode == 0 &&
            precision == TB_PREC_C64) {
            float t_st = 0.f, t_rg = 0.f;
            status = time_it([&] { return core_pass<R>(h, false, B[0], B[1], nv, st, precision); }, t_st);
            if (status == TB_OK) {
                h->core_regen_tuned = 1;
                status = time_it([&] { return core_pass<R>(h, false, B[0], B[1], nv, st, precision); }, t_rg);
                h->core_regen_tuned = (status == TB_OK && t_rg < t_st) ? 1 : 0;
            }
        }
        // fused level passes (complex64): RHS per work item, blocks per SM and
        // output rows per register chunk; every candidate accumulates each
        // output in the same order, so the choice does not change results
        if (std::is_same<R, float>::value && h->level_choice != 1) {
            const Pass fpasses[4] = {Pass::LeafIn, Pass::Split, Pass::Gather, Pass::LeafOut};
            for (int side = 0; side < 2 && status == TB_OK; ++side)
                for (Pass p : fpasses) {
                    const bool leaf = p == Pass::LeafIn || p == Pass::LeafOut;
                    for (int l = leaf ? 0 : 1; l <= (leaf ? 0 : h->Lc) && status == TB_OK; ++l) {
                        const void *in = p == Pass::LeafIn ? uin : B[0];
                        void *out = p == Pass::LeafOut ? uout : (p == Pass::LeafIn ? B[0] : B[1]);
                        tb::LevelTune best;
                        h->ltune[side][(int)p][l] = best;   // candidates start from the built-in rule
                        float tbest = 3.0e38f;
                        for (int vc : {1, 2, 4})
                            for (int cps : {2, 3, 4})
                                for (int ob : {0, 8}) {
                                    bool ok = false;
                                    status = level_pass_fused(h, p, false, side, l, in, out, nv, st, T[0],
                                                              h->ws.mbytes[0], ok, true, vc, cps, ob);
                                    if (status != TB_OK || !ok) continue;
                                    float t = 0.f;
                                    status = time_it(
                                        [&] {
                                            bool done = false;
                                            return level_pass_fused(h, p, false, side, l, in, out, nv, st, T[0],
                                                                    h->ws.mbytes[0], done, false, vc, cps, ob);
                                        },
                                        t);
                                    if (status != TB_OK) break;
                                    if (t < tbest) {
                                        tbest = t;
                                        best.mode = 2;
                                        best.vc = vc;
                                        best.cps = cps;
                                        best.obmax = ob;
                                    }
                                }
                        // split-BF16 applies: the tensor-core launch, RHS per work item
                        if (status == TB_OK && precision == TB_PREC_C64_SPLITBF16 &&
                            (h->level_choice == 0 || h->level_choice == 3)) {
                            for (int vc : {1, 2, 4}) {
                                bool ok = false;
                                status = level_pass_tc(h, p, false, side, l, in, out, nv, st, ok, true, vc);
                                if (status != TB_OK || !ok) continue;
                                float t = 0.f;
                                status = time_it(
                                    [&] {
                                        bool done = false;
                                        return level_pass_tc(h, p, false, side, l, in, out, nv, st, done, false, vc);
                                    },
                                    t);
                                if (status != TB_OK) break;
                                if (t < tbest) {
                                    tbest = t;
                                    best.mode = 3;
                                    best.tc_vc = vc;
                                }
                            }
                        }
                        if (status == TB_OK && best.mode >= 2 && h->level_choice == 0) {
                            // against the per-mode launches of the same pass (their shapes
                            // as tuned below are not known yet: the built-in ones)
                            float tmode = 3.0e38f;
                            status = time_it(
                                [&] { return level_pass<R>(h, p, false, side, l, in, out, nv, st, T); }, tmode);
                            if (status == TB_OK && tmode <= tbest) best.mode = 1;
                        }
                        h->ltune[side][(int)p][l] = best;
                    }
                }
        }
        const int ri = std::is_same<R, double>::value ? 1 : 0;
        const Pass passes[4] = {Pass::LeafIn, Pass::Split, Pass::Gather, Pass::LeafOut};
        const int waves[3] = {8, 32, 128};
        for (int side = 0; side < 2 && status == TB_OK; ++side)
            for (Pass p : passes) {
                const bool leaf = p == Pass::LeafIn || p == Pass::LeafOut;
                for (int l = leaf ? 0 : 1; l <= (leaf ? 0 : h->Lc) && status == TB_OK; ++l) {
                    const void *in = p == Pass::LeafIn ? uin : B[0];
                    void *out = p == Pass::LeafOut ? uout : (p == Pass::LeafIn ? B[0] : B[1]);
                    int o[TB_MAX_D];
                    pass_out_dims(h, p, side, l, o);
                    for (int k = 0; k < h->d && status == TB_OK; ++k) {
                        // rows per register tile: the even split of o_k into 1, 2 or 3 chunks
                        int obs[3], nob = 0;
                        for (int nch = 1; nch <= 3; ++nch) {
                            int ob = (o[k] + nch - 1) / nch;
                            ob += ob & 1;
                            if (ob == 22) ob = 24;
                            if (!mode_ob_valid(ob)) continue;
                            bool dup = false;
                            for (int i = 0; i < nob; ++i) dup = dup || obs[i] == ob;
                            if (!dup) obs[nob++] = ob;
                        }
                        // threads per column slice: the built-in (fewest covering a unit)
                        // and 128; slices per column: 1, 2, 4 (up to 128 threads)
                        const int bts[2] = {0, 128};
                        tb::ModeTune best;
                        float tbest = 3.0e38f;
                        for (int i = 0; i < nob && status == TB_OK; ++i)
                            for (int w : waves)
                                for (int rk = 0; rk < 2 && status == TB_OK; ++rk)
                                    for (int bi = 0, bt0 = 0; bi < 2 && status == TB_OK; ++bi)
                                        for (int sb = 1; sb <= 4 && status == TB_OK; sb *= 2) {
                                            if (bi == 1 && bt0 == 128) break;   // the same launches as bi = 0
                                            if (h->mode_slices && sb != h->mode_slices) continue;   // forced
                                            const int cw = bi == 0 ? bt0 : bts[bi];
                                            if (sb > 1 && (sb * cw > 128 || ri)) break;
                                            float t = 0.f;
                                            status = time_it(
                                                [&] {
                                                    return level_pass<R>(h, p, false, side, l, in, out, nv, st, T, k,
                                                                         obs[i], w, 0, -1, rk, bts[bi],
                                                                         bi == 0 ? &bt0 : nullptr, sb);
                                                },
                                                t);
                                            if (status != TB_OK) break;
                                            if (t < tbest) {
                                                tbest = t;
                                                best.ob = obs[i];
                                                best.waves = w;
                                                best.rank = rk;
                                                best.bt = bts[bi];
                                                best.sub = sb;
                                            }
                                        }
                        h->tune[ri][side][(int)p][l][k] = best;
                    }
                }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status == TB_OK) h->tuned.emplace_back(nv, precision);
    return status;
}

tb_status init_device_attrs(const tb_plan *h) {
    if (g_smem_optin == 0) {
        int v = 0, sms = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        g_num_sms = sms;
        g_smem_optin = (size_t)v;
    }
    return TB_OK;
}

bool is_tuned(const tb_plan *h, int64_t nv, int precision) {
    for (auto &t : h->tuned)
        if (t.first == nv && t.second == precision) return true;
    return false;
}

tb_status apply_common(tb_handle h, const void *in, void *out, int64_t nv, int precision, void *stream,
                       bool adjoint) {
    if (!h) return fail(TB_EINVAL, "handle is NULL");
    if (nv <= 0) return fail(TB_EINVAL, "nv must be positive");
    if (precision < TB_PREC_C128 || precision > TB_PREC_C64_SPLITBF16)
        return fail(TB_EINVAL, "unknown precision");
    if (!(h->precisions & (1u << precision)))
        return fail(TB_EUNSUPPORTED, "handle was built without precision " + std::to_string(precision));
    TB_TRY(check_device_ptr(in, adjoint ? "g" : "f"));
    TB_TRY(check_device_ptr(out, adjoint ? "v" : "u"));
    int64_t N = 1;
    for (int k = 0; k < h->d; ++k) N *= h->n[k];
    const size_t es = precision == TB_PREC_C128 ? 16 : 8;
    TB_TRY(check_nv(N, nv, es));
    const char *a0 = (const char *)in, *b0 = (const char *)out;
    const size_t bytes = (size_t)N * nv * es;
    if (a0 < b0 + bytes && b0 < a0 + bytes) return fail(TB_EINVAL, "input and output overlap");
    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice"); }
    if (g_smem_optin == 0) {
        int v = 0, sms = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        g_num_sms = sms;
        g_smem_optin = (size_t)v;
    }
    TB_TRY(ensure_workspace(h, nv));
    cudaStream_t st = (cudaStream_t)stream;
    if (h->autotune && !is_tuned(h, nv, precision)) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        TB_CK(cudaStreamIsCapturing(st, &cs));
        if (cs == cudaStreamCaptureStatusNone) {
            // the call's own tensors stand in for the user tensors; `out` is
            // overwritten by the apply below
            if (precision == TB_PREC_C128) TB_TRY(tune_impl<double>(h, nv, precision, st, in, out));
            else TB_TRY(tune_impl<float>(h, nv, precision, st, in, out));
        }
    }
    auto launch_all = [&](bool prof) -> tb_status {
        if (precision == TB_PREC_C128) return run_chain<double>(h, adjoint, in, out, nv, st, prof, precision);
        return run_chain<float>(h, adjoint, in, out, nv, st, prof, precision);
    };
    const bool prof = h->profiling != 0;
    if (!h->use_graphs || st == nullptr) return launch_all(prof);
    for (auto &g : h->graphs)
        if (g.in == in && g.out == out && g.nv == nv && g.prec == precision && g.adjoint == (int)adjoint &&
            g.stream == st) {
            TB_CK(cudaGraphLaunch(g.exec, st));
            return TB_OK;
        }
    // first call for these arguments: run eagerly once (sets kernel attributes), then capture
    TB_TRY(launch_all(prof));
    cudaGraph_t graph;
    TB_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    tb_status s = launch_all(false);
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s != TB_OK) return s;
    if (e != cudaSuccess) return fail(TB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(TB_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    h->graphs.push_back(GraphEntry{in, out, nv, precision, (int)adjoint, st, exec});
    return TB_OK;
}

}  // namespace

extern "C" tb_status tb_apply(tb_handle h, const void *f, void *u, int64_t nv, int precision, void *stream) {
    return apply_common(h, f, u, nv, precision, stream, false);
}

extern "C" tb_status tb_apply_adjoint(tb_handle h, const void *g, void *v, int64_t nv, int precision, void *stream) {
    return apply_common(h, g, v, nv, precision, stream, true);
}

extern "C" tb_status tb_autotune(tb_handle h, int64_t nv, int precision, void *stream) {
    if (!h) return fail(TB_EINVAL, "handle is NULL");
    if (nv <= 0) return fail(TB_EINVAL, "nv must be positive");
    if (precision < TB_PREC_C128 || precision > TB_PREC_C64_SPLITBF16)
        return fail(TB_EINVAL, "unknown precision");
    if (!(h->precisions & (1u << precision)))
        return fail(TB_EUNSUPPORTED, "handle was built without precision " + std::to_string(precision));
    int64_t N = 1;
    for (int k = 0; k < h->d; ++k) N *= h->n[k];
    TB_TRY(check_nv(N, nv, precision == TB_PREC_C128 ? 16 : 8));
    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice"); }
    TB_TRY(init_device_attrs(h));
    TB_TRY(ensure_workspace(h, nv));
    const size_t bytes = (size_t)N * nv * (precision == TB_PREC_C128 ? 16 : 8);
    void *uin = nullptr, *uout = nullptr;
    TB_CK(cudaMalloc(&uin, bytes));
    if (cudaMalloc(&uout, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(uin);
        return fail(TB_ENOMEM, "tb_autotune: temporary buffers");
    }
    tb_status s = cudaMemsetAsync(uin, 0, bytes, (cudaStream_t)stream) == cudaSuccess ? TB_OK
                                                                                     : fail(TB_ECUDA, "memset");
    if (s == TB_OK) {
        s = precision == TB_PREC_C128 ? tune_impl<double>(h, nv, precision, (cudaStream_t)stream, uin, uout)
                                      : tune_impl<float>(h, nv, precision, (cudaStream_t)stream, uin, uout);
    }
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(uin);
    cudaFree(uout);
    return s;
}

// ---------------------------------------------- partitioned (sharded) apply
namespace {

// One half of Alg. 2 restricted to a range of mid-level multisets:
// half 0 = steps 1 and 2 for the source multisets s in [f0, f1) (user tensor
// -> target-side mid-level tensor, tiles (t, s) for every t); half 1 = step 3
// for the target multisets t in [f0, f1) (mid-level tensor -> user tensor).
// Per-mode level launches (each unit outside the range returns at once).
template <class R>
tb_status run_half(tb_plan *h, int half, const void *in, void *out, int64_t nv, cudaStream_t st, int precision,
                   int64_t f0, int64_t f1) {
    void *B[2] = {h->ws.buf[0], h->ws.buf[1]};
    void *T[2] = {h->ws.mbuf[0], h->ws.mbuf[1]};
    const int Lc = h->Lc;
    if (half == 0) {
        int cur = 0;
        TB_TRY(level_pass<R>(h, Pass::LeafIn, false, 0, 0, in, B[cur], nv, st, T, -1, 0, 0, f0, f1));
        for (int l = 1; l <= Lc; ++l) {
            TB_TRY(level_pass<R>(h, Pass::Split, false, 0, l, B[cur], B[cur ^ 1], nv, st, T, -1, 0, 0, f0, f1));
            cur ^= 1;
        }
        return core_pass<R>(h, false, B[cur], out, nv, st, precision, f0, f1);
    }
    int cur = 0;
    const void *src = in;
    for (int l = Lc; l >= 1; --l) {
        TB_TRY(level_pass<R>(h, Pass::Gather, false, 1, l, src, B[cur], nv, st, T, -1, 0, 0, f0, f1));
        src = B[cur];
        cur ^= 1;
    }
    return level_pass<R>(h, Pass::LeafOut, false, 1, 0, src, out, nv, st, T, -1, 0, 0, f0, f1);
}

tb_status part_common(tb_handle h, int half, const void *in, void *out, int64_t nv, int64_t f0, int64_t f1,
                      int precision, void *stream) {
    if (!h) return fail(TB_EINVAL, "handle is NULL");
    if (nv <= 0) return fail(TB_EINVAL, "nv must be positive");
    if (h->separable) return fail(TB_EUNSUPPORTED, "partitioned applies are built for non-separable handles");
    if (precision != TB_PREC_C128 && precision != TB_PREC_C64)
        return fail(TB_EUNSUPPORTED, "partitioned applies support TB_PREC_C128 and TB_PREC_C64");
    if (!(h->precisions & (1u << precision)))
        return fail(TB_EUNSUPPORTED, "handle was built without precision " + std::to_string(precision));
    const int64_t nF = ipow2(h->d * h->Lc);
    if (f0 < 0 || f1 > nF || f0 > f1) return fail(TB_EINVAL, "multiset range outside [0, 2^(d Lc)]");
    TB_TRY(check_device_ptr(in, "input"));
    TB_TRY(check_device_ptr(out, "output"));
    int64_t N = 1;
    for (int k = 0; k < h->d; ++k) N *= h->n[k];
    TB_TRY(check_nv(N, nv, precision == TB_PREC_C128 ? 16 : 8));
    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice"); }
    TB_TRY(init_device_attrs(h));
    TB_TRY(ensure_workspace(h, nv));
    if (f0 == f1) return TB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == TB_PREC_C128) return run_half<double>(h, half, in, out, nv, st, precision, f0, f1);
    return run_half<float>(h, half, in, out, nv, st, precision, f0, f1);
}

}  // namespace

extern "C" tb_status tb_shard_plan(int64_t nmid, int nranks, int64_t *begin, int64_t *end) {
    if (nmid < 1 || nranks < 1 || !begin || !end) return fail(TB_EINVAL, "nmid, nranks must be positive, arrays non-NULL");
    for (int g = 0; g < nranks; ++g) {
        begin[g] = nmid * g / nranks;
        end[g] = nmid * (g + 1) / nranks;
    }
    return TB_OK;
}

extern "C" tb_status tb_apply_src_part(tb_handle h, const void *f, void *g_mid, int64_t nv, int64_t s_begin,
                                       int64_t s_end, int precision, void *stream) {
    return part_common(h, 0, f, g_mid, nv, s_begin, s_end, precision, stream);
}

extern "C" tb_status tb_apply_tgt_part(tb_handle h, const void *g_mid, void *u, int64_t nv, int64_t t_begin,
                                       int64_t t_end, int precision, void *stream) {
    return part_common(h, 1, g_mid, u, nv, t_begin, t_end, precision, stream);
}

// ------------------------------------------------------- factor export
extern "C" tb_status tb_export_factors(tb_handle h, int side, int level, int mode, int64_t *count, int *rows,
                                       int *cols, int *ranks, int *skel, void *blocks) {
    if (!h || !count || !rows || !cols) return fail(TB_EINVAL, "handle, count, rows and cols must be non-NULL");
    if (h->separable) return fail(TB_EUNSUPPORTED, "tb_export_factors: separable handles store per-mode factors");
    if (side != 0 && side != 1) return fail(TB_EINVAL, "side must be 0 (source) or 1 (target)");
    if (level < 0 || level > h->Lc) return fail(TB_EINVAL, "level out of range");
    if (mode < 0 || mode >= h->d) return fail(TB_EINVAL, "mode out of range");
    const SideLevel &S = side == 0 ? h->src[level] : h->tgt[level];
    *count = S.count[mode];
    *rows = S.R[mode];
    *cols = S.cin[mode];
    if (!ranks && !skel && !blocks) return TB_OK;
    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice"); }
    const int64_t cnt = S.count[mode];
    if (ranks) TB_CK(cudaMemcpy(ranks, S.rank[mode], (size_t)cnt * sizeof(int), cudaMemcpyDeviceToHost));
    if (skel) {
        const size_t w = (size_t)S.R[mode] * sizeof(int), sp = (size_t)S.cap[mode] * sizeof(int);
        TB_CK(cudaMemcpy2D(skel, w, S.skel[mode], sp, w, (size_t)cnt, cudaMemcpyDeviceToHost));
    }
    if (blocks)
        TB_CK(cudaMemcpy(blocks, S.fac64[mode], (size_t)cnt * S.R[mode] * S.cin[mode] * sizeof(c128),
                         cudaMemcpyDeviceToHost));
    return TB_OK;
}

extern "C" tb_status tb_export_cores(tb_handle h, int64_t *pairs, int64_t *entries, int64_t *offsets, int *dims,
                                     void *core) {
    if (!h || !pairs || !entries) return fail(TB_EINVAL, "handle, pairs and entries must be non-NULL");
    if (h->separable) return fail(TB_EUNSUPPORTED, "tb_export_cores: separable handles store per-mode cores");
    *pairs = h->P;
    *entries = h->core_entries;
    if (!offsets && !dims && !core) return TB_OK;
    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice"); }
    if (offsets) TB_CK(cudaMemcpy(offsets, h->core_off, (size_t)(h->P + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (dims) TB_CK(cudaMemcpy(dims, h->core_dims, (size_t)h->P * 2 * h->d * sizeof(int), cudaMemcpyDeviceToHost));
    if (core) {
        if (h->core64) {
            TB_CK(cudaMemcpy(core, h->core64, (size_t)h->core_entries * sizeof(c128), cudaMemcpyDeviceToHost));
        } else {   // built without complex128: the complex64 cores, widened
            std::vector<c64> tmp((size_t)h->core_entries);
            TB_CK(cudaMemcpy(tmp.data(), h->core32, tmp.size() * sizeof(c64), cudaMemcpyDeviceToHost));
            c128 *o = (c128 *)core;
            for (size_t i = 0; i < tmp.size(); ++i) o[i] = c128{(double)tmp[i].x, (double)tmp[i].y};
        }
    }
    return TB_OK;
}

extern "C" tb_status tb_export_order(tb_handle h, int axis, int *perm) {
    if (!h || !perm) return fail(TB_EINVAL, "handle and perm must be non-NULL");
    if (axis < 0 || axis >= h->d) return fail(TB_EINVAL, "axis out of range");
    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice"); }
    TB_CK(cudaMemcpy(perm, h->perm[axis], (size_t)h->n[axis] * sizeof(int), cudaMemcpyDeviceToHost));
    return TB_OK;
}

// ------------------------------------------------- least squares (CGLS)
namespace {

// Device buffers of one tb_cgls call.
struct CglsWork {
    void *r = nullptr, *s = nullptr, *p = nullptr, *q = nullptr;
    double *partial = nullptr, *hist = nullptr;
    CglsScalars *sc = nullptr;
    int *count = nullptr;
    ~CglsWork() {
        for (void *ptr : {r, s, p, q, (void *)partial, (void *)hist, (void *)sc, (void *)count})
            if (ptr) cudaFree(ptr);
    }
};

template <class R>
tb_status cgls_impl(tb_plan *h, const void *b, void *x, int64_t nv, int iters, int precision, bool graph,
                    double *resid, cudaStream_t st) {
    int64_t N = 1;
    for (int k = 0; k < h->d; ++k) N *= h->n[k];
    const size_t bytes = (size_t)N * nv * sizeof(cx<R>);
    CglsWork w;
    for (void **ptr : {&w.r, &w.s, &w.p, &w.q}) TB_CK(cudaMalloc(ptr, bytes));
    TB_CK(cudaMalloc(&w.partial, (size_t)cgls_blocks() * nv * sizeof(double)));
    TB_CK(cudaMalloc(&w.hist, (size_t)(iters + 1) * nv * sizeof(double)));
    TB_CK(cudaMalloc(&w.sc, (size_t)nv * sizeof(CglsScalars)));
    TB_CK(cudaMalloc(&w.count, sizeof(int)));
    TB_CK(cudaMemsetAsync(w.sc, 0, (size_t)nv * sizeof(CglsScalars), st));
    TB_CK(cudaMemsetAsync(w.count, 0, sizeof(int), st));
    TB_CK(cudaMemsetAsync(w.hist, 0, (size_t)(iters + 1) * nv * sizeof(double), st));
    cx<R> *X = (cx<R> *)x, *Rr = (cx<R> *)w.r, *S = (cx<R> *)w.s, *Pp = (cx<R> *)w.p, *Q = (cx<R> *)w.q;
    const cx<R> *B = (const cx<R> *)b;
    const int cap = iters + 1;
    // start: r = b - K x0, s = K^H r, p = s, gamma = ||s||^2 (eager; it also sets
    // every kernel's attributes before any capture)
    TB_TRY(run_chain<R>(h, false, X, Q, nv, st, false, precision));
    TB_CK(launch_cgls_sub<R>(Rr, B, Q, N, (int)nv, w.partial, st));
    TB_CK(launch_cgls_finalize(w.partial, (int)nv, CG_RESID, w.sc, w.hist, w.count, cap, st));
    TB_TRY(run_chain<R>(h, true, Rr, S, nv, st, false, precision));
    TB_CK(launch_cgls_sqnorm<R>(S, N, (int)nv, w.partial, st));
    TB_CK(launch_cgls_finalize(w.partial, (int)nv, CG_GAMMA0, w.sc, w.hist, w.count, cap, st));
    TB_CK(cudaMemcpyAsync(Pp, S, bytes, cudaMemcpyDeviceToDevice, st));
    // one iteration: q = K p, alpha = gamma / ||q||^2, x += alpha p, r -= alpha q,
    // s = K^H r, beta = ||s||^2 / gamma, p = s + beta p, record ||r||
    auto iteration = [&]() -> tb_status {
        TB_TRY(run_chain<R>(h, false, Pp, Q, nv, st, false, precision));
        TB_CK(launch_cgls_sqnorm<R>(Q, N, (int)nv, w.partial, st));
        TB_CK(launch_cgls_finalize(w.partial, (int)nv, CG_ALPHA, w.sc, w.hist, w.count, cap, st));
        TB_CK(launch_cgls_xr<R>(X, Rr, Pp, Q, w.sc, N, (int)nv, w.partial, st));
        TB_CK(launch_cgls_finalize(w.partial, (int)nv, CG_RESID, w.sc, w.hist, w.count, cap, st));
        TB_TRY(run_chain<R>(h, true, Rr, S, nv, st, false, precision));
        TB_CK(launch_cgls_sqnorm<R>(S, N, (int)nv, w.partial, st));
        TB_CK(launch_cgls_finalize(w.partial, (int)nv, CG_BETA, w.sc, w.hist, w.count, cap, st));
        TB_CK(launch_cgls_p<R>(Pp, S, w.sc, N, (int)nv, st));
        return TB_OK;
    };
    if (graph && iters > 0) {
        cudaGraph_t g;
        TB_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        tb_status s = iteration();
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (s != TB_OK) return s;
        if (e != cudaSuccess) return fail(TB_ECUDA, std::string("tb_cgls capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(TB_ECUDA, std::string("tb_cgls instantiate: ") + cudaGetErrorString(e));
        cudaError_t le = cudaSuccess;
        for (int it = 0; it < iters && le == cudaSuccess; ++it) le = cudaGraphLaunch(exec, st);
        cudaError_t se = cudaStreamSynchronize(st);
        cudaGraphExecDestroy(exec);
        if (le != cudaSuccess) return fail(TB_ECUDA, std::string("tb_cgls replay: ") + cudaGetErrorString(le));
        if (se != cudaSuccess) return fail(TB_ECUDA, std::string("tb_cgls: ") + cudaGetErrorString(se));
    } else {
        for (int it = 0; it < iters; ++it) TB_TRY(iteration());
    }
    if (resid) TB_CK(cudaMemcpyAsync(resid, w.hist, (size_t)(iters + 1) * nv * sizeof(double), cudaMemcpyDeviceToHost, st));
    TB_CK(cudaStreamSynchronize(st));
    return TB_OK;
}

}  // namespace

extern "C" tb_status tb_cgls(tb_handle h, const void *b, void *x, int64_t nv, int iters, int precision,
                             int use_graph, double *resid, void *stream) {
    if (!h) return fail(TB_EINVAL, "handle is NULL");
    if (nv <= 0) return fail(TB_EINVAL, "nv must be positive");
    if (iters < 0) return fail(TB_EINVAL, "iters must be >= 0");
    if (nv > cgls_max_nv()) return fail(TB_EUNSUPPORTED, "tb_cgls supports nv <= " + std::to_string(cgls_max_nv()));
    if (precision < TB_PREC_C128 || precision > TB_PREC_C64_SPLITBF16)
        return fail(TB_EINVAL, "unknown precision");
    if (!(h->precisions & (1u << precision)))
        return fail(TB_EUNSUPPORTED, "handle was built without precision " + std::to_string(precision));
    TB_TRY(check_device_ptr(b, "b"));
    TB_TRY(check_device_ptr(x, "x"));
    int64_t N = 1;
    for (int k = 0; k < h->d; ++k) N *= h->n[k];
    const size_t es = precision == TB_PREC_C128 ? 16 : 8;
    TB_TRY(check_nv(N, nv, es));
    const char *a0 = (const char *)b, *b0 = (const char *)x;
    if (a0 < b0 + (size_t)N * nv * es && b0 < a0 + (size_t)N * nv * es)
        return fail(TB_EINVAL, "b and x overlap");
    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice"); }
    TB_TRY(init_device_attrs(h));
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    TB_CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return fail(TB_EINVAL, "tb_cgls cannot run inside a stream capture");
    TB_TRY(ensure_workspace(h, nv));
    // launch-shape tuning on temporary buffers, so that x keeps the caller's start
    if (h->autotune && !is_tuned(h, nv, precision)) TB_TRY(tb_autotune(h, nv, precision, stream));
    // graphs need a capturable stream: the legacy default stream is not one
    const bool graph = use_graph != 0 && st != nullptr;
    if (precision == TB_PREC_C128) return cgls_impl<double>(h, b, x, nv, iters, precision, graph, resid, st);
    return cgls_impl<float>(h, b, x, nv, iters, precision, graph, resid, st);
}

// ------------------------------------------------- apply without allocating
// The scratch area of tb_apply_noalloc: a fixed device array compiled into the
// library.  In host code `g_noalloc_scratch` names a host-side stand-in, not
// device memory, so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached here.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TB_NOALLOC_SCRATCH_BYTES];
static void *g_noalloc_addr[64] = {nullptr};
static std::mutex g_noalloc_mu;

extern "C" tb_status tb_apply_noalloc(tb_handle h, const void *f, void *u, int64_t nv, int precision,
                                      void *stream) {
    if (!h) return fail(TB_EINVAL, "handle is NULL");
    if (nv <= 0) return fail(TB_EINVAL, "nv must be positive");
    if (precision < TB_PREC_C128 || precision > TB_PREC_C64_SPLITBF16)
        return fail(TB_EINVAL, "unknown precision");
    if (!(h->precisions & (1u << precision)))
        return fail(TB_EUNSUPPORTED, "handle was built without precision " + std::to_string(precision));
    TB_TRY(check_device_ptr(f, "f"));
    TB_TRY(check_device_ptr(u, "u"));
    int64_t N = 1;
    for (int k = 0; k < h->d; ++k) N *= h->n[k];
    const size_t es = precision == TB_PREC_C128 ? 16 : 8;
    TB_TRY(check_nv(N, nv, es));
    // reject by division first, so that no product below can wrap: the
    // scratch needs (2 level tensors + 2 mode intermediates) x nv x es bytes
    {
        const uint64_t per_rhs =
            (uint64_t)es * (2 * (uint64_t)h->level_max + (uint64_t)h->mode_max[0] + (uint64_t)h->mode_max[1]);
        if (per_rhs > 0 && (uint64_t)nv > (uint64_t)TB_NOALLOC_SCRATCH_BYTES / per_rhs)
            return fail(TB_EUNSUPPORTED, "tb_apply_noalloc: nv = " + std::to_string(nv) + " needs " +
                                             std::to_string(per_rhs) + " bytes of scratch per RHS; the fixed scratch holds " +
                                             std::to_string((size_t)TB_NOALLOC_SCRATCH_BYTES) + " (reduce nv)");
    }
    const char *a0 = (const char *)f, *b0 = (const char *)u;
    if (a0 < b0 + (size_t)N * nv * es && b0 < a0 + (size_t)N * nv * es)
        return fail(TB_EINVAL, "input and output overlap");
    // two level tensors (ping-pong) of the largest level and the two mode
    // intermediates, each 256-byte aligned
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t half = al((size_t)h->level_max * (size_t)nv * es);
    const size_t mreg[2] = {al((size_t)h->mode_max[0] * (size_t)nv * es), al((size_t)h->mode_max[1] * (size_t)nv * es)};
    const size_t total = 2 * half + mreg[0] + mreg[1];
    if (total > (size_t)TB_NOALLOC_SCRATCH_BYTES)
        return fail(TB_EUNSUPPORTED, "tb_apply_noalloc needs " + std::to_string(total) +
                                         " bytes of scratch; the fixed scratch holds " +
                                         std::to_string((size_t)TB_NOALLOC_SCRATCH_BYTES) + " (reduce nv)");
    if (h->device < 0 || h->device >= 64) return fail(TB_EINVAL, "device ordinal out of range");
    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice"); }
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[h->device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return fail(TB_ECUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch: ") +
                                          cudaGetErrorString(e));
            }
            g_noalloc_addr[h->device] = p;
        }
        base = g_noalloc_addr[h->device];
    }
    if (g_smem_optin == 0) {
        int v = 0, sms = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        g_num_sms = sms;
        g_smem_optin = (size_t)v;
    }
    unsigned char *sb = (unsigned char *)base;
    void *bufs[4] = {sb, sb + half, sb + 2 * half, sb + 2 * half + mreg[0]};
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == TB_PREC_C128) return run_chain<double>(h, false, f, u, nv, st, false, precision, bufs, mreg[0]);
    return run_chain<float>(h, false, f, u, nv, st, false, precision, bufs, mreg[0]);
}

extern "C" tb_status tb_apply_host(tb_handle h, const void *f, void *u, int64_t nv, int precision) {
    if (!h || !f || !u) return fail(TB_EINVAL, "handle, f and u must be non-NULL");
    if (nv <= 0) return fail(TB_EINVAL, "nv must be positive");
    int64_t N = 1;
    for (int k = 0; k < h->d; ++k) N *= h->n[k];
    const size_t es = precision == TB_PREC_C128 ? 16 : 8;
    TB_TRY(check_nv(N, nv, es));
    const size_t bytes = (size_t)N * nv * es;
    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice"); }
    if (bytes > h->ws.host_bytes) {
        TB_CK(cudaDeviceSynchronize());
        if (h->ws.host_in) cudaFree(h->ws.host_in);
        if (h->ws.host_out) cudaFree(h->ws.host_out);
        h->ws.host_in = h->ws.host_out = nullptr;
        h->ws.host_bytes = 0;
        TB_CK(cudaMalloc(&h->ws.host_in, bytes));
        TB_CK(cudaMalloc(&h->ws.host_out, bytes));
        h->ws.host_bytes = bytes;
    }
    TB_CK(cudaMemcpy(h->ws.host_in, f, bytes, cudaMemcpyHostToDevice));
    TB_TRY(apply_common(h, h->ws.host_in, h->ws.host_out, nv, precision, nullptr, false));
    TB_CK(cudaMemcpy(u, h->ws.host_out, bytes, cudaMemcpyDeviceToHost));
    return TB_OK;
}

extern "C" tb_status tb_apply_host_batch(tb_handle h, const void *const *f, void *const *u, int64_t count,
                                         int64_t nv, int precision) {
    if (!h || !f || !u) return fail(TB_EINVAL, "handle, f and u must be non-NULL");
    if (count < 1) return fail(TB_EINVAL, "count must be positive");
    if (nv <= 0) return fail(TB_EINVAL, "nv must be positive");
    for (int64_t i = 0; i < count; ++i)
        if (!f[i] || !u[i]) return fail(TB_EINVAL, "f[i] and u[i] must be non-NULL");
    int64_t N = 1;
    for (int k = 0; k < h->d; ++k) N *= h->n[k];
    TB_TRY(check_nv(N, nv, precision == TB_PREC_C128 ? 16 : 8));
    const size_t bytes = (size_t)N * nv * (precision == TB_PREC_C128 ? 16 : 8);
    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); return fail(TB_ECUDA, "cudaSetDevice"); }
    HostPipe &P = h->pipe;
    if (!P.s[0]) {
        for (int i = 0; i < 3; ++i) TB_CK(cudaStreamCreateWithFlags(&P.s[i], cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b)
            for (cudaEvent_t *e : {&P.in_ready[b], &P.in_free[b], &P.out_ready[b], &P.out_free[b]})
                TB_CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    if (bytes > P.bytes) {
        for (int i = 0; i < 3; ++i) TB_CK(cudaStreamSynchronize(P.s[i]));
        for (int b = 0; b < 2; ++b) {
            if (P.din[b]) cudaFree(P.din[b]);
            if (P.dout[b]) cudaFree(P.dout[b]);
            P.din[b] = P.dout[b] = nullptr;
        }
        P.bytes = 0;
        for (int b = 0; b < 2; ++b) {
            TB_CK(cudaMalloc(&P.din[b], bytes));
            TB_CK(cudaMalloc(&P.dout[b], bytes));
        }
        P.bytes = bytes;
    }
    auto body = [&]() -> tb_status {
        for (int64_t i = 0; i < count; ++i) {
            const int b = (int)(i & 1);
            // input i into din[b] once the apply of input i - 2 has read it
            if (i >= 2) TB_CK(cudaStreamWaitEvent(P.s[0], P.in_free[b], 0));
            TB_CK(cudaMemcpyAsync(P.din[b], f[i], bytes, cudaMemcpyHostToDevice, P.s[0]));
            TB_CK(cudaEventRecord(P.in_ready[b], P.s[0]));
            // apply once the input is there and result i - 2 has left dout[b]
            TB_CK(cudaStreamWaitEvent(P.s[1], P.in_ready[b], 0));
            if (i >= 2) TB_CK(cudaStreamWaitEvent(P.s[1], P.out_free[b], 0));
            TB_TRY(apply_common(h, P.din[b], P.dout[b], nv, precision, P.s[1], false));
            TB_CK(cudaEventRecord(P.in_free[b], P.s[1]));
            TB_CK(cudaEventRecord(P.out_ready[b], P.s[1]));
            // result i back to the host
            TB_CK(cudaStreamWaitEvent(P.s[2], P.out_ready[b], 0));
            TB_CK(cudaMemcpyAsync(u[i], P.dout[b], bytes, cudaMemcpyDeviceToHost, P.s[2]));
            TB_CK(cudaEventRecord(P.out_free[b], P.s[2]));
        }
        return TB_OK;
    };
    const tb_status st = body();
    for (int i = 0; i < 3; ++i) {
        const cudaError_t e = cudaStreamSynchronize(P.s[i]);
        if (e != cudaSuccess && st == TB_OK) return fail(TB_ECUDA, std::string("host batch: ") + cudaGetErrorString(e));
    }
    return st;
}

extern "C" tb_status tb_profile_enable(tb_handle h, int on) {
    if (!h) return fail(TB_EINVAL, "handle is NULL");
    h->profiling = on ? 1 : 0;
    return TB_OK;
}

extern "C" tb_status tb_profile_stats(tb_handle h, tb_pass_stat *stats, int cap, int *count) {
    if (!h || !count || (cap > 0 && !stats)) return fail(TB_EINVAL, "handle, stats and count must be non-NULL");
    std::vector<tb_pass_stat> agg;
    tb_status st = TB_OK;
    for (auto &r : h->prof) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.e0, r.e1);
        if (e != cudaSuccess && st == TB_OK) st = fail(TB_ECUDA, std::string("profile events: ") + cudaGetErrorString(e));
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
        tb_pass_stat *hit = nullptr;
        for (auto &a : agg)
            if (!std::strcmp(a.name, r.name) && a.level == r.level && a.adjoint == r.adjoint) hit = &a;
        if (!hit) {
            tb_pass_stat z;
            std::memset(&z, 0, sizeof(z));
            std::snprintf(z.name, sizeof(z.name), "%s", r.name);
            z.level = r.level;
            z.adjoint = r.adjoint;
            agg.push_back(z);
            hit = &agg.back();
        }
        hit->launches += 1;
        hit->kernels += r.kernels;
        hit->ms_total += ms;
        hit->bytes = r.bytes;
        hit->flops = r.flops;
    }
    h->prof.clear();
    *count = (int)std::min<size_t>(agg.size(), (size_t)std::max(cap, 0));
    for (int i = 0; i < *count; ++i) stats[i] = agg[(size_t)i];
    return st;
}

// Host-side check of the register-resident separable chains (tb_sep.cu),
// compiled by nvcc and run on the CPU by tests/test_sep_chain_host.py.
//
// 1. sepr_col reproduces the column pattern of the CSR steps that the builder
//    assembles from the factor blocks (source transfers W_l, Kronecker core,
//    target transfers P_l) for Lc = 1..3 and ranks 1..8.
// 2. The complex64 paired-FMA chains (seprf_chain, forward and adjoint, one or
//    two fibers), the scalar chains (sepr_chain, complex64 and complex128) and
//    the fused pair phases (seprf2_phase1/2, padded tile) equal the dense
//    product of their step matrices built from sepr_col, with the load / store
//    positions as permutations.
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../paper_2411_03029_gb300/csrc/tb_sep.cu"

namespace tb {
cudaError_t set_smem_once(const void *, size_t) { return cudaSuccess; }
}  // namespace tb
using namespace tb;
using C = std::complex<double>;

static double rnd() { return (double)rand() / RAND_MAX - 0.5; }

static int check_pattern() {
    int bad = 0;
    for (int Lc = 1; Lc <= 3; ++Lc)
        for (int R = 1; R <= 8; R *= 2) {
            const int nb = 1 << Lc, N = R * nb * nb;
            auto esrc = [&](int l, int s, int tau, int nu, int a) { return ((((s << l) + tau) << (Lc - l)) + nu) * R + a; };
            auto etgt = [&](int l, int t, int nu, int tau, int a) { return ((((t << l) + nu) << (Lc - l)) + tau) * R + a; };
            int st = 0;
            for (int l = 1; l <= Lc; ++l, ++st) {
                const int ns = 1 << (Lc - l);
                int row = 0;
                for (int s = 0; s < nb; ++s)
                    for (int tau = 0; tau < (1 << l); ++tau)
                        for (int nu = 0; nu < ns; ++nu)
                            for (int a = 0; a < R; ++a, ++row) {
                                if (row != esrc(l, s, tau, nu, a)) ++bad;
                                int j = 0;
                                for (int c = 0; c < 2; ++c)
                                    for (int q = 0; q < R; ++q, ++j)
                                        if (sepr_col(Lc, R, st, row, j) != esrc(l - 1, s, tau >> 1, 2 * nu + c, q)) ++bad;
                            }
                if (row != N) ++bad;
            }
            {
                int row = 0;
                for (int t = 0; t < nb; ++t)
                    for (int s = 0; s < nb; ++s)
                        for (int a = 0; a < R; ++a, ++row)
                            for (int q = 0; q < R; ++q)
                                if (sepr_col(Lc, R, st, row, q) != esrc(Lc, s, t, 0, q)) ++bad;
                ++st;
            }
            for (int l = Lc; l >= 1; --l, ++st) {
                const int ns = 1 << (Lc - l);
                int row = 0;
                for (int t = 0; t < nb; ++t)
                    for (int pn = 0; pn < (1 << (l - 1)); ++pn)
                        for (int tp = 0; tp < 2 * ns; ++tp)
                            for (int a = 0; a < R; ++a, ++row) {
                                int j = 0;
                                for (int c = 0; c < 2; ++c)
                                    for (int q = 0; q < R; ++q, ++j)
                                        if (sepr_col(Lc, R, st, row, j) != etgt(l, t, 2 * pn + c, tp >> 1, q)) ++bad;
                            }
                if (row != N) ++bad;
            }
            if (sepr_ncoef(Lc, R) != N * R * (4 * Lc + 1)) ++bad;
        }
    printf("pattern mismatches: %d\n", bad);
    return bad;
}

// dense N x N operator of a chain (forward, or its conjugate transpose)
template <int LC, int RK>
static std::vector<C> dense_chain(const std::vector<C> &cd, bool adj) {
    constexpr int N = RK << (2 * LC);
    std::vector<C> M(N * N, 0.0);
    for (int i = 0; i < N; ++i) M[i * N + i] = 1.0;
    for (int i = 0; i <= 2 * LC; ++i) {
        const int st = adj ? 2 * LC - i : i, K = sepr_width(LC, RK, st), off = sepr_off(LC, RK, st);
        std::vector<C> S(N * N, 0.0), T(N * N, 0.0);
        for (int e = 0; e < N; ++e)
            for (int j = 0; j < K; ++j) S[e * N + sepr_col(LC, RK, st, e, j)] += cd[off + e * K + j];
        if (adj) {
            std::vector<C> H(N * N);
            for (int r = 0; r < N; ++r)
                for (int c = 0; c < N; ++c) H[c * N + r] = std::conj(S[r * N + c]);
            S = H;
        }
        for (int r = 0; r < N; ++r)
            for (int c = 0; c < N; ++c)
                for (int m = 0; m < N; ++m) T[r * N + c] += S[r * N + m] * M[m * N + c];
        M = T;
    }
    return M;
}

static std::vector<float4> pack(const std::vector<C> &cd, bool adj) {
    std::vector<float4> f(cd.size());
    for (size_t i = 0; i < cd.size(); ++i) {
        const float re = (float)cd[i].real(), im = (float)cd[i].imag();
        f[i] = make_float4(re, re, im, adj ? -im : im);
    }
    return f;
}

template <int RK, int F>
static int check_chain() {
    constexpr int LC = 1, N = RK << 2, NC = sepr_ncoef(LC, RK);
    std::vector<C> cd(NC);
    for (auto &c : cd) c = C(rnd(), rnd());
    int bad = 0;
    for (int adj = 0; adj < 2; ++adj) {
        std::vector<float4> cf = pack(cd, adj);
        float2 x[F][N];
        std::vector<C> xr(F * N);
        for (int f = 0; f < F; ++f)
            for (int p = 0; p < N; ++p) {
                xr[f * N + p] = C(rnd(), rnd());
                x[f][p] = make_float2((float)xr[f * N + p].real(), (float)xr[f * N + p].imag());
            }
        if (adj) seprf_chain<LC, RK, true, F>(cf.data(), x);
        else seprf_chain<LC, RK, false, F>(cf.data(), x);
        const std::vector<C> M = dense_chain<LC, RK>(cd, adj);
        double num = 0, den = 0;
        for (int f = 0; f < F; ++f)
            for (int r = 0; r < N; ++r) {
                C acc = 0;
                for (int c = 0; c < N; ++c) acc += M[r * N + c] * xr[f * N + c];
                num += std::norm(C(x[f][r].x, x[f][r].y) - acc);
                den += std::norm(acc);
            }
        const double err = std::sqrt(num / den);
        printf("chain rk %d fibers %d adjoint %d: rel err %.2e\n", RK, F, adj, err);
        bad += err > 1e-5;
    }
    return bad;
}

// the scalar chain (sepr_chain: complex128, and the complex64 prefetching form)
template <class R, int RK>
static int check_scalar_chain() {
    constexpr int LC = 1, N = RK << 2, NC = sepr_ncoef(LC, RK);
    std::vector<C> cd(NC);
    for (auto &c : cd) c = C(rnd(), rnd());
    std::vector<cx<R>> cs(NC);
    for (int i = 0; i < NC; ++i) cs[i] = {(R)cd[i].real(), (R)cd[i].imag()};
    int bad = 0;
    for (int adj = 0; adj < 2; ++adj) {
        cx<R> x[N];
        std::vector<C> xr(N);
        for (int p = 0; p < N; ++p) {
            xr[p] = C(rnd(), rnd());
            x[p] = {(R)xr[p].real(), (R)xr[p].imag()};
        }
        if (adj) sepr_chain<R, LC, RK, true>(cs.data(), x);
        else sepr_chain<R, LC, RK, false>(cs.data(), x);
        const std::vector<C> M = dense_chain<LC, RK>(cd, adj);
        double num = 0, den = 0;
        for (int r = 0; r < N; ++r) {
            C acc = 0;
            for (int c = 0; c < N; ++c) acc += M[r * N + c] * xr[c];
            num += std::norm(C(x[r].x, x[r].y) - acc);
            den += std::norm(acc);
        }
        const double err = std::sqrt(num / den);
        printf("scalar chain rk %d bytes %zu adjoint %d: rel err %.2e\n", RK, sizeof(R), adj, err);
        bad += err > (sizeof(R) == 4 ? 1e-5 : 1e-13);
    }
    return bad;
}

template <int RK>
static int check_pair(int64_t outer, int64_t inner, bool adj) {
    constexpr int LC = 1, N = RK << 2, NC = sepr_ncoef(LC, RK);
    std::vector<C> ca(NC), cb(NC);
    for (int i = 0; i < NC; ++i) {
        ca[i] = C(rnd(), rnd());
        cb[i] = C(rnd(), rnd());
    }
    const std::vector<float4> fa = pack(ca, adj), fb = pack(cb, adj);
    std::vector<int> pa(N), pb(N), qa(N), qb(N);
    for (int i = 0; i < N; ++i) pa[i] = pb[i] = qa[i] = qb[i] = i;
    for (int i = N - 1; i > 0; --i) {
        std::swap(pa[i], pa[rand() % (i + 1)]);
        std::swap(pb[i], pb[rand() % (i + 1)]);
        std::swap(qa[i], qa[rand() % (i + 1)]);
        std::swap(qb[i], qb[rand() % (i + 1)]);
    }
    const int64_t total = outer * N * N * inner;
    std::vector<float2> in(total), out(total, make_float2(1e30f, 1e30f));
    std::vector<C> inc(total);
    for (int64_t i = 0; i < total; ++i) {
        inc[i] = C(rnd(), rnd());
        in[i] = make_float2((float)inc[i].real(), (float)inc[i].imag());
    }
    SepReg2Args<float> a;
    memset(&a, 0, sizeof(a));
    a.lc = 1;
    a.rk = RK;
    a.outer = outer;
    a.inner = inner;
    int lq = 0;
    while ((2 << lq) * N <= 128 && ((int64_t)2 << lq) <= inner) ++lq;
    a.lq = lq;
    a.q = 1 << lq;
    a.nchunks = (inner + a.q - 1) / a.q;
    a.in = (const cx<float> *)in.data();
    a.out = (cx<float> *)out.data();
    for (int p = 0; p < N; ++p) {
        a.ld_a[p] = pa[p];
        a.st_a[p] = qa[p];
        a.ld_b[p] = pb[p];
        a.st_b[p] = qb[p];
    }
    std::vector<float2> tile(N * ((N << lq) + SEPR2_PAD));
    const int T = N << lq;
    for (int64_t blk = 0; blk < outer * a.nchunks; ++blk) {
        for (int t = 0; t < T; ++t) {
            if (adj) seprf2_phase1<1, RK, true>(a, fb.data(), tile.data(), blk, t);
            else seprf2_phase1<1, RK, false>(a, fb.data(), tile.data(), blk, t);
        }
        for (int t = 0; t < T; ++t) {
            if (adj) seprf2_phase2<1, RK, true>(a, fa.data(), tile.data(), blk, t);
            else seprf2_phase2<1, RK, false>(a, fa.data(), tile.data(), blk, t);
        }
    }
    // mode operator: forward y = chain(x[ld]), out[st] = y; the adjoint swaps ld and st
    auto op = [&](const std::vector<C> &cd, const std::vector<int> &ld, const std::vector<int> &st) {
        const std::vector<C> Ch = dense_chain<LC, RK>(cd, adj);
        std::vector<C> M(N * N, 0.0);
        const std::vector<int> &L = adj ? st : ld, &S = adj ? ld : st;
        for (int p = 0; p < N; ++p)
            for (int q = 0; q < N; ++q) M[S[p] * N + L[q]] += Ch[p * N + q];
        return M;
    };
    const std::vector<C> Ma = op(ca, pa, qa), Mb = op(cb, pb, qb);
    double num = 0, den = 0;
    for (int64_t o = 0; o < outer; ++o)
        for (int ia = 0; ia < N; ++ia)
            for (int ib = 0; ib < N; ++ib)
                for (int64_t q = 0; q < inner; ++q) {
                    C acc = 0;
                    for (int ja = 0; ja < N; ++ja)
                        for (int jb = 0; jb < N; ++jb)
                            acc += Ma[ia * N + ja] * Mb[ib * N + jb] * inc[((o * N + ja) * N + jb) * inner + q];
                    const float2 g = out[((o * N + ia) * N + ib) * inner + q];
                    num += std::norm(C(g.x, g.y) - acc);
                    den += std::norm(acc);
                }
    const double err = std::sqrt(num / den);
    printf("pair rk %d outer %ld inner %ld adjoint %d (Q %d): rel err %.2e\n", RK, (long)outer, (long)inner, (int)adj,
           a.q, err);
    return err > 1e-5;
}

int main() {
    srand(12345);
    int bad = check_pattern();
    bad += check_chain<1, 2>() + check_chain<2, 2>() + check_chain<4, 2>() + check_chain<4, 1>() + check_chain<8, 1>();
    bad += check_scalar_chain<float, 1>() + check_scalar_chain<float, 2>() + check_scalar_chain<float, 4>() +
           check_scalar_chain<float, 8>() + check_scalar_chain<double, 1>() + check_scalar_chain<double, 2>();
    for (int adj = 0; adj < 2; ++adj)
        bad += check_pair<1>(2, 3, adj) + check_pair<2>(3, 8, adj) + check_pair<4>(2, 8, adj) +
               check_pair<4>(1, 21, adj) + check_pair<8>(2, 5, adj) + check_pair<4>(3, 1, adj);
    printf("failures: %d\n", bad);
    return bad != 0;
}

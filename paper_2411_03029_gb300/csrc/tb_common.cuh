// Internal definitions shared by the CUDA translation units of the tensor
// butterfly library: complex arithmetic, FP64 kernel evaluation, index helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tb.h"

#define TB_DEV __device__ __forceinline__
#define TB_HD __host__ __device__ __forceinline__

namespace tb {

constexpr int MAXD = TB_MAX_D;
constexpr int MAXL = TB_MAX_LEVELS;

// ---------------------------------------------------------------- complex
template <class R>
struct alignas(2 * sizeof(R)) cx {
    R x, y;
};
using c64 = cx<float>;
using c128 = cx<double>;

template <class R> TB_HD cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <class R> TB_HD cx<R> operator+(cx<R> a, cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <class R> TB_HD cx<R> operator-(cx<R> a, cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <class R> TB_HD cx<R> operator*(cx<R> a, cx<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class R> TB_HD cx<R> operator*(R s, cx<R> b) { return {s * b.x, s * b.y}; }
template <class R> TB_HD cx<R> conj(cx<R> a) { return {a.x, -a.y}; }
template <class R> TB_HD R norm2(cx<R> a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
template <class R> TB_HD void cmac(cx<R> &acc, cx<R> a, cx<R> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <class R> TB_HD void cmac_conj(cx<R> &acc, cx<R> a, cx<R> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

// Two consecutive complex values; one 16-byte vector load for complex64 (the
// caller guarantees 16-byte alignment of p).
TB_DEV void ld2(const cx<float> *p, cx<float> &a, cx<float> &b) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = cx<float>{v.x, v.y};
    b = cx<float>{v.z, v.w};
}
TB_DEV void ld2(const cx<double> *p, cx<double> &a, cx<double> &b) {
    a = p[0];
    b = p[1];
}

// ---------------------------------------------------------------- kernels
// Kernel descriptor as seen by device code.  For HELMHOLTZ, p[1] holds the
// squared perpendicular offset h^2 and p[2] holds kappa / (2 pi), so that the
// phase is formed in cycles.
struct KernelSpec {
    int kind;
    double p[4];
};

// K(x, y) in FP64.  The phase is accumulated in FP64 and reduced to the nearest
// integer number of cycles before the complex exponential (sincospi), so large
// oscillatory phases keep full relative accuracy.
TB_DEV c128 eval_kernel(const KernelSpec &ks, int d, const double *x, const double *y) {
    double s, c;
    if (ks.kind == TB_KERNEL_FOURIER) {
        // exp(-2 pi i x.y)
        double ph = 0.0;
        for (int k = 0; k < d; ++k) ph = fma(x[k], y[k], ph);
        ph -= rint(ph);
        sincospi(2.0 * ph, &s, &c);
        return {c, -s};
    } else if (ks.kind == TB_KERNEL_HELMHOLTZ) {
        // exp(i kappa rho) / rho
        double r2 = 0.0;
        for (int k = 0; k < d; ++k) {
            double t = x[k] - y[k];
            r2 = fma(t, t, r2);
        }
        double rho = sqrt(r2 + ks.p[1]);
        double ph = ks.p[2] * rho;
        ph -= rint(ph);
        sincospi(2.0 * ph, &s, &c);
        double inv = 1.0 / rho;
        return {c * inv, s * inv};
    } else if (ks.kind == TB_KERNEL_RADON_ANISO) {
        // exp(2 pi i (x.xi + sqrt(c1^2 xi_1^2 + c2^2 xi_2^2))), d = 2
        const double s1 = sinpi(2.0 * x[0]), s2 = sinpi(2.0 * x[1]);
        const double o1 = cospi(2.0 * x[0]), o2 = cospi(2.0 * x[1]);
        const double c1 = ks.p[0] + ks.p[1] * s1 * s2, c2 = ks.p[2] + ks.p[3] * o1 * o2;
        const double a1 = c1 * y[0], a2 = c2 * y[1];
        double xy = fma(x[0], y[0], x[1] * y[1]);
        double ph = xy - rint(xy);
        double ph2 = sqrt(fma(a1, a1, a2 * a2));
        ph2 -= rint(ph2);
        ph += ph2;
        sincospi(2.0 * ph, &s, &c);
        return {c, s};
    } else {
        // exp(2 pi i (x.xi + c(x) |xi|)),  c(x) = a + b prod_k sin(2 pi x_k)
        double xy = 0.0, yy = 0.0, sp = 1.0;
        for (int k = 0; k < d; ++k) {
            xy = fma(x[k], y[k], xy);
            yy = fma(y[k], y[k], yy);
            sp *= sinpi(2.0 * x[k]);
        }
        double cf = ks.p[0] + ks.p[1] * sp;
        double ph = xy - rint(xy);
        double ph2 = cf * sqrt(yy);
        ph2 -= rint(ph2);
        ph += ph2;
        sincospi(2.0 * ph, &s, &c);
        return {c, s};
    }
}

// Integer helpers
TB_HD int64_t ipow2(int e) { return (int64_t)1 << e; }

}  // namespace tb

// Measured FMA throughput of the device (tb_alu_peak): the denominator of the
// ALU roofline of the apply's CUDA-core kernels.  Each thread runs CHAINS
// independent multiply-add recurrences x <- x * a + b for ITERS steps (no
// data movement, enough independent chains to hide the pipe latency), on a
// grid of several blocks per SM; one warm-up launch, then one launch timed
// with CUDA events.  A thread stores the sum of its chains, so nothing is
// dead code.
#include <string>

#include "tb_kernels.cuh"

namespace tb {
namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_ITERS = 4096;

template <class T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(T a, T b, T *out) {
    T x[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < PEAK_ITERS; ++it) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
    out[blockIdx.x * PEAK_THREADS + threadIdx.x] = s;
}

template <class T>
cudaError_t time_peak(cudaStream_t st, double &tflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8;
    T *out = nullptr;
    e = cudaMalloc(&out, (size_t)blocks * PEAK_THREADS * sizeof(T));
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    // a and b keep x bounded (|a| < 1), so no chain overflows
    const T a = (T)0.999, b = (T)1e-4;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fma_peak<T><<<blocks, PEAK_THREADS, 0, st>>>(a, b, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        k_fma_peak<T><<<blocks, PEAK_THREADS, 0, st>>>(a, b, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    const double fmas = (double)blocks * PEAK_THREADS * PEAK_CHAINS * PEAK_ITERS;
    tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace
}  // namespace tb

extern "C" tb_status tb_alu_peak(int precision, void *cuda_stream, double *tflops) {
    if (!tflops) return tb::fail_status(TB_EINVAL, "tflops must be non-NULL");
    if (precision != TB_PREC_C64 && precision != TB_PREC_C128)
        return tb::fail_status(TB_EINVAL, "tb_alu_peak: precision must be TB_PREC_C64 (FP32) or TB_PREC_C128 (FP64)");
    double t = 0.0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e = precision == TB_PREC_C64 ? tb::time_peak<float>(st, t) : tb::time_peak<double>(st, t);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return tb::fail_status(TB_ECUDA, std::string("tb_alu_peak: ") + cudaGetErrorString(e));
    }
    *tflops = t;
    return TB_OK;
}

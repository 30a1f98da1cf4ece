// Level passes as one launch per mode product (k_mode, tb_mode.cuh): the
// launchers without rank bounds or column slices, and the dispatcher.
#include <type_traits>

#include "tb_mode.cuh"

namespace tb {

extern template cudaError_t launch_mode_rk<float, true, false>(int, int, int, const ModeArgs<float> &, cudaStream_t);
extern template cudaError_t launch_mode_rk<double, true, false>(int, int, int, const ModeArgs<double> &,
                                                                cudaStream_t);
extern template cudaError_t launch_mode_rk<float, false, true>(int, int, int, const ModeArgs<float> &, cudaStream_t);
extern template cudaError_t launch_mode_rk<float, true, true>(int, int, int, const ModeArgs<float> &, cudaStream_t);
template cudaError_t launch_mode_rk<float, false, false>(int, int, int, const ModeArgs<float> &, cudaStream_t);
template cudaError_t launch_mode_rk<double, false, false>(int, int, int, const ModeArgs<double> &, cudaStream_t);

template <class R>
cudaError_t launch_mode(int in_kind, int out_kind, int ob, int rank, const ModeArgs<R> &a, cudaStream_t st) {
    if (a.sub > 1) {   // column slices: complex64 only
        if constexpr (std::is_same<R, float>::value)
            return rank ? launch_mode_rk<R, true, true>(in_kind, out_kind, ob, a, st)
                        : launch_mode_rk<R, false, true>(in_kind, out_kind, ob, a, st);
        return cudaErrorInvalidValue;
    }
    return rank ? launch_mode_rk<R, true, false>(in_kind, out_kind, ob, a, st)
                : launch_mode_rk<R, false, false>(in_kind, out_kind, ob, a, st);
}

int mode_cols_per_thread() { return MODE_NC; }

template cudaError_t launch_mode<float>(int, int, int, int, const ModeArgs<float> &, cudaStream_t);
template cudaError_t launch_mode<double>(int, int, int, int, const ModeArgs<double> &, cudaStream_t);

}  // namespace tb

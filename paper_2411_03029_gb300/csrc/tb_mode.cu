// Level passes as one launch per mode product (k_mode, tb_mode.cuh): the
// launchers without rank bounds, and the dispatcher.
#include "tb_mode.cuh"

namespace tb {

extern template cudaError_t launch_mode_rk<float, true>(int, int, int, const ModeArgs<float> &, cudaStream_t);
extern template cudaError_t launch_mode_rk<double, true>(int, int, int, const ModeArgs<double> &, cudaStream_t);
template cudaError_t launch_mode_rk<float, false>(int, int, int, const ModeArgs<float> &, cudaStream_t);
template cudaError_t launch_mode_rk<double, false>(int, int, int, const ModeArgs<double> &, cudaStream_t);

template <class R>
cudaError_t launch_mode(int in_kind, int out_kind, int ob, int rank, const ModeArgs<R> &a, cudaStream_t st) {
    return rank ? launch_mode_rk<R, true>(in_kind, out_kind, ob, a, st)
                : launch_mode_rk<R, false>(in_kind, out_kind, ob, a, st);
}

int mode_cols_per_thread() { return MODE_NC; }

template cudaError_t launch_mode<float>(int, int, int, int, const ModeArgs<float> &, cudaStream_t);
template cudaError_t launch_mode<double>(int, int, int, int, const ModeArgs<double> &, cudaStream_t);

}  // namespace tb

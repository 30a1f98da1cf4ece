// Level passes as one launch per mode product (k_mode, tb_mode.cuh): the
// complex64 launchers with column slices and rank bounds.
#include "tb_mode.cuh"

namespace tb {

template cudaError_t launch_mode_rk<float, true, true>(int, int, int, const ModeArgs<float> &, cudaStream_t);

}  // namespace tb

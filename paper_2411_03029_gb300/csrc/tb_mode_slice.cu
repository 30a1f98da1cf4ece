// Level passes as one launch per mode product (k_mode, tb_mode.cuh): the
// complex64 launchers with column slices (2 or 4 groups of threads share each
// column; for launches whose units have few columns), without rank bounds.
#include "tb_mode.cuh"

namespace tb {

template cudaError_t launch_mode_rk<float, false, true>(int, int, int, const ModeArgs<float> &, cudaStream_t);

}  // namespace tb

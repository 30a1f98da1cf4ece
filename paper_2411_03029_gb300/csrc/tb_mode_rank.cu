// Level passes as one launch per mode product (k_mode, tb_mode.cuh): the
// launchers with rank bounds (a column computes only the output rows below its
// factor block's rank, or reads only the inputs below it).
#include "tb_mode.cuh"

namespace tb {

template cudaError_t launch_mode_rk<float, true, false>(int, int, int, const ModeArgs<float> &, cudaStream_t);
template cudaError_t launch_mode_rk<double, true, false>(int, int, int, const ModeArgs<double> &, cudaStream_t);

}  // namespace tb

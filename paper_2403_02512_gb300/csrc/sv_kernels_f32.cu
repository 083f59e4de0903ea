// complex64 instantiation of the state-vector kernels.
#define SV_LAUNCH_PART 1  // tile_adjoint: sv_kernels_f32_adjoint.cu
#include "sv_launch.cuh"

namespace sv {
template struct Launch<float>;
}  // namespace sv

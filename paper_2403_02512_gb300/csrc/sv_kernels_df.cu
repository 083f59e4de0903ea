// complex128 states computed in double-float arithmetic (FP32 pairs): global
// amplitudes stay IEEE complex128, tiles are converted on load and store.
#define SV_LAUNCH_PART 1  // tile_adjoint: sv_kernels_df_adjoint.cu
#include "sv_launch.cuh"

namespace sv {
template struct Launch<df>;
}  // namespace sv

// complex128 states in double-float arithmetic: the adjoint-sweep launcher and
// its kernel variants, compiled as a unit of their own beside sv_kernels_df.cu
// (which defines the other launchers).
#define SV_LAUNCH_PART 2
#include "sv_launch.cuh"

namespace sv {
template struct Launch<df>;
}  // namespace sv

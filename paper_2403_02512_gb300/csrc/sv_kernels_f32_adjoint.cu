// complex64: the adjoint-sweep launcher and its kernel variants, compiled as a
// unit of their own beside sv_kernels_f32.cu (which defines the other launchers).
#define SV_LAUNCH_PART 2
#include "sv_launch.cuh"

namespace sv {
template struct Launch<float>;
}  // namespace sv

// complex64 instantiation of the state-vector kernels.
#include "sv_launch.cuh"

namespace sv {
template struct Launch<float>;
}  // namespace sv

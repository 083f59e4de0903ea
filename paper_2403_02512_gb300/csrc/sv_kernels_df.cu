// complex128 states computed in double-float arithmetic (FP32 pairs): global
// amplitudes stay IEEE complex128, tiles are converted on load and store.
#include "sv_launch.cuh"

namespace sv {
template struct Launch<df>;
}  // namespace sv

// lb3_fp32.cu -- FP32 offset-population instantiation of the 3-D kernels
// (FMA contraction allowed).
#include "lb3_launch_impl.cuh"

namespace lbk3 {
template struct Launch3<float>;
}  // namespace lbk3

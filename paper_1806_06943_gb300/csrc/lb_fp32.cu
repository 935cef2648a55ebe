// lb_fp32.cu -- FP32 offset-population instantiation of the lattice
// Boltzmann kernels (FMA contraction allowed).
#include "lb_launch_impl.cuh"

namespace lbk {
template struct Launch<float>;
}

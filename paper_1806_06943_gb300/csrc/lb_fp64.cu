// lb_fp64.cu -- FP64 instantiation of the lattice Boltzmann kernels.
// Compiled with -fmad=false: every FP64 operation rounds once, in the order
// the kernels write it.
#include "lb_launch_impl.cuh"

namespace lbk {
template struct Launch<double>;
}

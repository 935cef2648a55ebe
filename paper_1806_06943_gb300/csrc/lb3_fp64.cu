// lb3_fp64.cu -- FP64 instantiation of the 3-D kernels.  Compiled with
// -fmad=false: every FP64 operation rounds once, in the order written.
#include "lb3_launch_impl.cuh"

namespace lbk3 {
template struct Launch3<double>;

cudaError_t reduce3(const double *partials, int n_tiles, double *out, cudaStream_t s)
{
    k3_reduce<<<1, 256, 0, s>>>(partials, n_tiles, out);
    return cudaGetLastError();
}
}  // namespace lbk3

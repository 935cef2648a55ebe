// lb_fp32.cu -- FP32 offset-population instantiation of the lattice
// Boltzmann kernels (FMA contraction allowed).
#include "lb_launch_impl.cuh"

namespace lbk {
template struct Launch<float>;
}

namespace lbk {
namespace {
// FP64 populations f_i = h_i + w_i R of an FP32 state (offsets h from the
// reference densities R), in the lattice's pitched layout.
__global__ void k_offset_to_f64(int nx, int ny, int pitch, size_t plane, const float *__restrict__ h,
                                const float *__restrict__ R, double *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx || y >= ny) return;
    const size_t c = (size_t)y * pitch + x;
    for (int k = 0; k < 2; ++k) {
        const double r = (double)R[(size_t)k * plane + c];
        for (int i = 0; i < 9; ++i) {
            const size_t q = (size_t)(k * 9 + i) * plane + c;
            out[q] = (double)h[q] + w9(i) * r;
        }
    }
}
}  // namespace

cudaError_t offset_to_f64(const Lat<float> &L, const float *h, const float *R, double *out, cudaStream_t s)
{
    k_offset_to_f64<<<dim3((L.nx + 127) / 128, L.ny), 128, 0, s>>>(L.nx, L.ny, L.pitch, L.plane, h, R, out);
    return cudaGetLastError();
}
}  // namespace lbk

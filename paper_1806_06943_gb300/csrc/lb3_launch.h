// lb3_launch.h -- host-side launchers of the 3-D kernels, one explicit
// instantiation per population format (lb3_fp64.cu, lb3_fp32.cu).
#pragma once

#include <cuda_runtime.h>

#include "lb3_kernels.cuh"

namespace lbk3 {

template <typename real>
struct Launch3 {
    static cudaError_t step(const Lat3<real> &L, int parity, cudaStream_t s);      // density pass + collide
    static cudaError_t density(const Lat3<real> &L, int parity, cudaStream_t s);
    static cudaError_t collide(const Lat3<real> &L, int parity, cudaStream_t s);
    static cudaError_t observe(const Lat3<real> &L, int parity, double *partials, double *rho, double *u,
                               cudaStream_t s);
    static cudaError_t init(const Lat3<real> &L, const double *rho, const double *u, int parity, cudaStream_t s);
    static cudaError_t get_pops(const Lat3<real> &L, int parity, double *out, cudaStream_t s);
};

cudaError_t reduce3(const double *partials, int n_tiles, double *out, cudaStream_t s);

extern template struct Launch3<double>;
extern template struct Launch3<float>;

}  // namespace lbk3

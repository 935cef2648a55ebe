// lb_launch_impl.cuh -- definitions of the launchers; included once per
// population format by lb_fp64.cu and lb_fp32.cu.
#pragma once

#include "lb_kernels.cuh"
#include "lb_launch.h"

namespace lbk {

template <typename real>
cudaError_t Launch<real>::density(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                                  cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    k_density<real><<<n_tiles, dim3(TX, TY), 0, s>>>(lats, tiles, tile_offset, parity);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::collide(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                                  cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    k_collide<real><<<n_tiles, dim3(TX, TY), 0, s>>>(lats, tiles, tile_offset, parity);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::observe(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                                  double *partials, double *rho, double *mom, double *ubar, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    k_observe<real><<<n_tiles, dim3(TX, TY), 0, s>>>(lats, tiles, tile_offset, parity, partials, rho, mom, ubar);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::finalize(const Lat<real> *lats, int n_lat, const double *partials, double *obs, cudaStream_t s)
{
    if (n_lat <= 0) return cudaSuccess;
    k_finalize<real><<<n_lat, 256, 0, s>>>(lats, partials, obs);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::init(const Lat<real> *lats, int lat, int nx, int ny, const double *rho, const double *u,
                               int parity, cudaStream_t s)
{
    k_init<real><<<dim3((nx + 127) / 128, ny), 128, 0, s>>>(lats, lat, rho, u, parity);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::get_pops(const Lat<real> *lats, int lat, int nx, int ny, int parity, double *out,
                                   cudaStream_t s)
{
    k_get_pops<real><<<dim3((nx + 127) / 128, ny), 128, 0, s>>>(lats, lat, parity, out);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::set_pops(const Lat<real> *lats, int lat, int nx, int ny, int parity, const double *in,
                                   cudaStream_t s)
{
    k_set_pops<real><<<dim3((nx + 127) / 128, ny), 128, 0, s>>>(lats, lat, parity, in);
    return cudaGetLastError();
}

}  // namespace lbk

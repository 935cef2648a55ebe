// lb_launch_impl.cuh -- definitions of the launchers; included once per
// population format by lb_fp64.cu and lb_fp32.cu.
#pragma once

#include "lb_kernels.cuh"
#include "lb_launch.h"

namespace lbk {

template <typename real>
cudaError_t Launch<real>::density(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                                  int ty, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    switch (ty) {
    case 2: k_density<real, 2><<<n_tiles, dim3(TX, 2), 0, s>>>(lats, tiles, tile_offset, parity); break;
    case 4: k_density<real, 4><<<n_tiles, dim3(TX, 4), 0, s>>>(lats, tiles, tile_offset, parity); break;
    case 8: k_density<real, 8><<<n_tiles, dim3(TX, 8), 0, s>>>(lats, tiles, tile_offset, parity); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::collide(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                                  int ty, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    switch (ty) {
    case 2: k_collide<real, 2><<<n_tiles, dim3(TX, 2), 0, s>>>(lats, tiles, tile_offset, parity); break;
    case 4: k_collide<real, 4><<<n_tiles, dim3(TX, 4), 0, s>>>(lats, tiles, tile_offset, parity); break;
    case 8: k_collide<real, 8><<<n_tiles, dim3(TX, 8), 0, s>>>(lats, tiles, tile_offset, parity); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::fused(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                                int ty, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    switch (ty) {
    case 2: k_fused<real, 2><<<n_tiles, dim3(TX, 2), 0, s>>>(lats, tiles, tile_offset, parity); break;
    case 4: k_fused<real, 4><<<n_tiles, dim3(TX, 4), 0, s>>>(lats, tiles, tile_offset, parity); break;
    case 8: k_fused<real, 8><<<n_tiles, dim3(TX, 8), 0, s>>>(lats, tiles, tile_offset, parity); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::persistent(const Lat<real> *lats, const int4 *tiles, const int *lat_ntiles, int n_tiles,
                                     int nsteps, int parity0,
                                     void *ctl, unsigned *dens_done, unsigned *coll_done, int *err,
                                     long long wait_cycles, int drop_tile, int ty, int blocks, cudaStream_t s)
{
    if (n_tiles <= 0 || nsteps <= 0) return cudaSuccess;
    PersistCtl *c = (PersistCtl *)ctl;
    switch (ty) {
    case 2:
        k_persistent<real, 2><<<blocks, dim3(TX, 2), 0, s>>>(lats, tiles, lat_ntiles, n_tiles, nsteps, parity0, c, dens_done,
                                                              coll_done, err, wait_cycles, drop_tile);
        break;
    case 4:
        k_persistent<real, 4><<<blocks, dim3(TX, 4), 0, s>>>(lats, tiles, lat_ntiles, n_tiles, nsteps, parity0, c, dens_done,
                                                              coll_done, err, wait_cycles, drop_tile);
        break;
    case 8:
        k_persistent<real, 8><<<blocks, dim3(TX, 8), 0, s>>>(lats, tiles, lat_ntiles, n_tiles, nsteps, parity0, c, dens_done,
                                                              coll_done, err, wait_cycles, drop_tile);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename real>
int Launch<real>::persistent_blocks_per_sm(int ty)
{
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ty == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<real, 2>, TX * 2, 0);
    if (ty == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<real, 4>, TX * 4, 0);
    if (ty == 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<real, 8>, TX * 8, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
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
cudaError_t Launch<real>::pressure(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                                   double *partials, double *out, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    k_pressure<real><<<n_tiles, dim3(TX, TY), 0, s>>>(lats, tiles, tile_offset, parity, partials, out);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::pressure_sum(const Lat<real> *lats, int n_lat, const double *partials, double *out,
                                       cudaStream_t s)
{
    if (n_lat <= 0) return cudaSuccess;
    k_pressure_sum<real><<<n_lat, 256, 0, s>>>(lats, partials, out);
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

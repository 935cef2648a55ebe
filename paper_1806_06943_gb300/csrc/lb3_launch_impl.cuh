// lb3_launch_impl.cuh -- definitions of the 3-D launchers; included once per
// population format.
#pragma once

#include "lb3_launch.h"

namespace lbk3 {

template <typename real>
cudaError_t Launch3<real>::density(const Lat3<real> &L, int parity, cudaStream_t s)
{
    const unsigned n = (unsigned)L.tiles_x * L.tiles_y * L.tiles_z;
    k3_density<real><<<n, dim3(TX, TY, TZ), 0, s>>>(L, parity);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch3<real>::collide(const Lat3<real> &L, int parity, cudaStream_t s)
{
    const unsigned n = (unsigned)L.tiles_x * L.tiles_y * L.tiles_z;
    cudaError_t e = cudaFuncSetAttribute(k3_collide<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kCollideSmem3<real>);
    if (e != cudaSuccess) return e;
    k3_collide<real><<<n, dim3(TX, TY, TZ), kCollideSmem3<real>, s>>>(L, parity);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch3<real>::step(const Lat3<real> &L, int parity, cudaStream_t s)
{
    cudaError_t e = density(L, parity, s);
    if (e == cudaSuccess) e = collide(L, parity, s);
    return e;
}

template <typename real>
cudaError_t Launch3<real>::observe(const Lat3<real> &L, int parity, double *partials, double *rho, double *u,
                                   cudaStream_t s)
{
    const unsigned n = (unsigned)L.tiles_x * L.tiles_y * L.tiles_z;
    cudaError_t e = cudaFuncSetAttribute(k3_observe<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kObserveSmem3<real>);
    if (e != cudaSuccess) return e;
    k3_observe<real><<<n, dim3(TX, TY, TZ), kObserveSmem3<real>, s>>>(L, parity, partials, rho, u);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch3<real>::init(const Lat3<real> &L, const double *rho, const double *u, int parity, cudaStream_t s)
{
    k3_init<real><<<dim3((L.nx + 127) / 128, L.ny, L.nz), 128, 0, s>>>(L, rho, u, parity);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch3<real>::get_pops(const Lat3<real> &L, int parity, double *out, cudaStream_t s)
{
    k3_get_pops<real><<<dim3((L.nx + 127) / 128, L.ny, L.nz), 128, 0, s>>>(L, parity, out);
    return cudaGetLastError();
}

}  // namespace lbk3

// lb_noalloc.cu -- observables of an FP64 lattice whose populations the caller
// holds, computed without allocating any memory.
//
// Some callers cannot allocate device memory while they run: code that owns
// a fixed memory budget (an embedding application with its own pool, a
// solver that must not trigger the driver's allocator between steps, or a
// process that is forbidden to call cudaMalloc after start-up).  This entry
// point serves them: it takes the populations and the output in the caller's
// device memory and keeps its only scratch (the per-tile partial sums of the
// reduction) in a file-scope device array of fixed size, which every GPU that
// loads the library holds until the process exits.
//
// The kernel is a variant of the observables reduction of lb_kernels.cuh that
// forms the densities of its tile and halo directly from the populations, so
// it needs no density field either.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "lb.h"
#include "lb_kernels.cuh"
#include "lb_launch.h"

namespace {

// Partial sums of at most kMaxTiles tiles of 32 x 4 nodes, kAccStride doubles
// each: 32768 * 16 * 8 bytes = 4 MiB of device memory.
constexpr int kMaxTiles = LB_STATIC_MAX_TILES;
static __device__ __align__(256) double g_partials[(size_t)kMaxTiles * lbk::kAccStride];

// Densities of the tile plus its halo from the populations, then psi.
__device__ __forceinline__ void stage_from_pops(const lbk::Lat<double> &L, const double *__restrict__ f, int x0, int y0,
                                                double (*srho)[lbk::SH][lbk::SW], double (*spsi)[lbk::SH][lbk::SW],
                                                int tid)
{
    using namespace lbk;
    const int nx = L.nx, ny = L.ny;
    const size_t n = (size_t)nx * ny;
    for (int idx = tid; idx < SW * SH; idx += kThreads) {
        const int sx = idx % SW, sy = idx / SW;
        const int gx = wrap_index(x0 + sx - HALO, nx);
        int gy = y0 + sy - HALO;
        double r[2];
        bool fixed = false;
        if (gy < 0 || gy >= ny) {
            if (L.walls) {
                if (L.wall_mode == 1) {
                    r[0] = L.wall_rho[0];
                    r[1] = L.wall_rho[1];
                    fixed = true;
                } else {
                    gy = gy < 0 ? -1 - gy : 2 * ny - 1 - gy;
                    gy = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
                }
            } else {
                gy = wrap_index(gy, ny);
            }
        }
        if (!fixed) {
            const size_t c = (size_t)gy * nx + gx;
            for (int k = 0; k < 2; ++k) {
                double v[9];
                for (int i = 0; i < 9; ++i) v[i] = f[(size_t)(k * 9 + i) * n + c];
                r[k] = zeroth_moment<double>(v);
            }
        }
        for (int k = 0; k < 2; ++k) {
            srho[k][sy][sx] = r[k];
            spsi[k][sy][sx] = psi_of<double>(r[k]);
        }
    }
}

__global__ void __launch_bounds__(lbk::kThreads) k_observe_static(const lbk::Lat<double> L,
                                                                  const double *__restrict__ f,
                                                                  double *__restrict__ partials)
{
    using namespace lbk;
    __shared__ double srho[2][SH][SW];
    __shared__ double spsi[2][SH][SW];
    __shared__ double sacc[kThreads / 32][kAccStride];
    const int tiles_x = (L.nx + TX - 1) / TX;
    const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    stage_from_pops(L, f, x0, y0, srho, spsi, tid);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    double acc[kNumAcc];
    for (int a = 0; a < kNumAcc; ++a) acc[a] = 0.0;
    if (x < L.nx && y < L.ny) {
        const int cx = threadIdx.x + HALO, cy = threadIdx.y + HALO;
        const size_t n = (size_t)L.nx * L.ny, c = (size_t)y * L.nx + x;
        double r[2], m[2][2];
        for (int k = 0; k < 2; ++k) {
            double fk[9];
            for (int i = 0; i < 9; ++i) fk[i] = f[(size_t)(k * 9 + i) * n + c];
            double Fx, Fy, jx, jy;
            force_at<double>(L, srho, spsi, k, cx, cy, Fx, Fy);
            first_moment<double>(fk, jx, jy);
            r[k] = srho[k][cy][cx];
            m[k][0] = jx + 0.5 * Fx;
            m[k][1] = jy + 0.5 * Fy;
        }
        const double rt = r[0] + r[1];
        const double ux = (m[0][0] + m[1][0]) / rt, uy = (m[0][1] + m[1][1]) / rt;
        acc[kMassA] = r[0];
        acc[kMassB] = r[1];
        acc[kMomAx] = m[0][0];
        acc[kMomAy] = m[0][1];
        acc[kMomBx] = m[1][0];
        acc[kMomBy] = m[1][1];
        acc[kSumUx] = ux;
        acc[kUmax] = sqrt(ux * ux + uy * uy);
        acc[kNonFinite] = (isfinite(r[0]) && isfinite(r[1]) && isfinite(ux) && isfinite(uy)) ? 0.0 : 1.0;
        if (L.has_probe) {
            double dx = fabs((double)x - L.probe[0]), dy = fabs((double)y - L.probe[1]);
            if (dx > 0.5 * L.nx) dx = L.nx - dx;
            if (!L.walls && dy > 0.5 * L.ny) dy = L.ny - dy;
            const double rr = sqrt(dx * dx + dy * dy), R = L.probe[2];
            const double psiA = 1.0 - exp(-r[0]), psiB = 1.0 - exp(-r[1]);
            const double Gs = L.G1 + L.G2;
            const double pb = (r[0] + 0.5 * Gs * psiA * psiA) / 3.0 + (r[1] + 0.5 * Gs * psiB * psiB) / 3.0
                            + L.GAB * r[0] * r[1] / 3.0;
            if (rr < 0.5 * R) { acc[kPIn] = pb; acc[kAIn] = r[0]; acc[kNIn] = 1.0; }
            if (rr > R + 6.0) { acc[kPOut] = pb; acc[kAOut] = r[0]; acc[kNOut] = 1.0; }
        }
    }
    const int warp = tid >> 5, lane = tid & 31;
    for (int a = 0; a < kNumAcc; ++a) {
        const double v = (a == kUmax) ? warp_max(acc[a]) : warp_sum(acc[a]);
        if (lane == 0) sacc[warp][a] = v;
    }
    __syncthreads();
    if (tid < kNumAcc) {
        double v = sacc[0][tid];
        for (int w = 1; w < kThreads / 32; ++w) v = (tid == kUmax) ? fmax(v, sacc[w][tid]) : v + sacc[w][tid];
        partials[(size_t)blockIdx.x * kAccStride + tid] = v;
    }
}

// One block: reduce the tile partials in a fixed order into the caller's
// record (the same slots and formulas as the library's observables).
__global__ void __launch_bounds__(256) k_finalize_static(const lbk::Lat<double> L,
                                                         const double *__restrict__ partials,
                                                         double *__restrict__ obs)
{
    using namespace lbk;
    __shared__ double sred[256 / 32][kAccStride];
    const int tid = threadIdx.x;
    double acc[kNumAcc];
    for (int a = 0; a < kNumAcc; ++a) acc[a] = 0.0;
    for (int tl = tid; tl < L.tile_end; tl += 256)
        for (int a = 0; a < kNumAcc; ++a) {
            const double v = partials[(size_t)tl * kAccStride + a];
            acc[a] = (a == kUmax) ? fmax(acc[a], v) : acc[a] + v;
        }
    const int warp = tid >> 5, lane = tid & 31;
    for (int a = 0; a < kNumAcc; ++a) {
        const double v = (a == kUmax) ? warp_max(acc[a]) : warp_sum(acc[a]);
        if (lane == 0) sred[warp][a] = v;
    }
    __syncthreads();
    if (tid != 0) return;
    double s[kNumAcc];
    for (int a = 0; a < kNumAcc; ++a) {
        double v = sred[0][a];
        for (int w = 1; w < 8; ++w) v = (a == kUmax) ? fmax(v, sred[w][a]) : v + sred[w][a];
        s[a] = v;
    }
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    obs[oMassA] = s[kMassA];
    obs[oMassB] = s[kMassB];
    obs[oMomAx] = s[kMomAx];
    obs[oMomAy] = s[kMomAy];
    obs[oMomBx] = s[kMomBx];
    obs[oMomBy] = s[kMomBy];
    obs[oQ] = s[kSumUx] / L.nx;
    if (L.walls && L.g_x != 0.0) {
        const double H = L.ny, nuB = (L.tau_B - 0.5) / 3.0;
        obs[oMuR] = L.g_x * (H * H * H + 0.5 * H) / (12.0 * nuB) / obs[oQ];
    } else {
        obs[oMuR] = nan;
    }
    if (L.has_probe && s[kNIn] > 0.0 && s[kNOut] > 0.0) {
        const double rin = s[kAIn] / s[kNIn], rout = s[kAOut] / s[kNOut];
        obs[oDp] = s[kPIn] / s[kNIn] - s[kPOut] / s[kNOut];
        obs[oReff] = sqrt((s[kMassA] - rout * (double)L.nx * (double)L.ny) / (3.14159265358979323846 * (rin - rout)));
    } else {
        obs[oDp] = nan;
        obs[oReff] = nan;
    }
    obs[oUmax] = s[kUmax];
    obs[oFinite] = s[kNonFinite] == 0.0 ? 1.0 : 0.0;
    for (int a = kNumObs; a < kObsStride; ++a) obs[a] = 0.0;
}

int set_fail(int code, const char *msg)
{
    lbk::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int lb_observables_static(const lb_params *p, const double *f, double cx, double cy, double R, double *obs)
{
    // set-up only: load this file's module on the current device (the driver
    // places g_partials then) and resolve the array's address; nothing runs
    const bool setup_only = !f && !obs;
    if (!setup_only) {
        if (!p || !f || !obs) return set_fail(LB_EINVAL, "lb_observables_static: NULL argument");
        if (lbk::validate_params(p, 0) != LB_OK) return LB_EINVAL;   // message recorded by the check
        if (p->precision != LB_FP64) return set_fail(LB_EINVAL, "lb_observables_static: populations must be LB_FP64");
        if (!std::isfinite(cx) || !std::isfinite(cy) || !std::isfinite(R))
            return set_fail(LB_EINVAL, "lb_observables_static: non-finite probe");
    }
    const long long tiles_x = setup_only ? 0 : (p->nx + lbk::TX - 1) / lbk::TX;
    const long long tiles_y = setup_only ? 0 : (p->ny + lbk::TY - 1) / lbk::TY;
    if (tiles_x * tiles_y > kMaxTiles)
        return set_fail(LB_EINVAL, "lb_observables_static: lattice exceeds LB_STATIC_MAX_TILES tiles of 32x4 nodes");

    // The host name g_partials is only a stand-in for the array, not a device
    // address: ask the runtime for the address on the current device.  The
    // lookup is repeated on every call, so a context torn down and created
    // again (cudaDeviceReset) never leaves a stale address behind; once the
    // module is loaded on the device the lookup allocates nothing.
    void *ptr = nullptr;
    cudaError_t ce = cudaGetSymbolAddress(&ptr, g_partials);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return set_fail(LB_ECUDA, "lb_observables_static: cudaGetSymbolAddress failed");
    }
    if (setup_only) return LB_OK;
    double *scratch = (double *)ptr;

    lbk::Lat<double> L;
    std::memset(&L, 0, sizeof L);
    L.nx = p->nx;
    L.ny = p->ny;
    L.pitch = p->nx;
    L.plane = (size_t)p->nx * p->ny;
    L.walls = p->walls;
    L.wall_mode = p->wall_mode;
    L.G1 = p->G1;
    L.G2 = p->G2;
    L.GAB = p->G_AB;
    L.g[0] = p->g[0];
    L.g[1] = p->g[1];
    L.wall_rho[0] = p->wall_rho[0];
    L.wall_rho[1] = p->wall_rho[1];
    L.tile_begin = 0;
    L.tile_end = (int)(tiles_x * tiles_y);
    L.has_probe = R > 0.0 ? 1 : 0;
    L.probe[0] = cx;
    L.probe[1] = cy;
    L.probe[2] = R;
    L.tau_B = p->tau[1];
    L.g_x = p->g[0];

    cudaStream_t s = (cudaStream_t)p->stream;
    k_observe_static<<<(unsigned)(tiles_x * tiles_y), dim3(lbk::TX, lbk::TY), 0, s>>>(L, f, scratch);
    if ((ce = cudaGetLastError()) != cudaSuccess) return set_fail(LB_ECUDA, "lb_observables_static: launch failed");
    k_finalize_static<<<1, 256, 0, s>>>(L, scratch, obs);
    if ((ce = cudaGetLastError()) != cudaSuccess)
        return set_fail(LB_ECUDA, "lb_observables_static: finalize launch failed");
    return LB_OK;
}

// lb3_kernels.cuh -- sm_103a kernels of the three-dimensional extension of the
// two-range pseudopotential lattice Boltzmann step (the paper is 2-D; its
// Sec. II carried to three dimensions):
//   fluid         D3Q19 (w = 1/3, 1/18, 1/36), BGK with Guo forcing (Eqs. 1-3,
//                 5, 6 in 3-D)
//   short range   sums of Eqs. (8) (first term) and (9) over the D3Q19
//                 neighbours with the weights w
//   mid range     sum of Eq. (8) (second term) over the 5 x 5 x 5
//                 neighbourhood with weights q(|e|^2): 47/90, 4/135, 1/63,
//                 2/315, 5/1512, 1/945, 1/1890, 1/15120 for |e|^2 = 0..6, 8
//                 (0 for 9 and 12), isotropic to eighth order with the D2Q25
//                 stencil's second and fourth moments
// Periodic in x, y and z.  Templated on the population format, as the 2-D
// kernels: real = double plain populations (this instantiation compiled
// without FMA contraction), real = float offsets h_i = f_i - w_i R from the
// node's density at the previous step R, with the stencil and momentum sums
// formed from differences of opposite neighbours.
//
// One time step is two launches over tiles of 32 x 4 x 2 nodes:
//   k3_density : rho_k = sum_i f_k,i (FP32: R + sum_i h_i) into copy parity^1
//   k3_collide : stages rho_k and psi_k of the tile plus a 2-node halo in
//                shared memory, forms the forces, moments, u^eq, relaxes with
//                the Guo term and pushes each population to x + e_i (FP32:
//                re-referenced to rho(x + e_i), the destination's next R).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

namespace lbk3 {

constexpr int TX = 32, TY = 4, TZ = 2, HALO = 2;
constexpr int SX = TX + 2 * HALO, SY = TY + 2 * HALO, SZ = TZ + 2 * HALO;
constexpr int kThreads = TX * TY * TZ;
constexpr int kNumAcc = 16;   // observation partial sums per tile

// D3Q19: rest, 6 axis directions, 12 edge directions
__host__ __device__ constexpr int ex(int i)
{
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1 : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i)
{
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1 : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
}
__host__ __device__ constexpr int ez(int i)
{
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1 : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
}
__host__ __device__ constexpr int e2(int i) { return ex(i) * ex(i) + ey(i) * ey(i) + ez(i) * ez(i); }
__host__ __device__ constexpr double w19(int i) { return e2(i) == 0 ? 1.0 / 3.0 : (e2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0); }
__host__ __device__ constexpr double q125(int e2v)
{
    return e2v == 0 ? 47.0 / 90.0 : e2v == 1 ? 4.0 / 135.0 : e2v == 2 ? 1.0 / 63.0 : e2v == 3 ? 2.0 / 315.0
         : e2v == 4 ? 5.0 / 1512.0 : e2v == 5 ? 1.0 / 945.0 : e2v == 6 ? 1.0 / 1890.0 : e2v == 8 ? 1.0 / 15120.0 : 0.0;
}

template <typename real>
constexpr bool kOffset3 = sizeof(real) == 4;

// Descriptor of one 3-D lattice (device-visible).
template <typename real>
struct Lat3 {
    real *f[2];          // ping-pong populations [2][19][nz][ny][pitch]
    real *rho[2];        // densities [2][nz][ny][pitch]
    size_t plane;        // elements per [nz][ny][pitch] volume
    int32_t nx, ny, nz, pitch;
    int32_t tiles_x, tiles_y, tiles_z, has_probe;
    real omega[2], aw[2][3];   // 1 / tau_k; (1 - omega_k / 2) w(|e|^2) for |e|^2 = 0, 1, 2
    real G1, G2, GAB;
    real g[3];
    double probe[4];     // cx, cy, cz, R
};

template <typename real> __device__ __forceinline__ real psi3(real r);
template <> __device__ __forceinline__ double psi3<double>(double r) { return 1.0 - exp(-r); }
template <> __device__ __forceinline__ float psi3<float>(float r) { return -expm1f(-r); }

__device__ __forceinline__ int wrap3(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

// a periodic index one period off at most (a in [-n, 2n)): no division
__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ void tile_origin(int tiles_x, int tiles_y, int b, int &x0, int &y0, int &z0)
{
    x0 = (b % tiles_x) * TX;
    y0 = ((b / tiles_x) % tiles_y) * TY;
    z0 = (b / (tiles_x * tiles_y)) * TZ;
}

template <typename real>
struct Stage3 {
    real rho[2][SZ][SY][SX];
    real psi[2][SZ][SY][SX];
};
static_assert(sizeof(Stage3<float>) % 16 == 0 && sizeof(Stage3<double>) % 16 == 0, "partials stay aligned");

template <typename real>
constexpr size_t kCollideSmem3 = sizeof(Stage3<real>);
template <typename real>
constexpr size_t kObserveSmem3 = sizeof(Stage3<real>) + (kThreads / 32) * kNumAcc * sizeof(double);

// rho and psi of the tile (x0, y0, z0) and its 2-node halo from density copy
// `rho` (periodic copies across every face).
template <typename real>
__device__ __forceinline__ void stage3(const Lat3<real> &L, const real *__restrict__ rho, int x0, int y0, int z0,
                                       Stage3<real> &sm, int tid)
{
    // the slots' coordinates lie within one period of the lattice when each
    // side is at least a tile plus both halos (a block-uniform choice)
    const bool near = L.nx >= SX && L.ny >= SY && L.nz >= SZ;
    for (int idx = tid; idx < SX * SY * SZ; idx += kThreads) {
        const int sx = idx % SX, sy = (idx / SX) % SY, sz = idx / (SX * SY);
        const int ax = x0 + sx - HALO, ay = y0 + sy - HALO, az = z0 + sz - HALO;
        const int gx = near ? wrap1(ax, L.nx) : wrap3(ax, L.nx), gy = near ? wrap1(ay, L.ny) : wrap3(ay, L.ny);
        const int gz = near ? wrap1(az, L.nz) : wrap3(az, L.nz);
        const size_t c = ((size_t)gz * L.ny + gy) * L.pitch + gx;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const real r = rho[(size_t)k * L.plane + c];
            sm.rho[k][sz][sy][sx] = r;
            sm.psi[k][sz][sy][sx] = psi3<real>(r);
        }
    }
}

// sum_i w_i s(x + e_i) e_i over D3Q19 (FP64: direction order; FP32:
// differences of opposite neighbours)
template <typename real>
__device__ __forceinline__ void q19_sum(const real (*s)[SY][SX], int cx, int cy, int cz, real (&out)[3])
{
    out[0] = out[1] = out[2] = (real)0;
    if constexpr (!kOffset3<real>) {
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const real a = (real)w19(i) * s[cz + ez(i)][cy + ey(i)][cx + ex(i)];
            if (ex(i)) out[0] += a * (real)ex(i);
            if (ey(i)) out[1] += a * (real)ey(i);
            if (ez(i)) out[2] += a * (real)ez(i);
        }
    } else {
#pragma unroll
        for (int i = 1; i < 19; i += 2) {   // directions come in opposite pairs (i, i + 1)
            const real d = s[cz + ez(i)][cy + ey(i)][cx + ex(i)] - s[cz - ez(i)][cy - ey(i)][cx - ex(i)];
            const real wd = (real)w19(i) * d;
            if (ex(i)) out[0] += ex(i) > 0 ? wd : -wd;
            if (ey(i)) out[1] += ey(i) > 0 ? wd : -wd;
            if (ez(i)) out[2] += ez(i) > 0 ? wd : -wd;
        }
    }
}

// sum_j q_j s(x + e_j) e_j over the 5 x 5 x 5 neighbourhood (FP64: raster
// order dz, dy, dx; FP32: differences of opposite neighbours, each pair once)
template <typename real>
__device__ __forceinline__ void q125_sum(const real (*s)[SY][SX], int cx, int cy, int cz, real (&out)[3])
{
    out[0] = out[1] = out[2] = (real)0;
#pragma unroll
    for (int j = 0; j < 125; ++j) {
        const int dx = j % 5 - 2, dy = (j / 5) % 5 - 2, dz = j / 25 - 2;
        const double qw = q125(dx * dx + dy * dy + dz * dz);
        if (qw == 0.0 || (dx == 0 && dy == 0 && dz == 0)) continue;
        if constexpr (!kOffset3<real>) {
            const real a = (real)qw * s[cz + dz][cy + dy][cx + dx];
            if (dx) out[0] += a * (real)dx;
            if (dy) out[1] += a * (real)dy;
            if (dz) out[2] += a * (real)dz;
        } else {
            // each opposite pair once: the member with dz > 0, or dz = 0 and
            // dy > 0, or dz = dy = 0 and dx > 0
            if (!(dz > 0 || (dz == 0 && dy > 0) || (dz == 0 && dy == 0 && dx > 0))) continue;
            const real d = (real)qw * (s[cz + dz][cy + dy][cx + dx] - s[cz - dz][cy - dy][cx - dx]);
            if (dx) out[0] += d * (real)dx;
            if (dy) out[1] += d * (real)dy;
            if (dz) out[2] += d * (real)dz;
        }
    }
}

// total force on species k at the staged node: Eq. (8) + Eq. (9) + rho_k g
template <typename real>
__device__ __forceinline__ void force3(const Lat3<real> &L, const Stage3<real> &sm, int k, int cx, int cy, int cz,
                                       real (&F)[3])
{
    real s1[3], s2[3], s3[3];
    q19_sum<real>(sm.psi[k], cx, cy, cz, s1);
    q125_sum<real>(sm.psi[k], cx, cy, cz, s2);
    q19_sum<real>(sm.rho[1 - k], cx, cy, cz, s3);
    const real psi = sm.psi[k][cz][cy][cx], rho = sm.rho[k][cz][cy][cx];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a] = -L.G1 * psi * s1[a] - L.G2 * psi * s2[a] - L.GAB * rho * s3[a] + rho * L.g[a];
}

template <typename real>
__global__ void __launch_bounds__(kThreads) k3_density(const Lat3<real> L, int parity)
{
    int x0, y0, z0;
    tile_origin(L.tiles_x, L.tiles_y, blockIdx.x, x0, y0, z0);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    if (x >= L.nx || y >= L.ny || z >= L.nz) return;
    const size_t c = ((size_t)z * L.ny + y) * L.pitch + x;
    const real *__restrict__ f = L.f[parity];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        real r = (real)0;
#pragma unroll
        for (int i = 0; i < 19; ++i) r += f[(size_t)(k * 19 + i) * L.plane + c];
        if constexpr (kOffset3<real>) r = L.rho[parity][(size_t)k * L.plane + c] + r;
        L.rho[parity ^ 1][(size_t)k * L.plane + c] = r;
    }
}

// Dynamic shared memory of the staging kernels (the FP64 stage is above the
// 48 KB of static shared memory): the stage, then the observation partials.
extern __shared__ __align__(16) unsigned char lb3_smem[];

// FP32: three blocks per SM (80 registers; the spill of a few values costs
// less than the latency a third block hides), FP64: as many as fit.
template <typename real>
__global__ void __launch_bounds__(kThreads, kOffset3<real> ? 3 : 1) k3_collide(const Lat3<real> L, int parity)
{
    Stage3<real> &sm = *reinterpret_cast<Stage3<real> *>(lb3_smem);
    int x0, y0, z0;
    tile_origin(L.tiles_x, L.tiles_y, blockIdx.x, x0, y0, z0);
    const int tid = (threadIdx.z * TY + threadIdx.y) * TX + threadIdx.x;
    stage3<real>(L, L.rho[parity ^ 1], x0, y0, z0, sm, tid);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    if (x >= L.nx || y >= L.ny || z >= L.nz) return;
    const int cx = threadIdx.x + HALO, cy = threadIdx.y + HALO, cz = threadIdx.z + HALO;
    const size_t c = ((size_t)z * L.ny + y) * L.pitch + x;
    const real *__restrict__ fc = L.f[parity];
    real *__restrict__ fn = L.f[parity ^ 1];
    real F[2][3], rho[2], m[2][3], delta[2] = {(real)0, (real)0}, dg[2] = {(real)0, (real)0};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        force3<real>(L, sm, k, cx, cy, cz, F[k]);
        rho[k] = sm.rho[k][cz][cy][cx];
        real j[3] = {(real)0, (real)0, (real)0}, s = (real)0;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const real fi = fc[(size_t)(k * 19 + i) * L.plane + c];
            if constexpr (!kOffset3<real>) {
                if (ex(i)) j[0] += ex(i) > 0 ? fi : -fi;
                if (ey(i)) j[1] += ey(i) > 0 ? fi : -fi;
                if (ez(i)) j[2] += ez(i) > 0 ? fi : -fi;
            } else {
                (void)s;
            }
        }
        if constexpr (kOffset3<real>) {
            // first moment from differences of opposite offsets; the offsets
            // from the node's current density h - w (rho - R), their sum dg
#pragma unroll
            for (int i = 1; i < 19; i += 2) {
                const real d = fc[(size_t)(k * 19 + i) * L.plane + c] - fc[(size_t)(k * 19 + i + 1) * L.plane + c];
                if (ex(i)) j[0] += ex(i) > 0 ? d : -d;
                if (ey(i)) j[1] += ey(i) > 0 ? d : -d;
                if (ez(i)) j[2] += ez(i) > 0 ? d : -d;
            }
            delta[k] = rho[k] - L.rho[parity][(size_t)k * L.plane + c];
            real sum = (real)0;
#pragma unroll
            for (int i = 0; i < 19; ++i) sum += fc[(size_t)(k * 19 + i) * L.plane + c] - (real)w19(i) * delta[k];
            dg[k] = sum;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) m[k][a] = j[a] + (real)0.5 * F[k][a];   // Eq. (6), half force
    }
    // Eq. (3)
    const real om0 = L.omega[0], om1 = L.omega[1];
    const real den = om0 * rho[0] + om1 * rho[1];
    real u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = (om0 * m[0][a] + om1 * m[1][a]) / den;
    const real uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const real om = L.omega[k];
        const real uF = u[0] * F[k][0] + u[1] * F[k][1] + u[2] * F[k][2];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int EX = ex(i), EY = ey(i), EZ = ez(i), C = e2(i);
            const real w = (real)w19(i);
            const real eu = (real)EX * u[0] + (real)EY * u[1] + (real)EZ * u[2];
            const real eF = (real)EX * F[k][0] + (real)EY * F[k][1] + (real)EZ * F[k][2];
            const real f = fc[(size_t)(k * 19 + i) * L.plane + c];
            real v;
            if constexpr (!kOffset3<real>) {
                // Eqs. (1), (2), (5)
                const real feq = w * rho[k] * ((real)1 + (real)3 * eu + (real)4.5 * eu * eu - (real)1.5 * uu);
                real Cg = (real)0;
                const real e[3] = {(real)EX, (real)EY, (real)EZ};
#pragma unroll
                for (int a = 0; a < 3; ++a) Cg += ((real)3 * (e[a] - u[a]) + (real)9 * eu * e[a]) * F[k][a];
                Cg = L.aw[k][C] * Cg;
                v = f - om * (f - feq) + Cg;
            } else {
                // offset form: Eq. (2) less w rho, Eq. (5) as 3 (1 - 1/2tau) w [(e.F)(1 + 3 e.u) - u.F]
                const real h = f - w * delta[k];
                const real geq = w * rho[k] * ((real)3 * eu + (real)4.5 * eu * eu - (real)1.5 * uu) + w * dg[k];
                const real Cg = (real)3 * L.aw[k][C] * (eF * ((real)1 + (real)3 * eu) - uF);
                v = (h + om * (geq - h)) + Cg;
                // re-referenced to the destination's density (its next R)
                if (i != 0) v += w * (rho[k] - sm.rho[k][cz + EZ][cy + EY][cx + EX]);
            }
            const int xd = wrap1(x + EX, L.nx), yd = wrap1(y + EY, L.ny), zd = wrap1(z + EZ, L.nz);
            fn[(size_t)(k * 19 + i) * L.plane + ((size_t)zd * L.ny + yd) * L.pitch + xd] = v;
        }
    }
}

// Per-node diagnostics reduced per tile into FP64 partials: masses, momenta
// with half force (Eq. 6), max |ubar| (Eq. 7), non-finite count, and the
// Laplace probe's inside / outside sums of the Eq. (11) bulk pressure and of
// rho_A; optional dense FP64 fields rho [2][nz][ny][nx], ubar [3][..].
template <typename real>
__global__ void __launch_bounds__(kThreads) k3_observe(const Lat3<real> L, int parity, double *__restrict__ partials,
                                                       double *__restrict__ out_rho, double *__restrict__ out_u)
{
    Stage3<real> &sm = *reinterpret_cast<Stage3<real> *>(lb3_smem);
    double(*sacc)[kNumAcc] = reinterpret_cast<double(*)[kNumAcc]>(lb3_smem + sizeof(Stage3<real>));
    int x0, y0, z0;
    tile_origin(L.tiles_x, L.tiles_y, blockIdx.x, x0, y0, z0);
    const int tid = (threadIdx.z * TY + threadIdx.y) * TX + threadIdx.x;
    stage3<real>(L, L.rho[parity ^ 1], x0, y0, z0, sm, tid);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    double acc[kNumAcc];
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) acc[a] = 0.0;
    if (x < L.nx && y < L.ny && z < L.nz) {
        const int cx = threadIdx.x + HALO, cy = threadIdx.y + HALO, cz = threadIdx.z + HALO;
        const size_t c = ((size_t)z * L.ny + y) * L.pitch + x;
        double r[2], m[2][3];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            real F[3];
            force3<real>(L, sm, k, cx, cy, cz, F);
            double j[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                const double fi = (double)L.f[parity][(size_t)(k * 19 + i) * L.plane + c];
                j[0] += fi * ex(i);
                j[1] += fi * ey(i);
                j[2] += fi * ez(i);
            }
            r[k] = (double)sm.rho[k][cz][cy][cx];
#pragma unroll
            for (int a = 0; a < 3; ++a) m[k][a] = j[a] + 0.5 * (double)F[a];
        }
        const double rt = r[0] + r[1];
        double ub[3], u2 = 0.0;
        bool fin = isfinite(r[0]) && isfinite(r[1]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ub[a] = (m[0][a] + m[1][a]) / rt;
            u2 += ub[a] * ub[a];
            fin = fin && isfinite(ub[a]);
        }
        acc[0] = r[0];
        acc[1] = r[1];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            acc[2 + a] = m[0][a];
            acc[5 + a] = m[1][a];
        }
        acc[8] = sqrt(u2);
        acc[9] = fin ? 0.0 : 1.0;
        if (L.has_probe) {
            const int Ls[3] = {L.nx, L.ny, L.nz};
            const int p[3] = {x, y, z};
            double rr2 = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double d = fabs((double)p[a] - L.probe[a]);
                if (d > 0.5 * Ls[a]) d = Ls[a] - d;
                rr2 += d * d;
            }
            const double rr = sqrt(rr2), R = L.probe[3];
            const double psiA = 1.0 - exp(-r[0]), psiB = 1.0 - exp(-r[1]);
            const double Gs = (double)L.G1 + (double)L.G2;
            const double pb = (r[0] + 0.5 * Gs * psiA * psiA) / 3.0 + (r[1] + 0.5 * Gs * psiB * psiB) / 3.0
                            + (double)L.GAB * r[0] * r[1] / 3.0;
            if (rr < 0.5 * R) { acc[10] = pb; acc[11] = r[0]; acc[12] = 1.0; }
            if (rr > R + 6.0) { acc[13] = pb; acc[14] = r[0]; acc[15] = 1.0; }
        }
        if (out_rho) {
            const size_t n = (size_t)L.nx * L.ny * L.nz, d = ((size_t)z * L.ny + y) * L.nx + x;
            out_rho[d] = r[0];
            out_rho[n + d] = r[1];
            if (out_u)
#pragma unroll
                for (int a = 0; a < 3; ++a) out_u[a * n + d] = ub[a];
        }
    }
    if (!partials) return;
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) {
        double v = acc[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v, o);
            v = a == 8 ? fmax(v, w) : v + w;
        }
        if (lane == 0) sacc[warp][a] = v;
    }
    __syncthreads();
    if (tid < kNumAcc) {
        double v = sacc[0][tid];
        for (int w = 1; w < kThreads / 32; ++w) v = tid == 8 ? fmax(v, sacc[w][tid]) : v + sacc[w][tid];
        partials[(size_t)blockIdx.x * kNumAcc + tid] = v;
    }
}

// one block: the tile partials summed (max for |u|) in a fixed order
static __global__ void __launch_bounds__(256) k3_reduce(const double *__restrict__ partials, int n_tiles,
                                                 double *__restrict__ out)
{
    __shared__ double sred[256 / 32][kNumAcc];
    const int tid = threadIdx.x;
    double acc[kNumAcc];
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) acc[a] = 0.0;
    for (int t = tid; t < n_tiles; t += 256)
#pragma unroll
        for (int a = 0; a < kNumAcc; ++a) {
            const double v = partials[(size_t)t * kNumAcc + a];
            acc[a] = a == 8 ? fmax(acc[a], v) : acc[a] + v;
        }
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) {
        double v = acc[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v, o);
            v = a == 8 ? fmax(v, w) : v + w;
        }
        if (lane == 0) sred[warp][a] = v;
    }
    __syncthreads();
    if (tid < kNumAcc) {
        double v = sred[0][tid];
        for (int w = 1; w < 8; ++w) v = tid == 8 ? fmax(v, sred[w][tid]) : v + sred[w][tid];
        out[tid] = v;
    }
}

// f = f^eq(rho_k, u) (Eq. 2) from dense FP64 fields; FP32 stores R = rho
// (rounded) and the offsets f^eq - w R
template <typename real>
__global__ void k3_init(const Lat3<real> L, const double *__restrict__ rho, const double *__restrict__ u, int parity)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    const size_t n = (size_t)L.nx * L.ny * L.nz, d = ((size_t)z * L.ny + y) * L.nx + x;
    const size_t c = ((size_t)z * L.ny + y) * L.pitch + x;
    const double ux = u ? u[d] : 0.0, uy = u ? u[n + d] : 0.0, uz = u ? u[2 * n + d] : 0.0;
    const double uu = ux * ux + uy * uy + uz * uz;
    for (int k = 0; k < 2; ++k) {
        const double r = rho[k * n + d];
        double R = 0.0;
        if constexpr (kOffset3<real>) {
            const real Rr = (real)r;
            L.rho[parity][(size_t)k * L.plane + c] = Rr;
            R = (double)Rr;
        }
        for (int i = 0; i < 19; ++i) {
            const double eu = ex(i) * ux + ey(i) * uy + ez(i) * uz;
            const double feq = w19(i) * r * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
            L.f[parity][(size_t)(k * 19 + i) * L.plane + c] = (real)(feq - w19(i) * R);
        }
    }
}

// populations as dense FP64 [2][19][nz][ny][nx] (FP32: w_i R added back)
template <typename real>
__global__ void k3_get_pops(const Lat3<real> L, int parity, double *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    const size_t n = (size_t)L.nx * L.ny * L.nz, d = ((size_t)z * L.ny + y) * L.nx + x;
    const size_t c = ((size_t)z * L.ny + y) * L.pitch + x;
    for (int k = 0; k < 2; ++k) {
        const double R = kOffset3<real> ? (double)L.rho[parity][(size_t)k * L.plane + c] : 0.0;
        for (int i = 0; i < 19; ++i)
            out[(size_t)(k * 19 + i) * n + d] = (double)L.f[parity][(size_t)(k * 19 + i) * L.plane + c] + w19(i) * R;
    }
}

}  // namespace lbk3

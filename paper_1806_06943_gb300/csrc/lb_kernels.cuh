// lb_kernels.cuh -- sm_103a kernels of the two-range pseudopotential lattice
// Boltzmann step (Fei et al., arXiv:1806.06943, Sec. II), templated on the
// population format:
//   real = double : plain populations f; this instantiation is compiled
//                   without fused multiply-add and evaluates every sum in the
//                   same order as a direct evaluation of the equations, so it
//                   reproduces a plain FP64 evaluation up to the last bit of exp().
//   real = float  : offset populations h_i = f_i - w_i R, R the node's density
//                   at the previous step (kept in the other density copy), so
//                   the stored numbers are the small deviations from the local
//                   equilibrium at rest and keep their low-order digits.  The
//                   stencil and momentum sums are formed from differences of
//                   opposite neighbours, which keeps them exactly antisymmetric
//                   under reflection even with fused multiply-add (no drift).
//
// One time step is two launches over a list of tiles (lattice, x0, y0):
//   k_density : rho_k = sum_i f_k,i                           (Eq. 6)
//   k_collide : stages rho_k of the tile plus a 2-node halo in shared memory,
//               psi_k = 1 - exp(-rho_k) (Sec. II B), the forces of Eqs. (8),
//               (9) and rho_k g, the moments of Eq. (6), u^eq of Eq. (3), the
//               BGK relaxation to Eq. (2) with the Guo term of Eq. (5), and
//               pushes each post-collision population to x + e_i, reflecting
//               it at a half-way bounce-back wall (Sec. III A).
// The populations at a node are the pre-collision values of the current time,
// so both passes read them at their own node with coalesced loads.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "lb_types.h"
#include "lb_vops.cuh"

#include <type_traits>

namespace lbk {

constexpr int TX = 32;           // tile width = threads in x
constexpr int TY = 4;            // tile height of the observation kernels = threads in y
constexpr int HALO = 2;          // reach of the D2Q25 stencil
constexpr int SW = TX + 2 * HALO;
constexpr int SH = TY + 2 * HALO;
constexpr int kThreads = TX * TY;
// Tile heights the time-step kernels are built for (chosen per batch by the
// autotuner); one thread per node, 32 nodes wide.
constexpr int kTileHeights[3] = {2, 4, 8};

template <typename real>
constexpr bool kOffset = sizeof(real) == 4;

// Resident blocks per SM the fused kernel is compiled for: the FP32 kernel is
// bound by HBM and needs the warps to keep enough loads in flight; the FP64
// kernel is bound by the FP64 pipe and keeps its registers.
template <typename real, int TYv>
constexpr int kCollideMinBlocks = (kOffset<real> ? 32 : 16) / TYv;

// ---- lattice tables (Sec. II A; Fig. 1; Sec. II B after Eq. 8) ------------
// D2Q9 order: rest, (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1).
__host__ __device__ constexpr int ex9(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int ey9(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp9(int i)
{
    return i == 0 ? 0 : i == 1 ? 3 : i == 2 ? 4 : i == 3 ? 1 : i == 4 ? 2 : i == 5 ? 7 : i == 6 ? 8 : i == 7 ? 5 : 6;
}
// w(|e|^2) class of direction i: 0 rest, 1 axis, 2 diagonal.
__host__ __device__ constexpr int cls9(int i) { return i == 0 ? 0 : (i <= 4 ? 1 : 2); }
__host__ __device__ constexpr double w9(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
// D2Q25 weights p(|e|^2).
__host__ __device__ constexpr double p25(int e2)
{
    return e2 == 0 ? 247.0 / 420.0 : e2 == 1 ? 4.0 / 63.0 : e2 == 2 ? 4.0 / 135.0 : e2 == 4 ? 1.0 / 180.0
         : e2 == 5 ? 2.0 / 945.0 : e2 == 8 ? 1.0 / 15120.0 : 0.0;
}
// the same weights rounded to FP32
struct P25f {
    __host__ __device__ constexpr float operator()(int e2) const { return (float)p25(e2); }
};
constexpr P25f p25f{};

template <typename real> __device__ __forceinline__ real psi_of(real r);
// psi = rho0 (1 - exp(-rho/rho0)), rho0 = 1 (Sec. II B)
template <> __device__ __forceinline__ double psi_of<double>(double r) { return 1.0 - exp(-r); }
// same function, written through expm1 so small densities keep their digits
template <> __device__ __forceinline__ float psi_of<float>(float r) { return -expm1f(-r); }

__device__ __forceinline__ int wrap_index(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

// Stage rho_k and psi_k of the tile plus its halo into shared memory from the
// density copy `rho`.  Periodic copies in x (and in y without walls); beyond a
// wall the ghost rows are either mirrored from the fluid or set to the fixed
// wall densities.
template <typename real, int SHv>
__device__ __forceinline__ void stage_tile(const Lat<real> &L, const real *__restrict__ rho, int x0, int y0,
                                           real (*srho)[SHv][SW], real (*spsi)[SHv][SW], int tid, int nthreads)
{
    constexpr int TYv = SHv - 2 * HALO;
    const int nx = L.nx, ny = L.ny;
    // tiles whose halo lies inside the lattice need no wrapping or ghosts
    const bool inner = x0 >= HALO && x0 + TX + HALO <= nx && y0 >= HALO && y0 + TYv + HALO <= ny;
    if (inner) {
        const real *__restrict__ base = rho + (size_t)(y0 - HALO) * L.pitch + (x0 - HALO);
        for (int idx = tid; idx < SW * SHv; idx += nthreads) {
            const int sx = idx % SW, sy = idx / SW;
            const size_t c = (size_t)sy * L.pitch + sx;
            const real rA = base[c], rB = base[L.plane + c];
            srho[0][sy][sx] = rA;
            srho[1][sy][sx] = rB;
            spsi[0][sy][sx] = psi_of<real>(rA);
            spsi[1][sy][sx] = psi_of<real>(rB);
        }
        return;
    }
    for (int idx = tid; idx < SW * SHv; idx += nthreads) {
        const int sx = idx % SW, sy = idx / SW;
        const int gx = wrap_index(x0 + sx - HALO, nx);
        int gy = y0 + sy - HALO;
        real rA, rB;
        bool fixed = false;
        if (gy < 0 || gy >= ny) {
            if (L.walls) {
                if (L.wall_mode == 1) {
                    rA = L.wall_rho[0];
                    rB = L.wall_rho[1];
                    fixed = true;
                } else {
                    gy = gy < 0 ? -1 - gy : 2 * ny - 1 - gy;
                    gy = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);  // rows no valid node reads
                }
            } else {
                gy = wrap_index(gy, ny);
            }
        }
        if (!fixed) {
            const size_t c = (size_t)gy * L.pitch + gx;
            rA = rho[c];
            rB = rho[L.plane + c];
        }
        srho[0][sy][sx] = rA;
        srho[1][sy][sx] = rB;
        spsi[0][sy][sx] = psi_of<real>(rA);
        spsi[1][sy][sx] = psi_of<real>(rB);
    }
}

// sum_{i=1..8} w_i s(x + e_i) e_i (Eqs. 8, 9).
// FP64: added in direction order.  FP32: differences of opposite neighbours.
template <typename real>
__device__ __forceinline__ void q9_sum(const real (*s)[SW], int cx, int cy, real &sx, real &sy)
{
    const real W1 = (real)(1.0 / 9.0), W2 = (real)(1.0 / 36.0);
    if constexpr (!kOffset<real>) {
        const real a1 = W1 * s[cy][cx + 1], a2 = W1 * s[cy + 1][cx], a3 = W1 * s[cy][cx - 1], a4 = W1 * s[cy - 1][cx];
        const real a5 = W2 * s[cy + 1][cx + 1], a6 = W2 * s[cy + 1][cx - 1];
        const real a7 = W2 * s[cy - 1][cx - 1], a8 = W2 * s[cy - 1][cx + 1];
        sx = ((((a1 - a3) + a5) - a6) - a7) + a8;
        sy = ((((a2 - a4) + a5) + a6) - a7) - a8;
    } else {
        (void)W1;
        (void)W2;
        vq9<float>([&](int dy, int dx) { return s[cy + dy][cx + dx]; }, sx, sy);
    }
}

// sum_j p_j s(x + e_j) e_j over D2Q25 (FP64), in raster order (dy outer, dx
// inner).  The FP32 step sums the psi terms with combined weights (vq25c).
template <typename real>
__device__ __forceinline__ void q25_sum(const real (*s)[SW], int cx, int cy, real &sx, real &sy)
{
    static_assert(!kOffset<real>, "FP64 only");
    sx = (real)0;
    sy = (real)0;
#pragma unroll
    for (int j = 0; j < 25; ++j) {
        const int dx = j % 5 - 2, dy = j / 5 - 2;
        if (dx == 0 && dy == 0) continue;
        const real pp = (real)p25(dx * dx + dy * dy) * s[cy + dy][cx + dx];
        if (dx != 0) sx += pp * (real)dx;
        if (dy != 0) sy += pp * (real)dy;
    }
}

// Total force on species k at the staged node (cx, cy): Eq. (8) + Eq. (9) + rho_k g.
template <typename real, int SHv>
__device__ __forceinline__ void force_at(const Lat<real> &L, const real (*srho)[SHv][SW], const real (*spsi)[SHv][SW],
                                         int k, int cx, int cy, real &Fx, real &Fy)
{
    const real psi = spsi[k][cy][cx], rho = srho[k][cy][cx];
    if constexpr (kOffset<real>) {
        // FP32: the two psi sums as one stencil with combined weights
        float msx, msy, s3x, s3y;
        const float(*sp)[SW] = spsi[k];
        vq25c<float>([&](int dy, int dx) { return sp[cy + dy][cx + dx]; }, L.cw, p25f, msx, msy);
        q9_sum<real>(srho[1 - k], cx, cy, s3x, s3y);
        vforce<float>(psi, rho, msx, msy, s3x, s3y, L.GAB, L.g[0], L.g[1], Fx, Fy);
    } else {
        real s1x, s1y, s2x, s2y, s3x, s3y;
        q9_sum<real>(spsi[k], cx, cy, s1x, s1y);
        q25_sum<real>(spsi[k], cx, cy, s2x, s2y);
        q9_sum<real>(srho[1 - k], cx, cy, s3x, s3y);
        const real G1 = L.G1, G2 = L.G2, GAB = L.GAB;
        Fx = -G1 * psi * s1x - G2 * psi * s2x - GAB * rho * s3x + rho * L.g[0];
        Fy = -G1 * psi * s1y - G2 * psi * s2y - GAB * rho * s3y + rho * L.g[1];
    }
}

// The staged density and psi tiles of the species as one [row][col] plane
// per species and field, as collide_site reads them: species k's density
// and force at a staged node, and rho_k(x) - rho_k(x + e), the difference a
// push re-references with.  collide_site asks for species 0, then 1.
template <typename real, int SHv>
struct SplitStage {
    const real (*srho)[SHv][SW];
    const real (*spsi)[SHv][SW];
    __device__ __forceinline__ real density(int k, int cy, int cx) const { return srho[k][cy][cx]; }
    __device__ __forceinline__ void force(const Lat<real> &L, int k, int cx, int cy, real &Fx, real &Fy) const
    {
        force_at<real, SHv>(L, srho, spsi, k, cx, cy, Fx, Fy);
    }
    // FP32: both species' forces and densities as (A, B) pairs
    __device__ __forceinline__ void force2(const Lat<float> &L, int cx, int cy, float2 &Fx, float2 &Fy) const
    {
        force_at<float, SHv>(L, srho, spsi, 0, cx, cy, Fx.x, Fy.x);
        force_at<float, SHv>(L, srho, spsi, 1, cx, cy, Fx.y, Fy.y);
    }
    __device__ __forceinline__ float2 density2(int cy, int cx) const
    {
        return make_float2(srho[0][cy][cx], srho[1][cy][cx]);
    }
    template <int EX, int EY>
    __device__ __forceinline__ real density_step(int k, int cx, int cy) const
    {
        return srho[k][cy][cx] - srho[k][cy + EY][cx + EX];
    }
    // FP32: both species' densities at the staged node (cx + EX, cy + EY)
    template <int EX, int EY>
    __device__ __forceinline__ float2 dest(int cx, int cy) const
    {
        return make_float2(srho[0][cy + EY][cx + EX], srho[1][cy + EY][cx + EX]);
    }
};

// e_i . u in the order e_x u_x + e_y u_y, zero products dropped.
template <typename real, int EX, int EY>
__device__ __forceinline__ real edot(real ux, real uy)
{
    if constexpr (EX == 0 && EY == 0) return (real)0;
    else if constexpr (EX == 0) return EY > 0 ? uy : -uy;
    else if constexpr (EY == 0) return EX > 0 ? ux : -ux;
    else return (EX > 0 ? ux : -ux) + (EY > 0 ? uy : -uy);
}

// (e_a - u_a)/cs^2 + (e.u) e_a / cs^4 for one component a.
template <typename real, int E>
__device__ __forceinline__ real guo_comp(real u, real eu)
{
    if constexpr (E == 0) return -((real)3 * u);
    else if constexpr (E > 0) return (real)3 * ((real)1 - u) + (real)9 * eu;
    else return (real)3 * ((real)-1 - u) - (real)9 * eu;
}

// BGK relaxation with Guo forcing for direction I of one species
// (Eqs. 1, 2, 5).  FP64: f -> f*.  FP32: the offset from the node's own
// density, f - w rho -> f* - w rho (its equilibrium is w rho (e.u terms)).
template <typename real, int I>
__device__ __forceinline__ real collide_dir(real f, real rho, real ux, real uy, real uu, real Fx, real Fy, real om,
                                            real aw)
{
    constexpr int EX = ex9(I), EY = ey9(I);
    const real w = (real)w9(I);
    const real eu = edot<real, EX, EY>(ux, uy);
    const real C = aw * (guo_comp<real, EX>(ux, eu) * Fx + guo_comp<real, EY>(uy, eu) * Fy);
    const real feq = w * rho * ((real)1 + (real)3 * eu + (real)4.5 * eu * eu - (real)1.5 * uu);
    return f - om * (f - feq) + C;
}

// Store the post-collision value of direction I of species k at x + e_i
// (half-way bounce-back: back to x, reversed).  FP32: re-reference the offset
// from rho(x) to rho(x + e_i), the reference the next step reads there
// (unless kReref is false: the caller did).
template <typename real, int I, bool kInner, class Stage, bool kReref = true>
__device__ __forceinline__ void push_dir(const Lat<real> &L, real *__restrict__ fn, const Stage &sg, int k, int x,
                                         int y, int cx, int cy, real v)
{
    constexpr int EX = ex9(I), EY = ey9(I);
    if constexpr (kOffset<real> && kReref && I != 0) {
        // the next step's reference at the destination is its density now
        if (kInner || !(EY != 0 && L.walls && (y + EY < 0 || y + EY >= L.ny)))
            v = cfma((float)w9(I), sg.template density_step<EX, EY>(k, cx, cy), v);
    }
    if constexpr (kInner) {
        // node and destination inside the lattice: a constant offset
        fn[(size_t)(k * 9 + I) * L.plane + ((size_t)y * L.pitch + x) + (EY * L.pitch + EX)] = v;
        return;
    } else {
        int xd = x + EX, yd = y + EY;
        if constexpr (EX != 0) {
            if (xd >= L.nx) xd -= L.nx;
            if (xd < 0) xd += L.nx;
        }
        int dir = I;
        if constexpr (EY != 0) {
            if (yd < 0 || yd >= L.ny) {
                if (L.walls) {       // half-way bounce-back: back to this node, reversed
                    dir = opp9(I);
                    xd = x;
                    yd = y;
                } else {
                    yd = yd < 0 ? yd + L.ny : yd - L.ny;
                }
            }
        }
        fn[(size_t)(k * 9 + dir) * L.plane + (size_t)yd * L.pitch + xd] = v;
    }
}

// Collision and push of direction I of both species (FP64), fk the node's
// populations; sg the staged densities.
template <typename real, int I, bool kInner, class Stage>
__device__ __forceinline__ void collide_push_dir(const Lat<real> &L, real *__restrict__ fn, const Stage &sg,
                                                 const real (&fk)[2][9], const real (&rho)[2], real ux, real uy,
                                                 real uu, const real (&F)[2][2], int x, int y, int cx, int cy)
{
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const real v = collide_dir<real, I>(fk[k][I], rho[k], ux, uy, uu, F[k][0], F[k][1], L.omega[k],
                                            L.aw[k][cls9(I)]);
        push_dir<real, I, kInner>(L, fn, sg, k, x, y, cx, cy, v);
    }
}

// Species momentum sum_i f e_i.  FP64: direction order, zero products
// dropped.  FP32: opposite-population differences.
template <typename real>
__device__ __forceinline__ void first_moment(const real (&f)[9], real &jx, real &jy)
{
    if constexpr (!kOffset<real>) {
        jx = ((((f[1] - f[3]) + f[5]) - f[6]) - f[7]) + f[8];
        jy = ((((f[2] - f[4]) + f[5]) + f[6]) - f[7]) - f[8];
    } else {
        vfirst<float>(f, jx, jy);
    }
}

template <typename real>
__device__ __forceinline__ real zeroth_moment(const real (&f)[9])
{
    if constexpr (!kOffset<real>) {
        return (((((((f[0] + f[1]) + f[2]) + f[3]) + f[4]) + f[5]) + f[6]) + f[7]) + f[8];
    } else {
        return vzeroth<float>(f);
    }
}

// ---- kernels ----------------------------------------------------------------

// Global loads of data that other blocks of the same launch may have written
// (the persistent kernel): through L2 only, never a stale L1 line.
template <bool kCG, typename real>
__device__ __forceinline__ real ldg_state(const real *p)
{
    if constexpr (kCG) return __ldcg(p);
    else return *p;
}

// rho_k = sum_i f_k,i of one tile into density copy parity^1 (FP32: R +
// sum_i h_i, R the density of the previous step in copy parity).
template <typename real, int TYv, bool kCG>
__device__ __forceinline__ void density_tile(const Lat<real> *__restrict__ lats, int4 t, int parity)
{
    const Lat<real> &L = lats[t.x];
    const int x = t.y + threadIdx.x, y = t.z + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const real *__restrict__ f = L.f[parity];
    const size_t c = (size_t)y * L.pitch + x;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        real v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = ldg_state<kCG>(&f[(size_t)(k * 9 + i) * L.plane + c]);
        real r = zeroth_moment<real>(v);
        if constexpr (kOffset<real>) r = ldg_state<kCG>(&L.rho[parity][(size_t)k * L.plane + c]) + r;
        L.rho[parity ^ 1][(size_t)k * L.plane + c] = r;
    }
}

template <typename real, int TYv>
__global__ void __launch_bounds__(TX *TYv) k_density(const Lat<real> *__restrict__ lats, const int4 *__restrict__ tiles,
                                                     int tile_offset, int parity)
{
    density_tile<real, TYv, false>(lats, tiles[tile_offset + blockIdx.x], parity);
}

// Shared memory of the fused kernel for a tile of height TYv.
template <typename real, int TYv>
struct CollideSmem {
    real srho[2][TYv + 2 * HALO][SW];
    real spsi[2][TYv + 2 * HALO][SW];
    Lat<real> L;   // descriptor copy: stores to the populations cannot alias it
};

// Moments of a node's FP32 offset populations that need no force, as
// (species A, species B) pairs: the first moment, the density change rho - R
// moved into the offsets and the offsets' residual sum dg after it
// (collide_site explains both).
struct NodeMoments {
    float2 jx, jy;
    float2 delta;
    float2 dg;
};

template <typename real, bool kInner, bool kBox = false, class Stage>
__device__ __forceinline__ void collide_site(const Lat<real> &L, real *__restrict__ fn, const Stage &sg,
                                             real (&fk)[2][9], const real (&Rn)[2], int x, int y, int cx, int cy,
                                             const real *__restrict__ box = nullptr, int box_plane = 0,
                                             const NodeMoments *pre = nullptr);

// Fused force + collision + push-streaming + bounce-back for one tile.  Every
// thread of the block calls it and returns from it; it ends after the tile's
// pushes are issued (the caller synchronises before reusing sm).
template <typename real, int TYv, bool kCG>
__device__ __forceinline__ void collide_tile(const Lat<real> *__restrict__ lats, int4 t, int parity,
                                             CollideSmem<real, TYv> &sm)
{
    const Lat<real> &G = lats[t.x];
    const int tid = threadIdx.y * TX + threadIdx.x;
    static_assert(sizeof(Lat<real>) % 4 == 0, "descriptor copied as 32-bit words");
    for (int i = tid; i < (int)(sizeof(Lat<real>) / 4); i += TX * TYv)
        reinterpret_cast<uint32_t *>(&sm.L)[i] = reinterpret_cast<const uint32_t *>(&G)[i];
    const int x = t.y + threadIdx.x, y = t.z + threadIdx.y;
    const bool valid = x < G.nx && y < G.ny;
    // issue the population loads first so their latency overlaps the staging
    const real *__restrict__ fc = G.f[parity];
    real *__restrict__ fn = G.f[parity ^ 1];
    const size_t c = valid ? (size_t)y * G.pitch + x : 0;
    real fk[2][9];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int i = 0; i < 9; ++i) fk[k][i] = valid ? ldg_state<kCG>(&fc[(size_t)(k * 9 + i) * G.plane + c]) : (real)0;
    if constexpr (kCG) {
        // staging reads the density copy through L2 as well
        constexpr int SHv = TYv + 2 * HALO;
        const int nx = G.nx, ny = G.ny;
        const real *__restrict__ rho = G.rho[parity ^ 1];
        for (int idx = tid; idx < SW * SHv; idx += TX * TYv) {
            const int sx = idx % SW, sy = idx / SW;
            const int gx = wrap_index(t.y + sx - HALO, nx);
            int gy = t.z + sy - HALO;
            real rA, rB;
            bool fixed = false;
            if (gy < 0 || gy >= ny) {
                if (G.walls) {
                    if (G.wall_mode == 1) {
                        rA = G.wall_rho[0];
                        rB = G.wall_rho[1];
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
                const size_t cc = (size_t)gy * G.pitch + gx;
                rA = __ldcg(&rho[cc]);
                rB = __ldcg(&rho[G.plane + cc]);
            }
            sm.srho[0][sy][sx] = rA;
            sm.srho[1][sy][sx] = rB;
            sm.spsi[0][sy][sx] = psi_of<real>(rA);
            sm.spsi[1][sy][sx] = psi_of<real>(rB);
        }
    } else {
        stage_tile<real, TYv + 2 * HALO>(G, G.rho[parity ^ 1], t.y, t.z, sm.srho, sm.spsi, tid, TX * TYv);
    }
    __syncthreads();
    if (!valid) return;
    const int cx = threadIdx.x + HALO, cy = threadIdx.y + HALO;
    real Rn[2] = {(real)0, (real)0};
    if constexpr (kOffset<real>) {
        Rn[0] = ldg_state<kCG>(&G.rho[parity][c]);
        Rn[1] = ldg_state<kCG>(&G.rho[parity][G.plane + c]);
    }
    // tiles whose pushes stay inside the lattice (no wrap, no wall) take constant offsets
    const bool inner = t.y >= 1 && t.y + TX + 1 <= sm.L.nx && t.z >= 1 && t.z + TYv + 1 <= sm.L.ny;
    const SplitStage<real, TYv + 2 * HALO> sg{sm.srho, sm.spsi};
    if (inner) collide_site<real, true>(sm.L, fn, sg, fk, Rn, x, y, cx, cy);
    else collide_site<real, false>(sm.L, fn, sg, fk, Rn, x, y, cx, cy);
}

template <typename real, int TYv>
__global__ void __launch_bounds__(TX *TYv, kCollideMinBlocks<real, TYv>)
    k_collide(const Lat<real> *__restrict__ lats, const int4 *__restrict__ tiles, int tile_offset, int parity)
{
    __shared__ CollideSmem<real, TYv> sm;
    collide_tile<real, TYv, false>(lats, tiles[tile_offset + blockIdx.x], parity, sm);
}

// The NodeMoments of a node from its offset populations h (both species as
// pairs), rho its densities and Rn its references: the same operations, in
// the same order, as collide_site's own.
__device__ __forceinline__ void node_moments(const float2 (&h)[9], float2 rho, float2 Rn, NodeMoments &nm)
{
    float2 f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = h[i];
    vfirst<float2>(f, nm.jx, nm.jy);
    nm.delta = vsub(rho, Rn);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = cfma(-(float)w9(i), nm.delta, f[i]);
    nm.dg = vzeroth<float2>(f);
}

// ---- velocity-shift forcing of the original model (FP64 only) ---------------

// Second-order equilibrium of direction I (Eq. 2), the same expression as
// collide_dir's.
template <typename real, int I>
__device__ __forceinline__ real feq_dir(real rho, real ux, real uy, real uu)
{
    constexpr int EX = ex9(I), EY = ey9(I);
    const real eu = edot<real, EX, EY>(ux, uy);
    return (real)w9(I) * rho * ((real)1 + (real)3 * eu + (real)4.5 * eu * eu - (real)1.5 * uu);
}

// BGK relaxation to f^eq(rho, u^eq) plus the velocity-shift term of Eq. (4),
// C = (1/tau) [f^eq(rho, u^eq + tau F / rho) - f^eq(rho, u^eq)], then the
// push of direction I of species k.
template <typename real, int I, bool kInner, class Stage>
__device__ __forceinline__ void shift_push_dir(const Lat<real> &L, real *__restrict__ fn, const Stage &sg, int k,
                                               real f, real rho, real ux, real uy, real uu, real sx, real sy, real ss,
                                               int x, int y, int cx, int cy)
{
    const real om = L.omega[k];
    const real feq = feq_dir<real, I>(rho, ux, uy, uu);
    const real feqs = feq_dir<real, I>(rho, sx, sy, ss);
    const real C = om * (feqs - feq);
    push_dir<real, I, kInner>(L, fn, sg, k, x, y, cx, cy, f - om * (f - feq) + C);
}

// The node's collision and pushes in the original model: u^eq of Eq. (3)
// from the momenta sum_i f e_i (no force), species k relaxed with the
// velocity-shift term of Eq. (4).
template <typename real, bool kInner, class Stage>
__device__ __forceinline__ void shift_collide_site(const Lat<real> &L, real *__restrict__ fn, const Stage &sg,
                                                   real (&fk)[2][9], int x, int y, int cx, int cy)
{
    real F[2][2], rho[2], m[2][2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        sg.force(L, k, cx, cy, F[k][0], F[k][1]);
        rho[k] = sg.density(k, cy, cx);
        first_moment<real>(fk[k], m[k][0], m[k][1]);
    }
    const real om0 = L.omega[0], om1 = L.omega[1];
    const real den = om0 * rho[0] + om1 * rho[1];
    const real ux = (om0 * m[0][0] + om1 * m[1][0]) / den;
    const real uy = (om0 * m[0][1] + om1 * m[1][1]) / den;
    const real uu = ux * ux + uy * uy;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const real sx = ux + L.tau[k] * F[k][0] / rho[k], sy = uy + L.tau[k] * F[k][1] / rho[k];
        const real ss = sx * sx + sy * sy;
        const real(&f)[9] = fk[k];
        const real r = rho[k];
        shift_push_dir<real, 0, kInner>(L, fn, sg, k, f[0], r, ux, uy, uu, sx, sy, ss, x, y, cx, cy);
        shift_push_dir<real, 1, kInner>(L, fn, sg, k, f[1], r, ux, uy, uu, sx, sy, ss, x, y, cx, cy);
        shift_push_dir<real, 2, kInner>(L, fn, sg, k, f[2], r, ux, uy, uu, sx, sy, ss, x, y, cx, cy);
        shift_push_dir<real, 3, kInner>(L, fn, sg, k, f[3], r, ux, uy, uu, sx, sy, ss, x, y, cx, cy);
        shift_push_dir<real, 4, kInner>(L, fn, sg, k, f[4], r, ux, uy, uu, sx, sy, ss, x, y, cx, cy);
        shift_push_dir<real, 5, kInner>(L, fn, sg, k, f[5], r, ux, uy, uu, sx, sy, ss, x, y, cx, cy);
        shift_push_dir<real, 6, kInner>(L, fn, sg, k, f[6], r, ux, uy, uu, sx, sy, ss, x, y, cx, cy);
        shift_push_dir<real, 7, kInner>(L, fn, sg, k, f[7], r, ux, uy, uu, sx, sy, ss, x, y, cx, cy);
        shift_push_dir<real, 8, kInner>(L, fn, sg, k, f[8], r, ux, uy, uu, sx, sy, ss, x, y, cx, cy);
    }
}

// Force, moments, u^eq, collision and push of the node (x, y), staged at
// (cx, cy).  Its populations are fk (updated in place), or with kBox (FP32)
// the shared-memory box: box[(k * 9 + i) * box_plane] is population i of
// species k, read again where it is used with the same density offset
// applied, which keeps 18 registers free; fk is then not used, and the
// force-free moments come precomputed in *pre (node_moments).
// The FP32 node collision: half-force momenta (Eq. 6), the offsets from the
// node's current density, u^eq and the terms shared by the directions, then
// the collision of each direction of both species and its push.
template <bool kInner, bool kBox, class Stage>
__device__ __forceinline__ void collide_site_off(const Lat<float> &L, float *__restrict__ fn, const Stage &sg,
                                                 float (&fk)[2][9], const float (&Rn)[2], int x, int y, int cx, int cy,
                                                 const float *__restrict__ box, int box_plane, const NodeMoments *pre)
{
    // both species at once, as (A, B) pairs
    float2 Fx, Fy, jx, jy, delta, dg;
    sg.force2(L, cx, cy, Fx, Fy);
    const float2 rho = sg.density2(cy, cx);
    float2 h[9];
    if constexpr (kBox) {
        (void)fk;
        (void)Rn;
        jx = pre->jx;
        jy = pre->jy;
        delta = pre->delta;
        dg = pre->dg;
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = make_float2(fk[0][i], fk[1][i]);
        vfirst<float2>(h, jx, jy);   // the reference density adds no momentum
        // offsets from the node's current density: h_i - w_i (rho - R).
        // rho - R is formed from the rounded density itself (exact: the two
        // are close), so f = h + w R is kept exactly whatever rho rounded to;
        // with sum_i h_i instead, density changes below half an ulp of R
        // would be dropped at every step and mass would drift.
        delta = vsub(rho, make_float2(Rn[0], Rn[1]));
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = cfma(-(float)w9(i), delta, h[i]);
        dg = vzeroth<float2>(h);
    }
    const float2 mx = cfma(0.5f, Fx, jx);   // Eq. (6), half force
    const float2 my = cfma(0.5f, Fy, jy);
    // the lattice constants of the collision, read once: stores to the
    // populations may alias shared memory as far as the compiler knows
    const float2 om = make_float2(L.omega[0], L.omega[1]);
    const float2 aw3[3] = {make_float2(L.aw3[0][0], L.aw3[1][0]), make_float2(L.aw3[0][1], L.aw3[1][1]),
                           make_float2(L.aw3[0][2], L.aw3[1][2])};
    OffTerms t;
    off_terms(om, rho, mx, my, Fx, Fy, dg, t);
    const size_t plane = L.plane;
    const int pitch = L.pitch;
    float *node = fn + ((size_t)y * pitch + x);
    // the populations of direction I, as the moments saw them
    auto pop = [&](int I) -> float2 {
        if constexpr (kBox)
            return cfma(-(float)w9(I), delta, make_float2(box[I * box_plane], box[(9 + I) * box_plane]));
        else return h[I];
    };
    auto dir = [&](auto Ic) {
        constexpr int I = decltype(Ic)::value;
        float2 v = off_collide<I>(t, om, aw3[cls9(I)], pop(I));
        // re-reference from rho(x) to rho(x + e_i), the reference the next
        // step reads there (not for a push that bounces back from a wall)
        constexpr int EX = ex9(I), EY = ey9(I);
        if constexpr (I != 0) {
            if (kInner || !(EY != 0 && L.walls && (y + EY < 0 || y + EY >= L.ny)))
                v = cfma((float)w9(I), vsub(rho, sg.template dest<EX, EY>(cx, cy)), v);
        }
        if constexpr (kInner) {
            // destination inside the lattice: a constant offset
            node[(size_t)I * plane + (EY * pitch + EX)] = v.x;
            node[(size_t)(9 + I) * plane + (EY * pitch + EX)] = v.y;
        } else {
            push_dir<float, I, kInner, Stage, false>(L, fn, sg, 0, x, y, cx, cy, v.x);
            push_dir<float, I, kInner, Stage, false>(L, fn, sg, 1, x, y, cx, cy, v.y);
        }
    };
    dir(std::integral_constant<int, 0>{});
    dir(std::integral_constant<int, 1>{});
    dir(std::integral_constant<int, 2>{});
    dir(std::integral_constant<int, 3>{});
    dir(std::integral_constant<int, 4>{});
    dir(std::integral_constant<int, 5>{});
    dir(std::integral_constant<int, 6>{});
    dir(std::integral_constant<int, 7>{});
    dir(std::integral_constant<int, 8>{});
}

// Force, moments, u^eq, collision and push of the node (x, y), staged at
// (cx, cy).  Its populations are fk (updated in place), or with kBox (FP32)
// the shared-memory box: box[(k * 9 + i) * box_plane] is population i of
// species k, read again where it is used with the same density offset
// applied, which keeps 18 registers free; fk is then not used, and the
// force-free moments come precomputed in *pre (node_moments).
template <typename real, bool kInner, bool kBox, class Stage>
__device__ __forceinline__ void collide_site(const Lat<real> &L, real *__restrict__ fn, const Stage &sg,
                                             real (&fk)[2][9], const real (&Rn)[2], int x, int y, int cx, int cy,
                                             const real *__restrict__ box, int box_plane, const NodeMoments *pre)
{
    static_assert(!kBox || kOffset<real>, "the box form is FP32 only");
    if constexpr (kOffset<real>) {
        collide_site_off<kInner, kBox>(L, fn, sg, fk, Rn, x, y, cx, cy, box, box_plane, pre);
    } else {
        (void)Rn;
        (void)box;
        (void)box_plane;
        (void)pre;
        if (L.forcing == 1) {   // the original model (Eq. 4), a block-uniform branch
            shift_collide_site<real, kInner>(L, fn, sg, fk, x, y, cx, cy);
            return;
        }
        real F[2][2], rho[2], m[2][2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            sg.force(L, k, cx, cy, F[k][0], F[k][1]);
            rho[k] = sg.density(k, cy, cx);
            real jx, jy;
            first_moment<real>(fk[k], jx, jy);
            m[k][0] = jx + (real)0.5 * F[k][0];   // Eq. (6), half force
            m[k][1] = jy + (real)0.5 * F[k][1];
        }
        // common velocity, Eq. (3)
        const real om0 = L.omega[0], om1 = L.omega[1];
        const real den = om0 * rho[0] + om1 * rho[1];
        const real ux = (om0 * m[0][0] + om1 * m[1][0]) / den;
        const real uy = (om0 * m[0][1] + om1 * m[1][1]) / den;
        const real uu = ux * ux + uy * uy;
        collide_push_dir<real, 0, kInner>(L, fn, sg, fk, rho, ux, uy, uu, F, x, y, cx, cy);
        collide_push_dir<real, 1, kInner>(L, fn, sg, fk, rho, ux, uy, uu, F, x, y, cx, cy);
        collide_push_dir<real, 2, kInner>(L, fn, sg, fk, rho, ux, uy, uu, F, x, y, cx, cy);
        collide_push_dir<real, 3, kInner>(L, fn, sg, fk, rho, ux, uy, uu, F, x, y, cx, cy);
        collide_push_dir<real, 4, kInner>(L, fn, sg, fk, rho, ux, uy, uu, F, x, y, cx, cy);
        collide_push_dir<real, 5, kInner>(L, fn, sg, fk, rho, ux, uy, uu, F, x, y, cx, cy);
        collide_push_dir<real, 6, kInner>(L, fn, sg, fk, rho, ux, uy, uu, F, x, y, cx, cy);
        collide_push_dir<real, 7, kInner>(L, fn, sg, fk, rho, ux, uy, uu, F, x, y, cx, cy);
        collide_push_dir<real, 8, kInner>(L, fn, sg, fk, rho, ux, uy, uu, F, x, y, cx, cy);
    }
}

// ---- one-pass step ------------------------------------------------------------

// Density of node (gx, gy) straight from its populations (FP32: plus its
// reference density): the same sum, in the same order, as the density pass.
template <typename real, bool kCG>
__device__ __forceinline__ real node_density(const Lat<real> &L, int k, int gx, int gy, int parity)
{
    const size_t c = (size_t)gy * L.pitch + gx;
    const real *__restrict__ f = L.f[parity];
    real v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = ldg_state<kCG>(&f[(size_t)(k * 9 + i) * L.plane + c]);
    real r = zeroth_moment<real>(v);
    if constexpr (kOffset<real>) r = ldg_state<kCG>(&L.rho[parity][(size_t)k * L.plane + c]) + r;
    return r;
}

// Densities of staged slot (sx, sy) of tile t (slot (HALO, HALO) is the
// tile's first node) from the populations of its node: x wraps; beyond the
// lattice in y, periodic wrap, or a wall ghost row (the mirrored fluid row,
// or the fixed wall densities).
template <typename real, bool kCG>
__device__ __forceinline__ void slot_densities(const Lat<real> &G, int4 t, int parity, int sx, int sy, real &rA,
                                               real &rB)
{
    const int nx = G.nx, ny = G.ny;
    const int gx = wrap_index(t.y + sx - HALO, nx);
    int gy = t.z + sy - HALO;
    if (gy < 0 || gy >= ny) {
        if (G.walls) {
            if (G.wall_mode == 1) {
                rA = G.wall_rho[0];
                rB = G.wall_rho[1];
                return;
            }
            gy = gy < 0 ? -1 - gy : 2 * ny - 1 - gy;
            gy = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);  // rows no valid node reads
        } else {
            gy = wrap_index(gy, ny);
        }
    }
    rA = node_density<real, kCG>(G, 0, gx, gy, parity);
    rB = node_density<real, kCG>(G, 1, gx, gy, parity);
}

// The same, staged with psi into the tile's density and psi planes.
template <typename real, int TYv, bool kCG>
__device__ __forceinline__ void stage_slot(const Lat<real> &G, int4 t, int parity, CollideSmem<real, TYv> &sm, int sx,
                                           int sy)
{
    real rA, rB;
    slot_densities<real, kCG>(G, t, parity, sx, sy, rA, rB);
    sm.srho[0][sy][sx] = rA;
    sm.srho[1][sy][sx] = rB;
    sm.spsi[0][sy][sx] = psi_of<real>(rA);
    sm.spsi[1][sy][sx] = psi_of<real>(rB);
}

// One time step of one tile in a single pass: each thread forms its node's
// densities from the populations it loads anyway; the 2-node halo (and the
// slots of a ragged tile's missing nodes) is formed from the neighbours'
// populations, mostly L2 hits.  The halo goes first, so that its loads and
// the node's own 18 populations are not held in registers at the same time.
// FP32 writes the node's density as the next step's reference.  Then the
// fused force + collision + push of collide_site.
template <typename real, int TYv, bool kCG>
__device__ __forceinline__ void fused_tile(const Lat<real> *__restrict__ lats, int4 t, int parity,
                                           CollideSmem<real, TYv> &sm)
{
    constexpr int SHv = TYv + 2 * HALO;
    const Lat<real> &G = lats[t.x];
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int i = tid; i < (int)(sizeof(Lat<real>) / 4); i += TX * TYv)
        reinterpret_cast<uint32_t *>(&sm.L)[i] = reinterpret_cast<const uint32_t *>(&G)[i];
    const int nx = G.nx, ny = G.ny;
    const int x = t.y + threadIdx.x, y = t.z + threadIdx.y;
    const bool valid = x < nx && y < ny;
    const real *__restrict__ fc = G.f[parity];
    real *__restrict__ fn = G.f[parity ^ 1];
    const size_t c = valid ? (size_t)y * G.pitch + x : 0;
    // the halo ring, enumerated compactly: two rows above, two below, then
    // the two columns on each side of the tile's rows
    constexpr int kRing = 4 * SW + 4 * TYv;
    for (int h = tid; h < kRing; h += TX * TYv) {
        int sx, sy;
        if (h < 2 * SW) {
            sy = h / SW;
            sx = h % SW;
        } else if (h < 4 * SW) {
            sy = TYv + HALO + (h - 2 * SW) / SW;
            sx = (h - 2 * SW) % SW;
        } else {
            const int q = h - 4 * SW;
            sy = HALO + q / 4;
            sx = (q % 4 < 2) ? q % 4 : TX + q % 4;
        }
        stage_slot<real, TYv, kCG>(G, t, parity, sm, sx, sy);
    }
    // a ragged tile's slots without a node of their own hold wrapped copies
    if (t.y + TX > nx || t.z + TYv > ny) {
        for (int q = tid; q < TX * TYv; q += TX * TYv) {
            const int sx = HALO + q % TX, sy = HALO + q / TX;
            if (t.y + sx - HALO >= nx || t.z + sy - HALO >= ny) stage_slot<real, TYv, kCG>(G, t, parity, sm, sx, sy);
        }
    }
    // then the node's own populations (kept in registers for the collision)
    real fk[2][9];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int i = 0; i < 9; ++i) fk[k][i] = valid ? ldg_state<kCG>(&fc[(size_t)(k * 9 + i) * G.plane + c]) : (real)0;
    const int cx = threadIdx.x + HALO, cy = threadIdx.y + HALO;
    real Rn[2] = {(real)0, (real)0};
    if (valid) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            real r = zeroth_moment<real>(fk[k]);
            if constexpr (kOffset<real>) {
                Rn[k] = ldg_state<kCG>(&G.rho[parity][(size_t)k * G.plane + c]);
                r = Rn[k] + r;
                G.rho[parity ^ 1][(size_t)k * G.plane + c] = r;
            }
            sm.srho[k][cy][cx] = r;
            sm.spsi[k][cy][cx] = psi_of<real>(r);
        }
    }
    __syncthreads();
    if (!valid) return;
    const bool inner = t.y >= 1 && t.y + TX + 1 <= sm.L.nx && t.z >= 1 && t.z + TYv + 1 <= sm.L.ny;
    const SplitStage<real, SHv> sg{sm.srho, sm.spsi};
    if (inner) collide_site<real, true>(sm.L, fn, sg, fk, Rn, x, y, cx, cy);
    else collide_site<real, false>(sm.L, fn, sg, fk, Rn, x, y, cx, cy);
}

template <typename real, int TYv>
__global__ void __launch_bounds__(TX *TYv, kCollideMinBlocks<real, TYv>)
    k_fused(const Lat<real> *__restrict__ lats, const int4 *__restrict__ tiles, int tile_offset, int parity)
{
    __shared__ CollideSmem<real, TYv> sm;
    fused_tile<real, TYv, false>(lats, tiles[tile_offset + blockIdx.x], parity, sm);
}

// ---- persistent launch over many time steps -----------------------------------

// Bounded wait until *ctr >= need.  Gives up when another block has flagged an
// error or after `limit` SM clock cycles, then flags LB_ETIMEOUT in *err.
__device__ __forceinline__ bool wait_geq(const unsigned *ctr, unsigned need, int *err, long long limit)
{
    if (need == 0) return true;
    const long long start = clock64();
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= need) return true;
        if (*(volatile int *)err) return false;
        if (clock64() - start > limit) {
            atomicExch(err, 1);
            return false;
        }
        __nanosleep(128);
    }
}

// Control block of a persistent launch (device memory, cleared before each
// launch): the work-queue head, then per-lattice counts of finished density
// and fused tiles.  The error word lives separately and survives launches.
struct PersistCtl {
    unsigned long long head;
};

// Advance nsteps time steps of every lattice in one launch.  Work items are
// (step, phase, tile) in this order, handed out by an atomic queue; an item
// waits only for the items of its own lattice it depends on (the density
// pass of step t waits for all fused tiles of step t-1, the fused tiles of
// step t for all density tiles of step t).  Every item it waits for has a
// smaller index and was claimed by a running block, so the wait always ends
// unless a block fails to signal; then the bounded wait flags the error and
// every block leaves.  drop_tile >= 0 makes that tile never signal (a test of
// the timeout path).
template <typename real, int TYv>
__global__ void __launch_bounds__(TX *TYv, kCollideMinBlocks<real, TYv>)
    k_persistent(const Lat<real> *__restrict__ lats, const int4 *__restrict__ tiles, const int *__restrict__ lat_ntiles,
                 int n_tiles, int nsteps, int parity0, PersistCtl *ctl, unsigned *dens_done, unsigned *coll_done,
                 int *err, long long wait_cycles, int drop_tile)
{
    __shared__ CollideSmem<real, TYv> sm;
    __shared__ long long s_item;
    __shared__ int s_ok;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const long long total = (long long)nsteps * 2 * n_tiles;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&ctl->head, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        const int t = (int)(item / (2 * n_tiles));
        const int r = (int)(item % (2 * n_tiles));
        const int phase = r / n_tiles, tile = r % n_tiles;
        const int4 tl = tiles[tile];
        const int nt_l = lat_ntiles[tl.x];
        const int parity = (parity0 + t) & 1;
        if (tid == 0) {
            const bool ok = phase == 0 ? wait_geq(&coll_done[tl.x], (unsigned)(t * nt_l), err, wait_cycles)
                                       : wait_geq(&dens_done[tl.x], (unsigned)((t + 1) * nt_l), err, wait_cycles);
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        if (phase == 0) density_tile<real, TYv, true>(lats, tl, parity);
        else collide_tile<real, TYv, true>(lats, tl, parity, sm);
        __syncthreads();
        if (tid == 0 && tile != drop_tile) {
            __threadfence();
            atomicAdd(phase == 0 ? &dens_done[tl.x] : &coll_done[tl.x], 1u);
        }
    }
}

// ---- observables ------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Per-node diagnostics (densities, momenta with half force, barycentric
// velocity, Eq. 11 bulk pressure) reduced per tile into FP64 partial sums;
// optionally also written as dense FP64 fields [..][ny][nx].  Reads the
// density copy parity^1 written by a density pass at the same time.
template <typename real>
__global__ void __launch_bounds__(kThreads) k_observe(const Lat<real> *__restrict__ lats, const int4 *__restrict__ tiles,
                                                      int tile_offset, int parity, double *__restrict__ partials,
                                                      double *__restrict__ out_rho, double *__restrict__ out_mom,
                                                      double *__restrict__ out_ubar)
{
    __shared__ real srho[2][SH][SW];
    __shared__ real spsi[2][SH][SW];
    __shared__ double sacc[kThreads / 32][kAccStride];
    const int4 t = tiles[tile_offset + blockIdx.x];
    const Lat<real> &L = lats[t.x];
    const int tid = threadIdx.y * TX + threadIdx.x;
    stage_tile<real, SH>(L, L.rho[parity ^ 1], t.y, t.z, srho, spsi, tid, kThreads);
    __syncthreads();
    const int x = t.y + threadIdx.x, y = t.z + threadIdx.y;
    double acc[kNumAcc];
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) acc[a] = 0.0;
    if (x < L.nx && y < L.ny) {
        const int cx = threadIdx.x + HALO, cy = threadIdx.y + HALO;
        const real *__restrict__ fc = L.f[parity];
        const size_t c = (size_t)y * L.pitch + x;
        double r[2], m[2][2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            real fk[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) fk[i] = fc[(size_t)(k * 9 + i) * L.plane + c];
            real Fx, Fy, jx, jy;
            force_at<real, SH>(L, srho, spsi, k, cx, cy, Fx, Fy);
            first_moment<real>(fk, jx, jy);   // FP32: the reference density adds no momentum
            r[k] = (double)srho[k][cy][cx];
            m[k][0] = (double)(jx + (real)0.5 * Fx);
            m[k][1] = (double)(jy + (real)0.5 * Fy);
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
            const double Gs = (double)L.G1 + (double)L.G2;
            const double pb = (r[0] + 0.5 * Gs * psiA * psiA) / 3.0 + (r[1] + 0.5 * Gs * psiB * psiB) / 3.0
                            + (double)L.GAB * r[0] * r[1] / 3.0;
            if (rr < 0.5 * R) { acc[kPIn] = pb; acc[kAIn] = r[0]; acc[kNIn] = 1.0; }
            if (rr > R + 6.0) { acc[kPOut] = pb; acc[kAOut] = r[0]; acc[kNOut] = 1.0; }
        }
        if (out_rho) {
            const size_t n = (size_t)L.nx * L.ny, d = (size_t)y * L.nx + x;
            out_rho[d] = r[0];
            out_rho[n + d] = r[1];
            if (out_mom) {
                out_mom[d] = m[0][0];
                out_mom[n + d] = m[0][1];
                out_mom[2 * n + d] = m[1][0];
                out_mom[3 * n + d] = m[1][1];
            }
            if (out_ubar) {
                out_ubar[d] = ux;
                out_ubar[n + d] = uy;
            }
        }
    }
    if (!partials) return;
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) {
        const double v = (a == kUmax) ? warp_max(acc[a]) : warp_sum(acc[a]);
        if (lane == 0) sacc[warp][a] = v;
    }
    __syncthreads();
    if (tid < kNumAcc) {
        double v = sacc[0][tid];
        for (int w = 1; w < kThreads / 32; ++w) v = (tid == kUmax) ? fmax(v, sacc[w][tid]) : v + sacc[w][tid];
        partials[(size_t)(tile_offset + blockIdx.x) * kAccStride + tid] = v;
    }
}

// One block per lattice: reduce its tile partials in a fixed order and
// derive the observables.
template <typename real>
__global__ void __launch_bounds__(256) k_finalize(const Lat<real> *__restrict__ lats, const double *__restrict__ partials,
                                                  double *__restrict__ obs)
{
    __shared__ double sred[256 / 32][kAccStride];
    const Lat<real> &L = lats[blockIdx.x];
    const int tid = threadIdx.x;
    double acc[kNumAcc];
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) acc[a] = 0.0;
    for (int tl = L.tile_begin + tid; tl < L.tile_end; tl += 256) {
#pragma unroll
        for (int a = 0; a < kNumAcc; ++a) {
            const double v = partials[(size_t)tl * kAccStride + a];
            acc[a] = (a == kUmax) ? fmax(acc[a], v) : acc[a] + v;
        }
    }
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
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
    double *o = obs + (size_t)blockIdx.x * kObsStride;
    o[oMassA] = s[kMassA];
    o[oMassB] = s[kMassB];
    o[oMomAx] = s[kMomAx];
    o[oMomAy] = s[kMomAy];
    o[oMomBx] = s[kMomBx];
    o[oMomBy] = s[kMomBy];
    o[oQ] = s[kSumUx] / L.nx;
    if (L.walls && L.g_x != 0.0) {
        const double H = L.ny, nuB = (L.tau_B - 0.5) / 3.0;
        const double Q0 = L.g_x * (H * H * H + 0.5 * H) / (12.0 * nuB);
        o[oMuR] = Q0 / o[oQ];
    } else {
        o[oMuR] = __longlong_as_double(0x7ff8000000000000ll);
    }
    if (L.has_probe && s[kNIn] > 0.0 && s[kNOut] > 0.0) {
        const double rin = s[kAIn] / s[kNIn], rout = s[kAOut] / s[kNOut];
        o[oDp] = s[kPIn] / s[kNIn] - s[kPOut] / s[kNOut];
        o[oReff] = sqrt((s[kMassA] - rout * (double)L.nx * (double)L.ny) / (3.14159265358979323846 * (rin - rout)));
    } else {
        o[oDp] = __longlong_as_double(0x7ff8000000000000ll);
        o[oReff] = __longlong_as_double(0x7ff8000000000000ll);
    }
    o[oUmax] = s[kUmax];
    o[oFinite] = s[kNonFinite] == 0.0 ? 1.0 : 0.0;
}

// ---- pressure tensor (Sec. II B-C) --------------------------------------------

// Slots of the pressure-tensor partial sums, per tile and per lattice.
enum PSlot { pKinXX = 0, pKinYY, pKinXY, pIntXX, pIntYY, pIntXY, kNumPSlots };
constexpr int kPStride = 8;

// Second moments sum_i w_i s(x + e_i) e_ia e_ib of a staged plane over the
// D2Q9 neighbours (xx, yy, xy), in FP64.
template <typename real>
__device__ __forceinline__ void q9_second(const real (*s)[SW], int cx, int cy, double (&m)[3])
{
    const double W1 = 1.0 / 9.0, W2 = 1.0 / 36.0;
    const double e = s[cy][cx + 1], w = s[cy][cx - 1], n = s[cy + 1][cx], so = s[cy - 1][cx];
    const double ne = s[cy + 1][cx + 1], nw = s[cy + 1][cx - 1], sw = s[cy - 1][cx - 1], se = s[cy - 1][cx + 1];
    const double diag = (ne + nw) + (sw + se);
    m[0] = W1 * (e + w) + W2 * diag;
    m[1] = W1 * (n + so) + W2 * diag;
    m[2] = W2 * ((ne + sw) - (nw + se));
}

// The same over the D2Q25 neighbours with the weights p(|e|^2).
template <typename real>
__device__ __forceinline__ void q25_second(const real (*s)[SW], int cx, int cy, double (&m)[3])
{
    m[0] = m[1] = m[2] = 0.0;
#pragma unroll
    for (int j = 0; j < 25; ++j) {
        const int dx = j % 5 - 2, dy = j / 5 - 2;
        if (dx == 0 && dy == 0) continue;
        const double a = p25(dx * dx + dy * dy) * (double)s[cy + dy][cx + dx];
        m[0] += a * (double)(dx * dx);
        m[1] += a * (double)(dy * dy);
        m[2] += a * (double)(dx * dy);
    }
}

// Per node, in FP64: the kinetic pressure tensor sum_k sum_i f e_a e_b of the
// pre-collision populations (Eq. 13) and the interaction tensor
//   P^int_ab = 1/2 sum_k [G1 psi_k S1_ab + G2 psi_k S2_ab + G_AB rho_k S3_ab],
// S1, S2 the D2Q9 and D2Q25 second moments of psi_k and S3 the D2Q9 second
// moment of the other species' density: each pair interaction of Eqs. (8),
// (9) shared equally by its two nodes, which gives the bulk pressure of
// Eq. (11) in a uniform state and satisfies Eq. (12) summed across a flat
// interface.  Reduced per tile into FP64 partials (slots PSlot); optionally
// also written as dense fields out[2][3][ny][nx] (kinetic, interaction; xx,
// yy, xy).  Reads the density copy parity^1 written by a density pass at the
// same time.
template <typename real>
__global__ void __launch_bounds__(kThreads) k_pressure(const Lat<real> *__restrict__ lats, const int4 *__restrict__ tiles,
                                                       int tile_offset, int parity, double *__restrict__ partials,
                                                       double *__restrict__ out)
{
    __shared__ real srho[2][SH][SW];
    __shared__ real spsi[2][SH][SW];
    __shared__ double sacc[kThreads / 32][kPStride];
    const int4 t = tiles[tile_offset + blockIdx.x];
    const Lat<real> &L = lats[t.x];
    const int tid = threadIdx.y * TX + threadIdx.x;
    stage_tile<real, SH>(L, L.rho[parity ^ 1], t.y, t.z, srho, spsi, tid, kThreads);
    __syncthreads();
    const int x = t.y + threadIdx.x, y = t.z + threadIdx.y;
    double acc[kNumPSlots];
#pragma unroll
    for (int a = 0; a < kNumPSlots; ++a) acc[a] = 0.0;
    if (x < L.nx && y < L.ny) {
        const int cx = threadIdx.x + HALO, cy = threadIdx.y + HALO;
        const real *__restrict__ fc = L.f[parity];
        const size_t c = (size_t)y * L.pitch + x;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const double R = kOffset<real> ? (double)L.rho[parity][(size_t)k * L.plane + c] : 0.0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const double fi = (double)fc[(size_t)(k * 9 + i) * L.plane + c] + w9(i) * R;
                acc[pKinXX] += fi * (double)(ex9(i) * ex9(i));
                acc[pKinYY] += fi * (double)(ey9(i) * ey9(i));
                acc[pKinXY] += fi * (double)(ex9(i) * ey9(i));
            }
            double s1[3], s2[3], s3[3];
            q9_second<real>(spsi[k], cx, cy, s1);
            q25_second<real>(spsi[k], cx, cy, s2);
            q9_second<real>(srho[1 - k], cx, cy, s3);
            const double psi = spsi[k][cy][cx], rho = srho[k][cy][cx];
            const double G1 = L.G1, G2 = L.G2, GAB = L.GAB;
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[pIntXX + a] += 0.5 * (G1 * psi * s1[a] + G2 * psi * s2[a] + GAB * rho * s3[a]);
        }
        if (out) {
            const size_t n = (size_t)L.nx * L.ny, d = (size_t)y * L.nx + x;
#pragma unroll
            for (int a = 0; a < kNumPSlots; ++a) out[(size_t)a * n + d] = acc[a];
        }
    }
    if (!partials) return;
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int a = 0; a < kNumPSlots; ++a) {
        const double v = warp_sum(acc[a]);
        if (lane == 0) sacc[warp][a] = v;
    }
    __syncthreads();
    if (tid < kNumPSlots) {
        double v = sacc[0][tid];
        for (int w = 1; w < kThreads / 32; ++w) v += sacc[w][tid];
        partials[(size_t)(tile_offset + blockIdx.x) * kPStride + tid] = v;
    }
}

// One block per lattice: the pressure-tensor partials of its tiles summed in
// a fixed order into out[lattice * kPStride + slot].
template <typename real>
__global__ void __launch_bounds__(256) k_pressure_sum(const Lat<real> *__restrict__ lats,
                                                      const double *__restrict__ partials, double *__restrict__ out)
{
    __shared__ double sred[256 / 32][kPStride];
    const Lat<real> &L = lats[blockIdx.x];
    const int tid = threadIdx.x;
    double acc[kNumPSlots];
#pragma unroll
    for (int a = 0; a < kNumPSlots; ++a) acc[a] = 0.0;
    for (int tl = L.tile_begin + tid; tl < L.tile_end; tl += 256)
#pragma unroll
        for (int a = 0; a < kNumPSlots; ++a) acc[a] += partials[(size_t)tl * kPStride + a];
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int a = 0; a < kNumPSlots; ++a) {
        const double v = warp_sum(acc[a]);
        if (lane == 0) sred[warp][a] = v;
    }
    __syncthreads();
    if (tid < kNumPSlots) {
        double v = sred[0][tid];
        for (int w = 1; w < 8; ++w) v += sred[w][tid];
        out[(size_t)blockIdx.x * kPStride + tid] = v;
    }
}

// ---- initialisation and population transfer ---------------------------------

// f_k,i = f^eq_i(rho_k, u) (Eq. 2) from dense FP64 fields.  FP32 stores the
// reference R = rho (rounded) in density copy `parity` and h = f^eq - w R.
template <typename real>
__global__ void k_init(const Lat<real> *__restrict__ lats, int lat, const double *__restrict__ rho,
                       const double *__restrict__ u, int parity)
{
    const Lat<real> &L = lats[lat];
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const size_t n = (size_t)L.nx * L.ny, d = (size_t)y * L.nx + x;
    const double ux = u ? u[d] : 0.0, uy = u ? u[n + d] : 0.0;
    const double uu = ux * ux + uy * uy;
    real *f = L.f[parity];
    const size_t c = (size_t)y * L.pitch + x;
    for (int k = 0; k < 2; ++k) {
        const double r = rho[k * n + d];
        double R = 0.0;
        if constexpr (kOffset<real>) {
            const real Rr = (real)r;
            L.rho[parity][(size_t)k * L.plane + c] = Rr;
            R = (double)Rr;
        }
        for (int i = 0; i < 9; ++i) {
            const double eu = ex9(i) * ux + ey9(i) * uy;
            const double feq = w9(i) * r * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
            f[(size_t)(k * 9 + i) * L.plane + c] = (real)(feq - w9(i) * R);
        }
    }
}

// dense FP64 [2][9][ny][nx] <-> native pitched populations (FP32: the
// reference density added back, or recomputed as sum_i f_i on input).
template <typename real>
__global__ void k_get_pops(const Lat<real> *__restrict__ lats, int lat, int parity, double *__restrict__ out)
{
    const Lat<real> &L = lats[lat];
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const size_t n = (size_t)L.nx * L.ny, d = (size_t)y * L.nx + x, c = (size_t)y * L.pitch + x;
    for (int k = 0; k < 2; ++k) {
        const double R = kOffset<real> ? (double)L.rho[parity][(size_t)k * L.plane + c] : 0.0;
        for (int i = 0; i < 9; ++i)
            out[(size_t)(k * 9 + i) * n + d] = (double)L.f[parity][(size_t)(k * 9 + i) * L.plane + c] + w9(i) * R;
    }
}

template <typename real>
__global__ void k_set_pops(const Lat<real> *__restrict__ lats, int lat, int parity, const double *__restrict__ in)
{
    const Lat<real> &L = lats[lat];
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const size_t n = (size_t)L.nx * L.ny, d = (size_t)y * L.nx + x, c = (size_t)y * L.pitch + x;
    for (int k = 0; k < 2; ++k) {
        double R = 0.0;
        if constexpr (kOffset<real>) {
            double s = 0.0;
            for (int i = 0; i < 9; ++i) s += in[(size_t)(k * 9 + i) * n + d];
            const real Rr = (real)s;
            L.rho[parity][(size_t)k * L.plane + c] = Rr;
            R = (double)Rr;
        }
        for (int i = 0; i < 9; ++i)
            L.f[parity][(size_t)(k * 9 + i) * L.plane + c] = (real)(in[(size_t)(k * 9 + i) * n + d] - w9(i) * R);
    }
}

}  // namespace lbk

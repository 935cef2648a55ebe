// lb_adjoint.cu -- discrete adjoint of one FP64 time step of the two-range
// pseudopotential lattice Boltzmann method (the step of lb_kernels.cuh:
// Eqs. 1-3, 5, 6, 8, 9 and half-way bounce-back), for gradients of an
// observable with respect to theta = (G_AB, G1, G2, tau_A, tau_B).
//
// Forward step at node x (species k, direction i):
//   rho_k = sum_i f_k,i,  psi_k = 1 - exp(-rho_k)
//   S1_k = sum_i w_i psi_k(x+e_i) e_i,  S2_k = sum_j p_j psi_k(x+e_j) e_j,
//   S3_k = sum_i w_i rho_kbar(x+e_i) e_i
//   F_k = -G1 psi_k S1_k - G2 psi_k S2_k - G_AB rho_k S3_k + rho_k g
//   m_k = sum_i f_k,i e_i + F_k / 2,  u = sum_k om_k m_k / sum_k om_k rho_k
//   f*_k,i = f_k,i - om_k (f_k,i - feq_i(rho_k, u)) + (1 - om_k/2) w_i [3(e_i - u) + 9 (e_i.u) e_i].F_k
//   f_k,i(x + e_i, t+1) = f*_k,i(x)   (or f_k,opp(i)(x, t+1) at a wall)
// Reverse of it, given lam = dJ/df(t+1):
//   lam*_k,i(x) = lam_k,i(x + e_i) (or lam_k,opp(i)(x) at a wall)      [pull]
//   phase A (local at x): the adjoints of u, F_k, m_k, the local parts of
//     the adjoints of rho_k and psi_k, the stencil sources
//     S1bar = -G1 psi F_bar, S2bar = -G2 psi F_bar, S3bar = -G_AB rho F_bar,
//     and the parameter-gradient contributions (block partials, FP64)
//   phase B (gather at y): psi_bar(y) += sum over the nodes x whose stencils
//     read y of w e . S1bar(x) + p e . S2bar(x); rho_bar(y) += exp(-rho) psi_bar
//     + w e . S3bar_kbar(x); lam_k,i(y, t) = (1 - om_k) lam*_k,i + m_bar_k . e_i + rho_bar_k.
// Ghost rows beyond a wall: a mirrored ghost passes its adjoint to the fluid
// node it copies; a fixed ghost is a constant and receives none.
#include <cuda_runtime.h>

#include "lb_kernels.cuh"
#include "lb_launch.h"

namespace lbk {

namespace {

// slots of the per-node buffer between the two phases
enum AdjSlot {
    aPsiA = 0, aPsiB, aRhoA, aRhoB,             // local psi_bar, rho_bar
    aMAx, aMAy, aMBx, aMBy,                      // m_bar
    aS1Ax, aS1Ay, aS1Bx, aS1By,                  // S1bar
    aS2Ax, aS2Ay, aS2Bx, aS2By,                  // S2bar
    aS3Ax, aS3Ay, aS3Bx, aS3By,                  // S3bar
    kAdjSlots
};
// parameter-gradient accumulators per tile
enum AdjGrad { gGAB = 0, gG1, gG2, gOmA, gOmB, kAdjGrads };

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// lam*(x, i): the adjoint of the population pushed from x in direction i
__device__ __forceinline__ double pull_lam(const Lat<double> &L, const double *__restrict__ lam, int k, int i, int x,
                                           int y)
{
    int xd = wrapi(x + ex9(i), L.nx), yd = y + ey9(i);
    int dir = i;
    if (yd < 0 || yd >= L.ny) {
        if (L.walls) {
            dir = opp9(i);
            xd = x;
            yd = y;
        } else {
            yd = wrapi(yd, L.ny);
        }
    }
    return lam[(size_t)(k * 9 + dir) * L.plane + (size_t)yd * L.pitch + xd];
}

}  // namespace

// Phase A.  seed_kind: 0 = adjoint of a time step (lam_next given); 1 = seed
// of mu_r at this state (d J / d Q in seed_a, per-node m_bar from ubar); 2 =
// seed of the Laplace pressure jump (c_in = seed_a for r < R/2, c_out = seed_b
// for r > R + 6, probe in L.probe).
__global__ void __launch_bounds__(kThreads) k_adj_local(const Lat<double> L, const double *__restrict__ f,
                                                        const double *__restrict__ rho, const double *__restrict__ lam_next,
                                                        double *__restrict__ abuf, double *__restrict__ gpart, int seed_kind,
                                                        double seed_a, double seed_b)
{
    __shared__ double srho[2][SH][SW];
    __shared__ double spsi[2][SH][SW];
    __shared__ double sred[kThreads / 32][8];
    const int tiles_x = (L.nx + TX - 1) / TX;
    const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    stage_tile<double, SH>(L, rho, x0, y0, srho, spsi, tid, kThreads);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    double gr[kAdjGrads] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (x < L.nx && y < L.ny) {
        const int cx = threadIdx.x + HALO, cy = threadIdx.y + HALO;
        const size_t c = (size_t)y * L.pitch + x;
        double r[2], ps[2], S1[2][2], S2[2][2], S3[2][2], F[2][2], m[2][2], fk[2][9];
        for (int k = 0; k < 2; ++k) {
            for (int i = 0; i < 9; ++i) fk[k][i] = f[(size_t)(k * 9 + i) * L.plane + c];
            q9_sum<double>(spsi[k], cx, cy, S1[k][0], S1[k][1]);
            q25_sum<double>(spsi[k], cx, cy, S2[k][0], S2[k][1]);
            q9_sum<double>(srho[1 - k], cx, cy, S3[k][0], S3[k][1]);
            r[k] = srho[k][cy][cx];
            ps[k] = spsi[k][cy][cx];
            for (int a = 0; a < 2; ++a)
                F[k][a] = -L.G1 * ps[k] * S1[k][a] - L.G2 * ps[k] * S2[k][a] - L.GAB * r[k] * S3[k][a] + r[k] * L.g[a];
            double jx, jy;
            first_moment<double>(fk[k], jx, jy);
            m[k][0] = jx + 0.5 * F[k][0];
            m[k][1] = jy + 0.5 * F[k][1];
        }
        const double om[2] = {L.omega[0], L.omega[1]};
        const double D = om[0] * r[0] + om[1] * r[1];
        const double u[2] = {(om[0] * m[0][0] + om[1] * m[1][0]) / D, (om[0] * m[0][1] + om[1] * m[1][1]) / D};
        const double uu = u[0] * u[0] + u[1] * u[1];

        double ub[2] = {0.0, 0.0}, Fb[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, rb[2] = {0.0, 0.0};
        double mb[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, omb[2] = {0.0, 0.0};
        if (seed_kind == 0) {
            for (int k = 0; k < 2; ++k) {
                const double a = 1.0 - 0.5 * om[k];
                for (int i = 0; i < 9; ++i) {
                    const double ls = pull_lam(L, lam_next, k, i, x, y);
                    const double e[2] = {(double)ex9(i), (double)ey9(i)}, w = w9(i);
                    const double eu = e[0] * u[0] + e[1] * u[1], eF = e[0] * F[k][0] + e[1] * F[k][1];
                    const double poly = 1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu;
                    const double feq = w * r[k] * poly;
                    for (int d = 0; d < 2; ++d) {
                        // d feq / d u and d C / d u
                        ub[d] += ls * (om[k] * w * r[k] * (3.0 * e[d] + 9.0 * eu * e[d] - 3.0 * u[d])
                                       + a * w * (-3.0 * F[k][d] + 9.0 * eF * e[d]));
                        // d C / d F
                        Fb[k][d] += ls * a * w * (3.0 * (e[d] - u[d]) + 9.0 * eu * e[d]);
                    }
                    rb[k] += ls * om[k] * w * poly;
                    const double guo = w * (3.0 * ((e[0] - u[0]) * F[k][0] + (e[1] - u[1]) * F[k][1]) + 9.0 * eu * eF);
                    omb[k] += ls * (-(fk[k][i] - feq) - 0.5 * guo);
                }
            }
            // u = N / D
            const double Nb[2] = {ub[0] / D, ub[1] / D};
            const double Db = -(ub[0] * u[0] + ub[1] * u[1]) / D;
            for (int k = 0; k < 2; ++k) {
                mb[k][0] = om[k] * Nb[0];
                mb[k][1] = om[k] * Nb[1];
                omb[k] += Nb[0] * m[k][0] + Nb[1] * m[k][1] + Db * r[k];
                rb[k] += om[k] * Db;
            }
        } else if (seed_kind == 1) {
            // J = Q0 / Q, Q = (1/nx) sum ubar_x, ubar = (m_A + m_B) / (rho_A + rho_B)
            const double rt = r[0] + r[1], ubx = (m[0][0] + m[1][0]) / rt;
            const double s = seed_a / L.nx;
            for (int k = 0; k < 2; ++k) {
                mb[k][0] = s / rt;
                rb[k] = -s * ubx / rt;
            }
        } else {
            // J = <p_b>_in - <p_b>_out, Eq. (11)
            double dx = fabs((double)x - L.probe[0]), dy = fabs((double)y - L.probe[1]);
            if (dx > 0.5 * L.nx) dx = L.nx - dx;
            if (!L.walls && dy > 0.5 * L.ny) dy = L.ny - dy;
            const double rr = sqrt(dx * dx + dy * dy), R = L.probe[2];
            const double cw = (rr < 0.5 * R ? seed_a : 0.0) + (rr > R + 6.0 ? seed_b : 0.0);
            if (cw != 0.0) {
                const double Gs = L.G1 + L.G2;
                for (int k = 0; k < 2; ++k)
                    rb[k] = cw * ((1.0 + Gs * ps[k] * exp(-r[k])) / 3.0 + L.GAB * r[1 - k] / 3.0);
                gr[gG1] += cw * 0.5 * (ps[0] * ps[0] + ps[1] * ps[1]) / 3.0;
                gr[gG2] += cw * 0.5 * (ps[0] * ps[0] + ps[1] * ps[1]) / 3.0;
                gr[gGAB] += cw * r[0] * r[1] / 3.0;
            }
        }
        // m = j + F/2
        for (int k = 0; k < 2; ++k) {
            Fb[k][0] += 0.5 * mb[k][0];
            Fb[k][1] += 0.5 * mb[k][1];
        }
        // F = -G1 psi S1 - G2 psi S2 - G_AB rho S3 + rho g
        double psb[2], S1b[2][2], S2b[2][2], S3b[2][2];
        for (int k = 0; k < 2; ++k) {
            psb[k] = -(Fb[k][0] * (L.G1 * S1[k][0] + L.G2 * S2[k][0]) + Fb[k][1] * (L.G1 * S1[k][1] + L.G2 * S2[k][1]));
            rb[k] += Fb[k][0] * (L.g[0] - L.GAB * S3[k][0]) + Fb[k][1] * (L.g[1] - L.GAB * S3[k][1]);
            for (int d = 0; d < 2; ++d) {
                S1b[k][d] = -L.G1 * ps[k] * Fb[k][d];
                S2b[k][d] = -L.G2 * ps[k] * Fb[k][d];
                S3b[k][d] = -L.GAB * r[k] * Fb[k][d];
            }
            gr[gG1] += -ps[k] * (Fb[k][0] * S1[k][0] + Fb[k][1] * S1[k][1]);
            gr[gG2] += -ps[k] * (Fb[k][0] * S2[k][0] + Fb[k][1] * S2[k][1]);
            gr[gGAB] += -r[k] * (Fb[k][0] * S3[k][0] + Fb[k][1] * S3[k][1]);
        }
        gr[gOmA] += omb[0];
        gr[gOmB] += omb[1];
        const double vals[kAdjSlots] = {psb[0], psb[1], rb[0], rb[1], mb[0][0], mb[0][1], mb[1][0], mb[1][1],
                                        S1b[0][0], S1b[0][1], S1b[1][0], S1b[1][1], S2b[0][0], S2b[0][1],
                                        S2b[1][0], S2b[1][1], S3b[0][0], S3b[0][1], S3b[1][0], S3b[1][1]};
        for (int s = 0; s < kAdjSlots; ++s) abuf[(size_t)s * L.plane + c] = vals[s];
    }
    // per-tile gradient partials, added to the tile's running sums (one block
    // per tile per step: a fixed order)
    for (int a = 0; a < kAdjGrads; ++a) {
        const double v = warp_sum(gr[a]);
        if ((tid & 31) == 0) sred[tid >> 5][a] = v;
    }
    __syncthreads();
    if (tid < kAdjGrads) {
        double v = sred[0][tid];
        for (int w = 1; w < kThreads / 32; ++w) v += sred[w][tid];
        gpart[(size_t)blockIdx.x * 8 + tid] += v;
    }
}

// Rows x_y of the nodes whose stencil vector of y-component ey reads row y_y
// (mirror ghosts included): writes up to 3 rows into rows[], returns count.
__device__ __forceinline__ int source_rows(const Lat<double> &L, int yy, int ey, int rows[3])
{
    int n = 0;
    const int r1 = yy - ey;
    if (!L.walls) {
        rows[n++] = wrapi(r1 < 0 ? r1 + L.ny : r1, L.ny);   // |ey| <= 2 < ny
        return n;
    }
    if (r1 >= 0 && r1 < L.ny) rows[n++] = r1;
    if (L.wall_mode == 0) {
        const int r2 = -1 - yy - ey;                 // read ghost row r2 + ey < 0 mirrored to yy
        if (r2 >= 0 && r2 < L.ny && r2 + ey < 0) rows[n++] = r2;
        const int r3 = 2 * L.ny - 1 - yy - ey;       // ghost row >= ny mirrored to yy
        if (r3 >= 0 && r3 < L.ny && r3 + ey >= L.ny) rows[n++] = r3;
    }
    return n;
}

// Phase B: gather the stencil adjoints and form lam(t).
__global__ void __launch_bounds__(kThreads) k_adj_gather(const Lat<double> L, const double *__restrict__ rho,
                                                         const double *__restrict__ lam_next,
                                                         const double *__restrict__ abuf, double *__restrict__ lam_out,
                                                         int seed)
{
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const size_t c = (size_t)y * L.pitch + x;
    auto A = [&](int slot, int xx, int yy) { return abuf[(size_t)slot * L.plane + (size_t)yy * L.pitch + xx]; };
    double psb[2] = {A(aPsiA, x, y), A(aPsiB, x, y)};
    double rb[2] = {A(aRhoA, x, y), A(aRhoB, x, y)};
    // D2Q25 (p weights) and D2Q9 (w weights) transposed stencils
    for (int j = 0; j < 25; ++j) {
        const int dx = j % 5 - 2, dy = j / 5 - 2;
        if (dx == 0 && dy == 0) continue;
        const double p = p25(dx * dx + dy * dy);
        const bool q9 = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1;
        const double w = q9 ? w9(dx == 0 ? (dy > 0 ? 2 : 4) : (dy == 0 ? (dx > 0 ? 1 : 3) : 5)) : 0.0;
        const int xs = wrapi(x - dx, L.nx);
        int rows[3];
        const int nr = source_rows(L, y, dy, rows);
        for (int q = 0; q < nr; ++q) {
            const int ys = rows[q];
            for (int k = 0; k < 2; ++k) {
                psb[k] += p * (dx * A(k == 0 ? aS2Ax : aS2Bx, xs, ys) + dy * A(k == 0 ? aS2Ay : aS2By, xs, ys));
                if (q9) {
                    psb[k] += w * (dx * A(k == 0 ? aS1Ax : aS1Bx, xs, ys) + dy * A(k == 0 ? aS1Ay : aS1By, xs, ys));
                    // S3 of the other species reads this species' density
                    rb[k] += w * (dx * A(k == 0 ? aS3Bx : aS3Ax, xs, ys) + dy * A(k == 0 ? aS3By : aS3Ay, xs, ys));
                }
            }
        }
    }
    for (int k = 0; k < 2; ++k) rb[k] += exp(-rho[(size_t)k * L.plane + c]) * psb[k];
    const double mb[2][2] = {{A(aMAx, x, y), A(aMAy, x, y)}, {A(aMBx, x, y), A(aMBy, x, y)}};
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < 9; ++i) {
            const double ls = seed ? 0.0 : pull_lam(L, lam_next, k, i, x, y);
            lam_out[(size_t)(k * 9 + i) * L.plane + c] =
                (1.0 - L.omega[k]) * ls + mb[k][0] * ex9(i) + mb[k][1] * ey9(i) + rb[k];
        }
}

// rho_k = sum_i f_k,i for the adjoint's recomputed states
__global__ void k_adj_density(const Lat<double> L, const double *__restrict__ f, double *__restrict__ rho)
{
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const size_t c = (size_t)y * L.pitch + x;
    for (int k = 0; k < 2; ++k) {
        double v[9];
        for (int i = 0; i < 9; ++i) v[i] = f[(size_t)(k * 9 + i) * L.plane + c];
        rho[(size_t)k * L.plane + c] = zeroth_moment<double>(v);
    }
}

// Fixed-order reduction of the per-tile gradient sums.
__global__ void k_adj_reduce(const double *__restrict__ gpart, int n_tiles, double *__restrict__ out)
{
    __shared__ double s[256];
    for (int a = 0; a < kAdjGrads; ++a) {
        double v = 0.0;
        for (int t = threadIdx.x; t < n_tiles; t += 256) v += gpart[(size_t)t * 8 + a];
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[a] = s[0];
        __syncthreads();
    }
}

cudaError_t adj_density(const Lat<double> &L, const double *f, double *rho, cudaStream_t s)
{
    k_adj_density<<<dim3((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY), dim3(TX, TY), 0, s>>>(L, f, rho);
    return cudaGetLastError();
}

cudaError_t adj_step(const Lat<double> &L, const double *f, const double *rho, const double *lam_next, double *abuf,
                     double *gpart, double *lam_out, int seed_kind, double seed_a, double seed_b, cudaStream_t s)
{
    const int tiles = ((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY);
    k_adj_local<<<tiles, dim3(TX, TY), 0, s>>>(L, f, rho, lam_next, abuf, gpart, seed_kind, seed_a, seed_b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adj_gather<<<dim3((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY), dim3(TX, TY), 0, s>>>(L, rho, lam_next, abuf,
                                                                                          lam_out, seed_kind != 0);
    return cudaGetLastError();
}

cudaError_t adj_reduce(const double *gpart, int n_tiles, double *out, cudaStream_t s)
{
    k_adj_reduce<<<1, 256, 0, s>>>(gpart, n_tiles, out);
    return cudaGetLastError();
}

}  // namespace lbk

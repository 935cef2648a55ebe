// lb_types.h -- device-visible descriptors shared by the host engine and the
// kernels of the two-range pseudopotential lattice Boltzmann library.
//
// Memory layout in HBM (one lattice):
//   populations  f[species][dir][y][pitch]   two ping-pong copies
//   densities    rho[species][y][pitch]       two copies: the density pass of
//                                              a step with parity p writes copy
//                                              p^1, the fused kernel reads it
// pitch = nx rounded up to 32 elements, so every row starts on a 128-byte
// (FP32) or 256-byte (FP64) boundary and a warp's row segment is one or two
// full cache lines.  A batch of lattices shares one allocation; each lattice
// starts on a 256-byte boundary.
#pragma once

#include <stddef.h>
#include <stdint.h>
#include <cstdint>

namespace lbk {

// Accumulator slots of the observable reduction, per tile and per lattice.
enum Acc {
    kMassA = 0, kMassB, kMomAx, kMomAy, kMomBx, kMomBy, kSumUx, kUmax, kNonFinite,
    kPIn, kPOut, kAIn, kAOut, kNIn, kNOut, kNumAcc
};
constexpr int kAccStride = 16;

// Slots of the final per-lattice observable record written by the finalize
// kernel (all FP64).
enum Obs {
    oMassA = 0, oMassB, oMomAx, oMomAy, oMomBx, oMomBy, oQ, oMuR, oDp, oReff, oUmax, oFinite, kNumObs
};
constexpr int kObsStride = 16;

template <typename real>
struct Lat {
    real *f[2];          // ping-pong population buffers
    real *rho[2];        // density of the previous step (FP32 reference) / of this step
    size_t plane;        // elements per [y][pitch] plane = ny * pitch
    int32_t nx, ny, pitch;
    int32_t walls;       // 0 periodic, 1 bounce-back walls in y
    int32_t wall_mode;   // 0 mirror, 1 fixed ghost densities
    int32_t tile_begin, tile_end;
    int32_t has_probe;
    int32_t forcing;     // 0 Guo forcing (Eqs. 5, 6), 1 velocity shift (Eq. 4; FP64 only)
    // model parameters in the compute precision
    real omega[2];       // 1 / tau_k
    real tau[2];         // tau_k (the velocity shift tau_k F_k / rho_k of Eq. 4)
    real aw[2][3];       // (1 - omega_k / 2) * w(|e|^2) for |e|^2 = 0, 1, 2
    real aw3[2][3];      // 3 aw, rounded in the compute precision (the FP32 Guo term)
    real cw[3];          // FP32: -(G1 w + G2 p) for |e|^2 = 1, 2 and -G2 (Eq. 8; vq25c)
    real G1, G2, GAB;
    real g[2];
    real wall_rho[2];
    // observable settings, always FP64
    double probe[3];     // cx, cy, R
    double tau_B;        // for the closed-form flux Q0
    double g_x;
};

}  // namespace lbk

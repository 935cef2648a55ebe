// lb_launch.h -- host-side launchers of the lattice Boltzmann kernels, one
// explicit instantiation per population format (lb_fp64.cu, lb_fp32.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lb_types.h"

struct lb_params;

namespace lbk {

template <typename real>
struct Launch {
    // one kernel launch over tiles [tile_offset, tile_offset + n_tiles) of
    // height ty (2, 4 or 8)
    static cudaError_t density(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                               int ty, cudaStream_t s);
    static cudaError_t collide(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                               int ty, cudaStream_t s);
    // one time step in one pass (densities formed in the kernel)
    static cudaError_t fused(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                             int ty, cudaStream_t s);
    // nsteps time steps of all tiles in one persistent launch of `blocks`
    // blocks (ctl, dens_done, coll_done cleared by the caller beforehand)
    static cudaError_t persistent(const Lat<real> *lats, const int4 *tiles, const int *lat_ntiles, int n_tiles,
                                  int nsteps, int parity0,
                                  void *ctl, unsigned *dens_done, unsigned *coll_done, int *err, long long wait_cycles,
                                  int drop_tile, int ty, int blocks, cudaStream_t s);
    // resident blocks per SM of the persistent kernel for tile height ty
    static int persistent_blocks_per_sm(int ty);
    static cudaError_t observe(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                               double *partials, double *rho, double *mom, double *ubar, cudaStream_t s);
    static cudaError_t finalize(const Lat<real> *lats, int n_lat, const double *partials, double *obs, cudaStream_t s);
    // pressure tensor per node of tiles [tile_offset, tile_offset + n_tiles)
    // of height 4 (partials: 8 doubles per tile; out: dense [6][ny][nx] of
    // one lattice, or NULL), and its per-lattice sums (8 doubles per lattice)
    static cudaError_t pressure(const Lat<real> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                                double *partials, double *out, cudaStream_t s);
    static cudaError_t pressure_sum(const Lat<real> *lats, int n_lat, const double *partials, double *out, cudaStream_t s);
    // one lattice, dense FP64 host-layout buffers in device memory
    static cudaError_t init(const Lat<real> *lats, int lat, int nx, int ny, const double *rho, const double *u,
                            int parity, cudaStream_t s);
    static cudaError_t get_pops(const Lat<real> *lats, int lat, int nx, int ny, int parity, double *out, cudaStream_t s);
    static cudaError_t set_pops(const Lat<real> *lats, int lat, int nx, int ny, int parity, const double *in,
                                cudaStream_t s);
};

extern template struct Launch<double>;
extern template struct Launch<float>;

// Tensor maps of one FP32 lattice for the TMA-staged one-pass step
// (lb_tma.cu): for each tile height (2, 4, 8) and population copy, the 18
// population planes and the 2 reference-density planes as 3-D tensors
// (x, y, plane), with a box of the tile plus 4 columns on each side and 2 rows
// above and below.  Zero-filled where unused (lattices narrower than the box).
struct TmaMaps {
    CUtensorMap pop[3][2];
    CUtensorMap ref[3][2];
};
constexpr int kTmaBoxW = 40;             // 32 + 2 x 4 columns: x offsets stay 16-byte aligned
// The tile (x0, y0) of height ty of an nx x ny lattice is staged by TMA.
__host__ __device__ inline bool tma_box_tile(int nx, int ny, int x0, int y0, int ty)
{
    return x0 + 32 <= nx && y0 + ty <= ny && nx >= kTmaBoxW && ny >= ty + 4;
}
// Fourth field (w) of a tile record that tma_box_tile accepted, set where
// the host sorts a list into box tiles and the rest (the others keep 0), so
// that the TMA kernel checks its tile without loading its lattice first.
constexpr int kTmaBoxMark = 1;
// Shared-memory opt-in of the TMA kernels on the current device; call once
// before the first launch_fused_tma, outside stream capture.
cudaError_t prepare_fused_tma();
// One time step of the FP32 tiles [tile_offset, tile_offset + n_tiles) in
// one pass, one block per tile, each tile staged by one TMA copy of its
// population box and one of its reference-density box.  Every tile must be
// full and of a lattice at least kTmaBoxW x (ty + 4) nodes (tma_box_tile)
// and carry w = kTmaBoxMark; the others go to Launch<float>::fused.  A copy
// not complete after wait_cycles SM clocks sets *err = 1 and ends the block,
// a tile without the mark sets *err = 2 (and starts no copy); the copy of
// tile drop_tile (a test hook, -1 for none) is never started.
cudaError_t launch_fused_tma(const Lat<float> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                             const TmaMaps *maps, int *err, long long wait_cycles, int drop_tile, int ty, cudaStream_t s);

// Discrete adjoint of the FP64 step (lb_adjoint.cu).  Buffers use the
// lattice's pitched layout; abuf holds 20 planes, gpart 8 doubles per tile of
// 32 x 4 nodes.  seed_kind: 0 adjoint step (lam_next = dJ/df(t+1)), 1 seed of
// mu_r (seed_a = dJ/dQ), 2 seed of the Laplace pressure jump (seed_a = 1/n_in,
// seed_b = -1/n_out, probe in L).
cudaError_t adj_density(const Lat<double> &L, const double *f, double *rho, cudaStream_t s);
cudaError_t adj_step(const Lat<double> &L, const double *f, const double *rho, const double *lam_next, double *abuf,
                     double *gpart, double *lam_out, int seed_kind, double seed_a, double seed_b, cudaStream_t s);
cudaError_t adj_reduce(const double *gpart, int n_tiles, double *out, cudaStream_t s);
// FP64 populations f_i = h_i + w_i R of an FP32 state (18 offset planes h,
// 2 reference-density planes R), pitched like the lattice (lb_fp32.cu).
cudaError_t offset_to_f64(const Lat<float> &L, const float *h, const float *R, double *out, cudaStream_t s);
constexpr int kAdjSlotCount = 20;

// Record msg as the calling thread's lb_last_error() message.
void set_last_error(const char *msg);
// The parameter check of lb_create for lattice `index` of a batch: LB_OK,
// or LB_EINVAL with the message recorded (lb_api.cu).
int validate_params(const ::lb_params *p, int index);

}  // namespace lbk

// lb_api.cu -- C-ABI of the lattice Boltzmann library (declared in lb.h):
// parameter validation, device memory, tile lists, stream ordering, CUDA-graph
// replay of the time loop, and host<->device transfers.  All arithmetic of the
// method runs in the kernels of lb_kernels.cuh.
//
// Host code of this file is compiled with -ffp-contract=off so the derived
// FP64 parameters (1/tau, (1 - 1/(2 tau)) w) round exactly as written.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <limits>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "lb.h"
#include "lb_kernels.cuh"
#include "lb_launch.h"
#include "lb_types.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(LB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LB_CUDA(call)                                    \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr int kGraphSteps = 32;   // steps per captured graph (even: parity returns)
constexpr int kPersistSteps = 64; // time steps per persistent launch
constexpr int kChains = 2;         // chains of time steps of a batch's step graph
constexpr int kTileHeights[3] = {2, 4, 8};

int ty_index(int ty) { return ty == 2 ? 0 : (ty == 4 ? 1 : (ty == 8 ? 2 : -1)); }
constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool is_fin(double v) { return std::isfinite(v); }

int validate(const lb_params *p, int i)
{
    char buf[160];
    if (!p) return fail(LB_EINVAL, "params is NULL");
    if (p->nx < 5 || p->ny < 5) {
        snprintf(buf, sizeof buf, "lattice %d: nx=%d ny=%d, both must be >= 5", i, p->nx, p->ny);
        return fail(LB_EINVAL, buf);
    }
    if ((long long)p->nx * p->ny > (1ll << 31)) return fail(LB_EINVAL, "lattice too large (nx*ny > 2^31)");
    for (int k = 0; k < 2; ++k)
        if (!is_fin(p->tau[k]) || !(p->tau[k] > 0.5)) {
            snprintf(buf, sizeof buf, "lattice %d: tau[%d]=%g must be finite and > 1/2", i, k, p->tau[k]);
            return fail(LB_EINVAL, buf);
        }
    const double vals[] = {p->G_AB, p->G1, p->G2, p->g[0], p->g[1], p->wall_rho[0], p->wall_rho[1]};
    for (double v : vals)
        if (!is_fin(v)) return fail(LB_EINVAL, "non-finite coupling, force or wall density");
    if (p->walls != LB_PERIODIC && p->walls != LB_WALLS_Y) return fail(LB_EINVAL, "walls must be 0 or 1");
    if (p->wall_mode != LB_WALL_MIRROR && p->wall_mode != LB_WALL_FIXED) return fail(LB_EINVAL, "wall_mode must be 0 or 1");
    if (p->precision != LB_FP64 && p->precision != LB_FP32) return fail(LB_EINVAL, "precision must be LB_FP64 or LB_FP32");
    if (p->forcing != LB_FORCING_GUO && p->forcing != LB_FORCING_SHIFT)
        return fail(LB_EINVAL, "forcing must be LB_FORCING_GUO or LB_FORCING_SHIFT");
    if (p->forcing == LB_FORCING_SHIFT && p->precision != LB_FP64)
        return fail(LB_EINVAL, "forcing LB_FORCING_SHIFT is built for LB_FP64 populations only");
    return LB_OK;
}

template <typename real>
void fill_lat(lbk::Lat<real> &L, const lb_params &p)
{
    std::memset(&L, 0, sizeof L);
    L.nx = p.nx;
    L.ny = p.ny;
    L.pitch = (int)align_up((size_t)p.nx, 32);
    L.plane = (size_t)L.pitch * p.ny;
    L.walls = p.walls;
    L.wall_mode = p.wall_mode;
    L.forcing = p.forcing;
    const double wcls[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
    for (int k = 0; k < 2; ++k) {
        const double omega = 1.0 / p.tau[k];
        L.omega[k] = (real)omega;
        L.tau[k] = (real)p.tau[k];
        for (int c = 0; c < 3; ++c) L.aw[k][c] = (real)((1.0 - 0.5 * omega) * wcls[c]);
        for (int c = 0; c < 3; ++c) L.aw3[k][c] = (real)3 * L.aw[k][c];
        L.g[k] = (real)p.g[k];
        L.wall_rho[k] = (real)p.wall_rho[k];
    }
    L.G1 = (real)p.G1;
    L.G2 = (real)p.G2;
    L.GAB = (real)p.G_AB;
    // the combined psi-sum weights of Eq. (8) on the inner ring,
    // c(|e|^2) = G1 w(|e|^2) + G2 p(|e|^2) for |e|^2 = 1, 2, and G2 for the
    // outer ring, negated
    L.cw[0] = (real)(-(p.G1 / 9.0 + p.G2 * (4.0 / 63.0)));
    L.cw[1] = (real)(-(p.G1 / 36.0 + p.G2 * (4.0 / 135.0)));
    L.cw[2] = (real)(-p.G2);
    L.tau_B = p.tau[1];
    L.g_x = p.g[0];
}

// cuTensorMapEncodeTiled from the driver, looked up once (no link against
// the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

struct lb_engine {
    int precision = LB_FP64;
    int n = 0;
    int device = 0;
    cudaStream_t stream = nullptr;   // the caller's stream, or one the engine owns
    bool own_stream = false;
    std::vector<lb_params> P;
    std::vector<lbk::Lat<double>> L64;
    std::vector<lbk::Lat<float>> L32;
    std::vector<int4> tiles;          // 32 x 4 tiles of the observation kernels
    void *d_lats = nullptr;
    int4 *d_tiles = nullptr;
    // time-step tiles for each tile height (2, 4, 8) and per-lattice counts
    std::vector<int4> stiles[3];
    int4 *d_stiles[3] = {nullptr, nullptr, nullptr};
    int *d_sntiles[3] = {nullptr, nullptr, nullptr};
    // execution configuration (autotuned or set by the caller)
    int mode = LB_MODE_LAUNCH;
    int ty = 4;
    // persistent launches: control block (queue head + per-lattice counters),
    // sticky error word, blocks per SM per tile height, bounded-wait limit
    void *d_ctl = nullptr;
    int *d_err = nullptr;
    int sm_count = 0;
    int persist_bps[3] = {0, 0, 0};
    long long wait_cycles = 0;
    int drop_tile = -1;
    void *d_pool = nullptr;
    size_t pool_bytes = 0;
    // LB_MODE_TMA: one set of tensor maps per lattice (FP32 only), and per
    // tile height the time-step tiles reordered: the n_box tiles staged by TMA
    // first, then the others
    lbk::TmaMaps *d_tmaps = nullptr;
    int4 *d_btiles[3] = {nullptr, nullptr, nullptr};
    int n_box[3] = {0, 0, 0};
    bool tma_ok = false;
    std::string tma_why = "LB_MODE_TMA needs LB_FP32 populations";
    double *d_partials = nullptr;
    double *d_obs = nullptr;
    double *d_psum = nullptr;         // pressure-tensor sums, kPStride doubles per lattice
    double *d_tmp = nullptr;
    size_t tmp_elems = 0;
    int64_t t = 0;
    int parity = 0;
    cudaGraphExec_t gexec = nullptr;
    // Chains of time steps for a batch: the lattices split into kChains
    // groups of about equal node counts, each group's steps launched on its
    // own stream (the engine's for group 0, an auxiliary one for each other)
    // and captured as independent branches of the step graph, so that the
    // launches of one group fill the last waves of the others'.  Per tile
    // height, the tiles of group 0 (the TMA box tiles first, then the rest),
    // then those of group 1, and so on.
    int nchains = 1;
    cudaStream_t aux[kChains] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kChains] = {};
    int4 *d_ctiles[3] = {nullptr, nullptr, nullptr};
    int c_off[3][kChains] = {}, c_box[3][kChains] = {}, c_cnt[3][kChains] = {};

    ~lb_engine()
    {
        if (stream) cudaStreamSynchronize(stream);
        if (gexec) cudaGraphExecDestroy(gexec);
        cudaFree(d_lats);
        cudaFree(d_tiles);
        for (int i = 0; i < 3; ++i) {
            cudaFree(d_stiles[i]);
            cudaFree(d_sntiles[i]);
            cudaFree(d_btiles[i]);
        }
        cudaFree(d_ctl);
        cudaFree(d_err);
        cudaFree(d_pool);
        cudaFree(d_tmaps);
        cudaFree(d_partials);
        cudaFree(d_obs);
        cudaFree(d_psum);
        cudaFree(d_tmp);
        for (int i = 0; i < 3; ++i) cudaFree(d_ctiles[i]);
        for (int g = 0; g < kChains; ++g) {
            if (aux[g]) {
                cudaStreamSynchronize(aux[g]);
                cudaStreamDestroy(aux[g]);
            }
            if (ev_join[g]) cudaEventDestroy(ev_join[g]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (stream && own_stream) cudaStreamDestroy(stream);
    }

    size_t real_size() const { return precision == LB_FP64 ? 8 : 4; }
    int nx(int l) const { return P[l].nx; }
    int ny(int l) const { return P[l].ny; }
    int tile_begin(int l) const { return precision == LB_FP64 ? L64[l].tile_begin : L32[l].tile_begin; }
    int tile_end(int l) const { return precision == LB_FP64 ? L64[l].tile_end : L32[l].tile_end; }
    size_t plane(int l) const { return precision == LB_FP64 ? L64[l].plane : L32[l].plane; }
    void *fbuf(int l, int par) const
    {
        return precision == LB_FP64 ? (void *)L64[l].f[par] : (void *)L32[l].f[par];
    }
    void *rbuf(int l, int par) const
    {
        return precision == LB_FP64 ? (void *)L64[l].rho[par] : (void *)L32[l].rho[par];
    }
    // bytes of the state a checkpoint holds: populations, plus the FP32
    // reference densities
    size_t pop_bytes(int l) const { return 18 * plane(l) * real_size(); }
    size_t ref_bytes(int l) const { return precision == LB_FP32 ? 2 * plane(l) * real_size() : 0; }

    int begin()
    {
        if (cudaSetDevice(device) != cudaSuccess) return fail(LB_ECUDA, "cudaSetDevice failed");
        return LB_OK;
    }
    int end() { return LB_OK; }

    // density pass over tiles of the observation list (height 4)
    cudaError_t launch_density_obs(int par, int off, int cnt)
    {
        if (precision == LB_FP64)
            return lbk::Launch<double>::density((const lbk::Lat<double> *)d_lats, d_tiles, off, cnt, par, 4, stream);
        return lbk::Launch<float>::density((const lbk::Lat<float> *)d_lats, d_tiles, off, cnt, par, 4, stream);
    }
    // one time step over the time-step tiles of height ty: two launches, or
    // one in the fused mode
    cudaError_t launch_step(int par)
    {
        const int ti = ty_index(ty), nt = (int)stiles[ti].size();
        cudaError_t e;
        if (precision == LB_FP64) {
            const lbk::Lat<double> *L = (const lbk::Lat<double> *)d_lats;
            if (mode == LB_MODE_FUSED) return lbk::Launch<double>::fused(L, d_stiles[ti], 0, nt, par, ty, stream);
            e = lbk::Launch<double>::density(L, d_stiles[ti], 0, nt, par, ty, stream);
            if (e == cudaSuccess) e = lbk::Launch<double>::collide(L, d_stiles[ti], 0, nt, par, ty, stream);
        } else {
            const lbk::Lat<float> *L = (const lbk::Lat<float> *)d_lats;
            if (mode == LB_MODE_FUSED) return lbk::Launch<float>::fused(L, d_stiles[ti], 0, nt, par, ty, stream);
            if (mode == LB_MODE_TMA) return launch_tma(L, ti, nt, par);
            e = lbk::Launch<float>::density(L, d_stiles[ti], 0, nt, par, ty, stream);
            if (e == cudaSuccess) e = lbk::Launch<float>::collide(L, d_stiles[ti], 0, nt, par, ty, stream);
        }
        return e;
    }
    // LB_MODE_TMA step: the TMA kernel over the box tiles, the plain one-pass
    // kernel over the rest
    cudaError_t launch_tma(const lbk::Lat<float> *L, int ti, int nt, int par)
    {
        cudaError_t e = lbk::launch_fused_tma(L, d_btiles[ti], 0, n_box[ti], par, d_tmaps, d_err, wait_cycles, drop_tile,
                                              ty, stream);
        if (e == cudaSuccess && nt > n_box[ti])
            e = lbk::Launch<float>::fused(L, d_btiles[ti], n_box[ti], nt - n_box[ti], par, ty, stream);
        return e;
    }
    size_t ctl_bytes() const { return 8 + 2 * sizeof(unsigned) * (size_t)n; }
    // nsteps time steps in one persistent launch (counters cleared first)
    cudaError_t launch_persistent(int par, int nsteps)
    {
        const int ti = ty_index(ty), nt = (int)stiles[ti].size();
        cudaError_t e = cudaMemsetAsync(d_ctl, 0, ctl_bytes(), stream);
        if (e != cudaSuccess) return e;
        unsigned *dens = (unsigned *)((char *)d_ctl + 8), *coll = dens + n;
        int blocks = persist_bps[ti] * sm_count;
        if (blocks <= 0) blocks = sm_count > 0 ? sm_count : 1;
        if (precision == LB_FP64)
            return lbk::Launch<double>::persistent((const lbk::Lat<double> *)d_lats, d_stiles[ti], d_sntiles[ti], nt,
                                                   nsteps, par, d_ctl, dens, coll, d_err, wait_cycles, drop_tile, ty,
                                                   blocks, stream);
        return lbk::Launch<float>::persistent((const lbk::Lat<float> *)d_lats, d_stiles[ti], d_sntiles[ti], nt,
                                              nsteps, par, d_ctl, dens, coll, d_err, wait_cycles, drop_tile, ty,
                                              blocks, stream);
    }
    // one time step of the lattices of chain g on stream s
    cudaError_t launch_chain_step(int g, int par, cudaStream_t s)
    {
        const int ti = ty_index(ty), off = c_off[ti][g], nb = c_box[ti][g], cnt = c_cnt[ti][g];
        const int4 *T = d_ctiles[ti];
        if (cnt == 0) return cudaSuccess;
        cudaError_t e;
        if (precision == LB_FP64) {
            const lbk::Lat<double> *L = (const lbk::Lat<double> *)d_lats;
            if (mode == LB_MODE_FUSED) return lbk::Launch<double>::fused(L, T, off, cnt, par, ty, s);
            e = lbk::Launch<double>::density(L, T, off, cnt, par, ty, s);
            if (e == cudaSuccess) e = lbk::Launch<double>::collide(L, T, off, cnt, par, ty, s);
            return e;
        }
        const lbk::Lat<float> *L = (const lbk::Lat<float> *)d_lats;
        if (mode == LB_MODE_FUSED) return lbk::Launch<float>::fused(L, T, off, cnt, par, ty, s);
        if (mode == LB_MODE_TMA) {
            e = lbk::launch_fused_tma(L, T, off, nb, par, d_tmaps, d_err, wait_cycles, drop_tile, ty, s);
            if (e == cudaSuccess && cnt > nb) e = lbk::Launch<float>::fused(L, T, off + nb, cnt - nb, par, ty, s);
            return e;
        }
        e = lbk::Launch<float>::density(L, T, off, cnt, par, ty, s);
        if (e == cudaSuccess) e = lbk::Launch<float>::collide(L, T, off, cnt, par, ty, s);
        return e;
    }
    // time steps in the current mode, as captured into one graph: with
    // chains, chains 1.. fork onto their auxiliary streams and join the
    // engine's stream again at the end (also after a failed launch, so that
    // a capture always ends joined)
    cudaError_t launch_chunk(int par, int nsteps)
    {
        if (mode == LB_MODE_PERSISTENT) return launch_persistent(par, nsteps);
        cudaError_t e = cudaSuccess;
        if (nchains < 2) {
            for (int s = 0; s < nsteps && e == cudaSuccess; ++s) e = launch_step((par + s) & 1);
            return e;
        }
        e = cudaEventRecord(ev_fork, stream);
        int forked = 1;
        for (; forked < nchains && e == cudaSuccess; ++forked) e = cudaStreamWaitEvent(aux[forked], ev_fork, 0);
        if (e != cudaSuccess) --forked;
        for (int s = 0; s < nsteps && e == cudaSuccess; ++s)
            for (int g = 0; g < nchains && e == cudaSuccess; ++g)
                e = launch_chain_step(g, (par + s) & 1, g ? aux[g] : stream);
        cudaError_t j = cudaSuccess;
        for (int g = 1; g < forked; ++g) {
            cudaError_t r = cudaEventRecord(ev_join[g], aux[g]);
            if (r == cudaSuccess) r = cudaStreamWaitEvent(stream, ev_join[g], 0);
            if (j == cudaSuccess) j = r;
        }
        return e != cudaSuccess ? e : j;
    }
    int chunk_steps() const { return mode == LB_MODE_PERSISTENT ? kPersistSteps : kGraphSteps; }
    void drop_graph()
    {
        if (gexec) {
            cudaGraphExecDestroy(gexec);
            gexec = nullptr;
        }
    }
    // Tensor maps of every FP32 lattice for LB_MODE_TMA: per tile height and
    // population copy, the 18 population planes and the 2 reference-density
    // planes as (x, y, plane) tensors, box 40 x (ty + 4) x planes.  Leaves
    // tma_ok false, with the reason, where the driver cannot encode them.
    int build_tma_maps()
    {
        EncodeTiledFn enc = tensor_map_encoder();
        if (!enc) {
            tma_why = "LB_MODE_TMA: the driver offers no cuTensorMapEncodeTiled";
            return LB_OK;
        }
        std::vector<lbk::TmaMaps> maps(n);
        std::memset((void *)maps.data(), 0, maps.size() * sizeof(lbk::TmaMaps));
        for (int l = 0; l < n; ++l) {
            const lbk::Lat<float> &L = L32[l];
            const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * 4, (cuuint64_t)L.plane * 4};
            const cuuint64_t dim_p[3] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny, 18};
            const cuuint64_t dim_r[3] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny, 2};
            const cuuint32_t estr[3] = {1, 1, 1};
            for (int ti = 0; ti < 3; ++ti) {
                const cuuint32_t h = (cuuint32_t)(kTileHeights[ti] + 2 * lbk::HALO);
                if (L.nx < lbk::kTmaBoxW || L.ny < (int)h) continue;   // no tile's box fits: never used
                const cuuint32_t box_p[3] = {(cuuint32_t)lbk::kTmaBoxW, h, 18};
                const cuuint32_t box_r[3] = {(cuuint32_t)lbk::kTmaBoxW, h, 2};
                for (int par = 0; par < 2; ++par) {
                    const CUresult r1 = enc(&maps[l].pop[ti][par], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)L.f[par],
                                            dim_p, strides, box_p, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                    const CUresult r2 = enc(&maps[l].ref[ti][par], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                                            (void *)L.rho[par], dim_r, strides, box_r, estr,
                                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                    if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
                        tma_why = "LB_MODE_TMA: cuTensorMapEncodeTiled rejected a lattice's layout";
                        return LB_OK;
                    }
                }
            }
        }
        if (lbk::prepare_fused_tma() != cudaSuccess) {
            cudaGetLastError();
            tma_why = "LB_MODE_TMA: the TMA kernels cannot get their shared memory on this device";
            return LB_OK;
        }
        if (cudaMalloc((void **)&d_tmaps, maps.size() * sizeof(lbk::TmaMaps)) != cudaSuccess) {
            cudaGetLastError();
            return fail(LB_ENOMEM, "cudaMalloc of the tensor maps failed");
        }
        cudaError_t ce = cudaMemcpyAsync(d_tmaps, maps.data(), maps.size() * sizeof(lbk::TmaMaps),
                                         cudaMemcpyHostToDevice, stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        if (ce != cudaSuccess) return cuda_fail(ce, "tensor map upload");
        for (int ti = 0; ti < 3; ++ti) {
            const int tyv = kTileHeights[ti];
            std::vector<int4> box, rest;
            for (const int4 &t : stiles[ti]) {
                if (lbk::tma_box_tile(P[t.x].nx, P[t.x].ny, t.y, t.z, tyv))
                    box.push_back(make_int4(t.x, t.y, t.z, lbk::kTmaBoxMark));
                else
                    rest.push_back(t);
            }
            n_box[ti] = (int)box.size();
            box.insert(box.end(), rest.begin(), rest.end());
            if (cudaMalloc((void **)&d_btiles[ti], box.size() * sizeof(int4)) != cudaSuccess) {
                cudaGetLastError();
                return fail(LB_ENOMEM, "cudaMalloc of the TMA tile lists failed");
            }
            ce = cudaMemcpyAsync(d_btiles[ti], box.data(), box.size() * sizeof(int4), cudaMemcpyHostToDevice, stream);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
            if (ce != cudaSuccess) return cuda_fail(ce, "TMA tile list upload");
        }
        tma_ok = true;
        return LB_OK;
    }

    // a bounded device-side wait that ran out is reported once, then cleared
    int check_timeout()
    {
        int h = 0;
        LB_CUDA(cudaMemcpyAsync(&h, d_err, sizeof h, cudaMemcpyDeviceToHost, stream));
        LB_CUDA(cudaStreamSynchronize(stream));
        if (h) {
            LB_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), stream));
            LB_CUDA(cudaStreamSynchronize(stream));
            if (h == 2) return fail(LB_ECUDA, "internal: a tile of the TMA list is not a box tile; the state is invalid");
            return fail(LB_ETIMEOUT, "a bounded device-side wait expired (persistent kernel or TMA copy); the state is invalid");
        }
        return LB_OK;
    }
    cudaError_t launch_observe(int par, int off, int cnt, double *partials, double *rho, double *mom, double *ubar)
    {
        if (precision == LB_FP64)
            return lbk::Launch<double>::observe((const lbk::Lat<double> *)d_lats, d_tiles, off, cnt, par, partials,
                                                rho, mom, ubar, stream);
        return lbk::Launch<float>::observe((const lbk::Lat<float> *)d_lats, d_tiles, off, cnt, par, partials, rho,
                                           mom, ubar, stream);
    }
    cudaError_t launch_finalize()
    {
        if (precision == LB_FP64)
            return lbk::Launch<double>::finalize((const lbk::Lat<double> *)d_lats, n, d_partials, d_obs, stream);
        return lbk::Launch<float>::finalize((const lbk::Lat<float> *)d_lats, n, d_partials, d_obs, stream);
    }

    int ensure_tmp(size_t elems)
    {
        if (elems <= tmp_elems) return LB_OK;
        if (d_tmp) {
            LB_CUDA(cudaStreamSynchronize(stream));
            cudaFree(d_tmp);
            d_tmp = nullptr;
            tmp_elems = 0;
        }
        if (cudaMalloc(&d_tmp, elems * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(LB_ENOMEM, "cudaMalloc of the transfer buffer failed");
        }
        tmp_elems = elems;
        return LB_OK;
    }

    int build_graph()
    {
        cudaGraph_t g = nullptr;
        LB_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = launch_chunk(0, chunk_steps());
        cudaError_t ce = cudaStreamEndCapture(stream, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(le, "kernel launch during graph capture");
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        cudaError_t ie = cudaGraphInstantiate(&gexec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            gexec = nullptr;
            return cuda_fail(ie, "cudaGraphInstantiate");
        }
        return LB_OK;
    }

    int step(int64_t nsteps)
    {
        if (nsteps < 0) return fail(LB_EINVAL, "negative step count");
        int rc = begin();
        if (rc) return rc;
        const int chunk = chunk_steps();
        while (nsteps > 0) {
            if (parity == 0 && nsteps >= chunk) {
                if (!gexec && (rc = build_graph())) return rc;
                LB_CUDA(cudaGraphLaunch(gexec, stream));
                nsteps -= chunk;
                t += chunk;
            } else {
                const int k = mode == LB_MODE_PERSISTENT ? (int)std::min<int64_t>(nsteps, parity ? 1 : chunk) : 1;
                LB_CUDA(launch_chunk(parity, k));
                parity ^= (k & 1);
                nsteps -= k;
                t += k;
            }
        }
        return end();
    }

    int set_config(int m, int tyv)
    {
        if (m != LB_MODE_LAUNCH && m != LB_MODE_PERSISTENT && m != LB_MODE_FUSED && m != LB_MODE_TMA)
            return fail(LB_EINVAL, "mode must be LB_MODE_LAUNCH, LB_MODE_PERSISTENT, LB_MODE_FUSED or LB_MODE_TMA");
        if (m == LB_MODE_TMA && !tma_ok) return fail(LB_EINVAL, tma_why.c_str());
        if (ty_index(tyv) < 0) return fail(LB_EINVAL, "tile height must be 2, 4 or 8");
        if (m != mode || tyv != ty) drop_graph();
        mode = m;
        ty = tyv;
        return LB_OK;
    }

    int profile(int32_t nsteps, void *flush, size_t flush_bytes, double ms[3])
    {
        if (nsteps < 1 || !ms) return fail(LB_EINVAL, "profile needs nsteps >= 1 and ms");
        if (flush_bytes > 0 && !flush) return fail(LB_EINVAL, "flush_bytes > 0 with a NULL flush buffer");
        int rc = begin();
        if (rc) return rc;
        std::vector<cudaEvent_t> ev(3 * (size_t)nsteps, nullptr);
        auto cleanup = [&]() {
            for (auto &x : ev)
                if (x) cudaEventDestroy(x);
        };
        for (auto &x : ev)
            if (cudaEventCreate(&x) != cudaSuccess) {
                cleanup();
                return fail(LB_ECUDA, "cudaEventCreate failed");
            }
        const int ti = ty_index(ty), nt = (int)stiles[ti].size();
        cudaError_t ce = cudaSuccess;
        for (int s = 0; s < nsteps && ce == cudaSuccess; ++s) {
            if (flush_bytes) ce = cudaMemsetAsync(flush, s & 0xff, flush_bytes, stream);
            if (ce == cudaSuccess) ce = cudaEventRecord(ev[3 * s], stream);
            const bool one = mode == LB_MODE_FUSED || mode == LB_MODE_TMA;
            if (precision == LB_FP64) {
                const lbk::Lat<double> *L = (const lbk::Lat<double> *)d_lats;
                if (ce == cudaSuccess && !one) ce = lbk::Launch<double>::density(L, d_stiles[ti], 0, nt, parity, ty, stream);
                if (ce == cudaSuccess) ce = cudaEventRecord(ev[3 * s + 1], stream);
                if (ce == cudaSuccess)
                    ce = one ? lbk::Launch<double>::fused(L, d_stiles[ti], 0, nt, parity, ty, stream)
                             : lbk::Launch<double>::collide(L, d_stiles[ti], 0, nt, parity, ty, stream);
            } else {
                const lbk::Lat<float> *L = (const lbk::Lat<float> *)d_lats;
                if (ce == cudaSuccess && !one) ce = lbk::Launch<float>::density(L, d_stiles[ti], 0, nt, parity, ty, stream);
                if (ce == cudaSuccess) ce = cudaEventRecord(ev[3 * s + 1], stream);
                if (ce == cudaSuccess)
                    ce = mode == LB_MODE_TMA ? launch_tma(L, ti, nt, parity)
                         : one ? lbk::Launch<float>::fused(L, d_stiles[ti], 0, nt, parity, ty, stream)
                               : lbk::Launch<float>::collide(L, d_stiles[ti], 0, nt, parity, ty, stream);
            }
            if (ce == cudaSuccess) ce = cudaEventRecord(ev[3 * s + 2], stream);
            if (ce == cudaSuccess) {
                parity ^= 1;
                t += 1;
            }
        }
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int s = 0; s < nsteps && ce == cudaSuccess; ++s) {
            float a = 0.f, b = 0.f, c = 0.f;
            ce = cudaEventElapsedTime(&a, ev[3 * s], ev[3 * s + 1]);
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&b, ev[3 * s + 1], ev[3 * s + 2]);
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&c, ev[3 * s], ev[3 * s + 2]);
            acc[0] += a;
            acc[1] += b;
            acc[2] += c;
        }
        cleanup();
        if (ce != cudaSuccess) return cuda_fail(ce, "profiled time steps");
        for (int k = 0; k < 3; ++k) ms[k] = acc[k] / nsteps;
        return end();
    }

    // key of the autotuning cache: device, precision and lattice shapes
    std::string tune_key() const
    {
        cudaDeviceProp prop;
        std::string dev = "unknown";
        if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) dev = prop.name;
        for (char &c : dev)
            if (c == ' ' || c == '\t') c = '_';
        unsigned long long h = 1469598103934665603ull;   // FNV-1a over the shapes
        auto mix = [&](long long v) {
            for (int b = 0; b < 8; ++b) {
                h ^= (unsigned long long)((v >> (8 * b)) & 0xff);
                h *= 1099511628211ull;
            }
        };
        for (const lb_params &p : P) {
            mix(p.nx);
            mix(p.ny);
            mix(p.walls);
        }
        std::ostringstream os;
        os << dev << "|" << (precision == LB_FP64 ? "fp64" : "fp32") << "|n" << n << "|" << std::hex << h;
        return os.str();
    }

    // Time every (mode, tile height) on trial_steps steps of the current state
    // (restored after each trial) and keep the fastest; results are cached in
    // cache_path (one "key mode ty ms" line per configuration) when given.
    int autotune(int trial_steps, const char *cache_path, double *best_ms)
    {
        if (trial_steps < 1) return fail(LB_EINVAL, "trial_steps must be >= 1");
        const std::string key = tune_key();
        std::vector<std::string> lines;
        if (cache_path) {
            std::ifstream in(cache_path);
            std::string ln;
            while (std::getline(in, ln)) {
                std::istringstream is(ln);
                std::string k;
                int m = -1, tyv = -1;
                double ms = 0.0;
                if (!(is >> k >> m >> tyv >> ms)) continue;
                if (k == key && set_config(m, tyv) == LB_OK) {
                    if (best_ms) *best_ms = ms;
                    return LB_OK;
                }
                lines.push_back(ln);
            }
        }
        int rc = begin();
        if (rc) return rc;
        void *snap = nullptr;
        if (cudaMalloc(&snap, pool_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(LB_ENOMEM, "autotune: no room for a snapshot of the state");
        }
        const int64_t t0 = t;
        const int par0 = parity;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        double best = std::numeric_limits<double>::infinity();
        int bm = mode, bty = ty;
        cudaError_t ce = cudaMemcpyAsync(snap, d_pool, pool_bytes, cudaMemcpyDeviceToDevice, stream);
        const int last_mode = tma_ok ? LB_MODE_TMA : LB_MODE_FUSED;
        for (int m = LB_MODE_LAUNCH; m <= last_mode && ce == cudaSuccess && rc == LB_OK; ++m)
            for (int tyv : kTileHeights) {
                if ((rc = set_config(m, tyv))) break;
                if ((rc = step(chunk_steps()))) break;            // warm-up, builds the graph
                ce = cudaEventRecord(e0, stream);
                if (ce == cudaSuccess && (rc = step(trial_steps))) break;
                if (ce == cudaSuccess) ce = cudaEventRecord(e1, stream);
                if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
                if (ce != cudaSuccess) break;
                if ((rc = check_timeout())) break;
                const double per = (double)ms / trial_steps;
                if (per < best) {
                    best = per;
                    bm = m;
                    bty = tyv;
                }
                ce = cudaMemcpyAsync(d_pool, snap, pool_bytes, cudaMemcpyDeviceToDevice, stream);
                t = t0;
                parity = par0;
            }
        cudaStreamSynchronize(stream);
        cudaMemcpy(d_pool, snap, pool_bytes, cudaMemcpyDeviceToDevice);
        t = t0;
        parity = par0;
        cudaFree(snap);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        if (ce != cudaSuccess) return cuda_fail(ce, "autotune trial");
        set_config(bm, bty);
        if (best_ms) *best_ms = best;
        if (cache_path) {
            std::ostringstream os;
            os << key << " " << bm << " " << bty << " " << best;
            lines.push_back(os.str());
            const std::string tmp = std::string(cache_path) + ".tmp";
            {
                std::ofstream out(tmp, std::ios::trunc);
                for (const auto &ln : lines) out << ln << "\n";
                if (!out) return fail(LB_EINVAL, "autotune: cannot write the cache file");
            }
            if (std::rename(tmp.c_str(), cache_path) != 0) return fail(LB_EINVAL, "autotune: cannot replace the cache file");
        }
        return end();
    }

    // Gradient of an observable of the state after nsteps steps with respect
    // to (G_AB, G1, G2, tau_A, tau_B), by the discrete adjoint with a
    // checkpoint every ckpt steps and recomputation of each segment.
    int grad(int64_t nsteps, int ckpt, int objective, double *J, double dJ[5])
    {
        if (nsteps < 1 || ckpt < 1) return fail(LB_EINVAL, "lb_grad needs nsteps >= 1 and ckpt_every >= 1");
        if (P[0].forcing != LB_FORCING_GUO) return fail(LB_EINVAL, "lb_grad is the adjoint of the Guo-forcing step only");
        if (!J || !dJ) return fail(LB_EINVAL, "J and dJ must not be NULL");
        const bool f32 = precision == LB_FP32;
        const lb_params &p = P[0];
        // the FP64 descriptor the adjoint kernels read (FP32 forward: the same
        // layout and parameters in FP64)
        lbk::Lat<double> L;
        if (!f32) {
            L = L64[0];
        } else {
            fill_lat(L, p);
            L.pitch = L32[0].pitch;
            L.plane = L32[0].plane;
            L.has_probe = L32[0].has_probe;
            for (int c = 0; c < 3; ++c) L.probe[c] = L32[0].probe[c];
        }
        if (objective == LB_OBJ_MU_R) {
            if (!p.walls || p.g[0] == 0.0) return fail(LB_EINVAL, "mu_r needs walls and a body force g_x");
        } else if (objective == LB_OBJ_DP) {
            if (!L.has_probe) return fail(LB_EINVAL, "the Laplace objective needs a probe (lb_set_probe)");
        } else {
            return fail(LB_EINVAL, "objective must be LB_OBJ_MU_R or LB_OBJ_DP");
        }
        int rc = begin();
        if (rc) return rc;
        // pop64: one FP64 state, the adjoint's unit; state: one state of the
        // forward precision (FP32: offsets + reference densities)
        const size_t plane_b = plane(0) * sizeof(double), pop64 = 18 * plane_b;
        const size_t state = pop_bytes(0) + ref_bytes(0);
        const int64_t nseg = (nsteps + ckpt - 1) / ckpt;
        const int seg_len = (int)std::min<int64_t>(ckpt, nsteps);
        const int tiles_x = (p.nx + lbk::TX - 1) / lbk::TX, tiles_y = (p.ny + lbk::TY - 1) / lbk::TY;
        const int ntl = tiles_x * tiles_y;
        char *mem = nullptr;
        const size_t bytes = (size_t)nseg * state + (size_t)seg_len * pop64 + 2 * pop64 + state + (f32 ? pop64 : 0) +
                             lbk::kAdjSlotCount * plane_b + 2 * plane_b + (size_t)ntl * 8 * sizeof(double) +
                             8 * sizeof(double);
        if (cudaMalloc((void **)&mem, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(LB_ENOMEM, "lb_grad: no room for checkpoints and adjoint buffers");
        }
        char *q = mem;
        auto take = [&](size_t b) { char *r = q; q += b; return r; };
        char *ckpts = take((size_t)nseg * state), *seg = take((size_t)seg_len * pop64);
        double *lam[2] = {(double *)take(pop64), (double *)take(pop64)};
        char *final_state = take(state);
        double *fT64 = f32 ? (double *)take(pop64) : nullptr;
        double *abuf = (double *)take(lbk::kAdjSlotCount * plane_b), *rho = (double *)take(2 * plane_b);
        double *gpart = (double *)take((size_t)ntl * 8 * sizeof(double)), *gout = (double *)take(8 * sizeof(double));
        cudaError_t ce = cudaMemsetAsync(gpart, 0, (size_t)ntl * 8 * sizeof(double), stream);
        auto done = [&](int code) {
            cudaStreamSynchronize(stream);
            cudaFree(mem);
            return code;
        };
        // the engine's state of population copy par <-> a compact state buffer
        auto save_state = [&](char *dst, int par) {
            cudaError_t e = cudaMemcpyAsync(dst, fbuf(0, par), pop_bytes(0), cudaMemcpyDeviceToDevice, stream);
            if (e == cudaSuccess && f32)
                e = cudaMemcpyAsync(dst + pop_bytes(0), rbuf(0, par), ref_bytes(0), cudaMemcpyDeviceToDevice, stream);
            return e;
        };
        auto load_state = [&](const char *src, int par) {
            cudaError_t e = cudaMemcpyAsync(fbuf(0, par), src, pop_bytes(0), cudaMemcpyDeviceToDevice, stream);
            if (e == cudaSuccess && f32)
                e = cudaMemcpyAsync(rbuf(0, par), src + pop_bytes(0), ref_bytes(0), cudaMemcpyDeviceToDevice, stream);
            return e;
        };
        // FP64 populations of the engine's population copy par
        auto state_f64 = [&](int par, double *out) {
            if (!f32) return cudaMemcpyAsync(out, fbuf(0, par), pop64, cudaMemcpyDeviceToDevice, stream);
            return lbk::offset_to_f64(L32[0], (const float *)fbuf(0, par), (const float *)rbuf(0, par), out, stream);
        };
        // forward sweep, keeping a checkpoint at the start of every segment
        for (int64_t s = 0; s < nseg && ce == cudaSuccess; ++s) {
            ce = save_state(ckpts + s * state, parity);
            if (ce == cudaSuccess && (rc = step(std::min<int64_t>(ckpt, nsteps - s * ckpt)))) return done(rc);
        }
        if (ce != cudaSuccess) return done(cuda_fail(ce, "lb_grad forward sweep"));
        lb_obs o;
        if ((rc = observables(&o))) return done(rc);
        double seed_a = 0.0, seed_b = 0.0;
        const int kind = objective == LB_OBJ_MU_R ? 1 : 2;
        if (objective == LB_OBJ_MU_R) {
            *J = o.mu_r;
            seed_a = -o.mu_r / o.flux_Q;   // d(Q0/Q)/dQ
        } else {
            *J = o.dp_laplace;
            double nin = 0, nout = 0;
            for (int y = 0; y < p.ny; ++y)
                for (int x = 0; x < p.nx; ++x) {
                    double dx = std::fabs(x - L.probe[0]), dy = std::fabs(y - L.probe[1]);
                    if (dx > 0.5 * p.nx) dx = p.nx - dx;
                    if (!p.walls && dy > 0.5 * p.ny) dy = p.ny - dy;
                    const double rr = std::sqrt(dx * dx + dy * dy);
                    if (rr < 0.5 * L.probe[2]) nin += 1;
                    if (rr > L.probe[2] + 6.0) nout += 1;
                }
            seed_a = 1.0 / nin;
            seed_b = -1.0 / nout;
        }
        ce = save_state(final_state, parity);
        // seed: lam(T) = dJ/df(T)
        const double *fT = f32 ? fT64 : (const double *)fbuf(0, parity);
        if (ce == cudaSuccess && f32) ce = state_f64(parity, fT64);
        if (ce == cudaSuccess) ce = lbk::adj_density(L, fT, rho, stream);
        if (ce == cudaSuccess) ce = lbk::adj_step(L, fT, rho, nullptr, abuf, gpart, lam[0], kind, seed_a, seed_b, stream);
        int cur = 0;
        // backward over the segments, recomputing each from its checkpoint in
        // the forward precision; the adjoint steps read the FP64 populations
        for (int64_t s = nseg - 1; s >= 0 && ce == cudaSuccess; --s) {
            const int len = (int)std::min<int64_t>(ckpt, nsteps - s * ckpt);
            ce = load_state(ckpts + s * state, 0);
            if (ce == cudaSuccess) ce = state_f64(0, (double *)seg);
            int par = 0;
            for (int j = 1; j < len && ce == cudaSuccess; ++j) {
                ce = launch_step(par);
                par ^= 1;
                if (ce == cudaSuccess) ce = state_f64(par, (double *)(seg + (size_t)j * pop64));
            }
            for (int j = len - 1; j >= 0 && ce == cudaSuccess; --j) {
                const double *ft = (const double *)(seg + (size_t)j * pop64);
                ce = lbk::adj_density(L, ft, rho, stream);
                if (ce == cudaSuccess)
                    ce = lbk::adj_step(L, ft, rho, lam[cur], abuf, gpart, lam[cur ^ 1], 0, 0.0, 0.0, stream);
                cur ^= 1;
            }
        }
        if (ce == cudaSuccess) ce = lbk::adj_reduce(gpart, ntl, gout, stream);
        double g[8] = {0};
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(g, gout, 8 * sizeof(double), cudaMemcpyDeviceToHost, stream);
        // put the final state back (the recomputation used both population copies)
        if (ce == cudaSuccess) ce = load_state(final_state, 0);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        if (ce != cudaSuccess) return done(cuda_fail(ce, "lb_grad adjoint sweep"));
        parity = 0;
        drop_graph();
        if ((rc = check_timeout())) return done(rc);
        // theta = (G_AB, G1, G2, tau_A, tau_B); d omega / d tau = -omega^2
        dJ[0] = g[0];
        dJ[1] = g[1];
        dJ[2] = g[2];
        dJ[3] = -g[3] * L.omega[0] * L.omega[0];
        dJ[4] = -g[4] * L.omega[1] * L.omega[1];
        if (objective == LB_OBJ_MU_R) dJ[4] += -o.mu_r / (3.0 * ((p.tau[1] - 0.5) / 3.0));   // Q0(tau_B)
        return done(end());
    }

    // One adjoint step at the current state (FP64): out = (dStep/df)^T w and
    // dtheta = <w, dStep/dtheta>, theta = (G_AB, G1, G2, tau_A, tau_B); host
    // arrays [2][9][ny][nx]; the state is left as it was.
    int step_vjp(const double *w, double *out, double dtheta[5])
    {
        if (precision != LB_FP64) return fail(LB_EINVAL, "lb_step_vjp needs LB_FP64 populations");
        if (P[0].forcing != LB_FORCING_GUO) return fail(LB_EINVAL, "lb_step_vjp is the adjoint of the Guo-forcing step only");
        if (!w) return fail(LB_EINVAL, "w is NULL");
        int rc = begin();
        if (rc) return rc;
        const lb_params &p = P[0];
        const lbk::Lat<double> &L = L64[0];
        const size_t plane_b = plane(0) * sizeof(double), pop64 = 18 * plane_b;
        const int ntl = ((p.nx + lbk::TX - 1) / lbk::TX) * ((p.ny + lbk::TY - 1) / lbk::TY);
        const size_t bytes = 2 * pop64 + lbk::kAdjSlotCount * plane_b + 2 * plane_b + (size_t)ntl * 8 * sizeof(double) +
                             8 * sizeof(double);
        char *mem = nullptr;
        if (cudaMalloc((void **)&mem, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(LB_ENOMEM, "lb_step_vjp: no room for the adjoint buffers");
        }
        char *q = mem;
        auto take = [&](size_t b) { char *r = q; q += b; return r; };
        double *lam_in = (double *)take(pop64), *lam_out = (double *)take(pop64);
        double *abuf = (double *)take(lbk::kAdjSlotCount * plane_b), *rho = (double *)take(2 * plane_b);
        double *gpart = (double *)take((size_t)ntl * 8 * sizeof(double)), *gout = (double *)take(8 * sizeof(double));
        const double *f = (const double *)fbuf(0, parity);
        const size_t row = (size_t)p.nx * sizeof(double), prow = (size_t)L.pitch * sizeof(double);
        cudaError_t ce = cudaMemsetAsync(mem, 0, 2 * pop64, stream);   // the pitch padding stays zero
        if (ce == cudaSuccess) ce = cudaMemsetAsync(gpart, 0, (size_t)ntl * 8 * sizeof(double), stream);
        if (ce == cudaSuccess)
            ce = cudaMemcpy2DAsync(lam_in, prow, w, row, row, (size_t)18 * p.ny, cudaMemcpyHostToDevice, stream);
        if (ce == cudaSuccess) ce = lbk::adj_density(L, f, rho, stream);
        if (ce == cudaSuccess) ce = lbk::adj_step(L, f, rho, lam_in, abuf, gpart, lam_out, 0, 0.0, 0.0, stream);
        if (ce == cudaSuccess) ce = lbk::adj_reduce(gpart, ntl, gout, stream);
        double g[8] = {0};
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(g, gout, 8 * sizeof(double), cudaMemcpyDeviceToHost, stream);
        if (ce == cudaSuccess && out)
            ce = cudaMemcpy2DAsync(out, row, lam_out, prow, row, (size_t)18 * p.ny, cudaMemcpyDeviceToHost, stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        cudaStreamSynchronize(stream);
        cudaFree(mem);
        if (ce != cudaSuccess) return cuda_fail(ce, "lb_step_vjp");
        if (dtheta) {   // d omega / d tau = -omega^2
            dtheta[0] = g[0];
            dtheta[1] = g[1];
            dtheta[2] = g[2];
            dtheta[3] = -g[3] * L.omega[0] * L.omega[0];
            dtheta[4] = -g[4] * L.omega[1] * L.omega[1];
        }
        return end();
    }

    int observables(lb_obs *o)
    {
        int rc = begin();
        if (rc) return rc;
        const int nt = (int)tiles.size();
        if ((rc = check_timeout())) return rc;
        LB_CUDA(launch_density_obs(parity, 0, nt));
        LB_CUDA(launch_observe(parity, 0, nt, d_partials, nullptr, nullptr, nullptr));
        LB_CUDA(launch_finalize());
        std::vector<double> h((size_t)n * lbk::kObsStride);
        LB_CUDA(cudaMemcpyAsync(h.data(), d_obs, h.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
        LB_CUDA(cudaStreamSynchronize(stream));
        bool all_finite = true;
        for (int l = 0; l < n; ++l) {
            const double *s = &h[(size_t)l * lbk::kObsStride];
            lb_obs &r = o[l];
            std::memset(&r, 0, sizeof r);
            r.t = t;
            r.mass[0] = s[lbk::oMassA];
            r.mass[1] = s[lbk::oMassB];
            r.mom[0][0] = s[lbk::oMomAx];
            r.mom[0][1] = s[lbk::oMomAy];
            r.mom[1][0] = s[lbk::oMomBx];
            r.mom[1][1] = s[lbk::oMomBy];
            r.flux_Q = s[lbk::oQ];
            r.mu_r = s[lbk::oMuR];
            r.dp_laplace = s[lbk::oDp];
            r.R_eff = s[lbk::oReff];
            r.umax = s[lbk::oUmax];
            r.finite = s[lbk::oFinite] != 0.0 ? 1 : 0;
            all_finite = all_finite && r.finite;
        }
        rc = end();
        if (rc) return rc;
        if (!all_finite) return fail(LB_EUNSTABLE, "a density or velocity is not finite");
        return LB_OK;
    }

    // Pressure tensor at the current time (k_pressure): the lattice sums of
    // its six components for lattice l into sums[6] and, when P is given, the
    // dense per-node field of lattice l into P [2][3][ny][nx]; host memory.
    int pressure(int l, double *P, double *sums)
    {
        int rc = begin();
        if (rc) return rc;
        if ((rc = check_timeout())) return rc;
        if (!d_psum && cudaMalloc((void **)&d_psum, (size_t)n * lbk::kPStride * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            d_psum = nullptr;
            return fail(LB_ENOMEM, "cudaMalloc of the pressure-tensor sums failed");
        }
        const int nt = (int)tiles.size();
        const size_t cells = (size_t)nx(l) * ny(l);
        if (P && (rc = ensure_tmp(6 * cells))) return rc;
        LB_CUDA(launch_density_obs(parity, 0, nt));
        if (precision == LB_FP64) {
            const lbk::Lat<double> *L = (const lbk::Lat<double> *)d_lats;
            LB_CUDA(lbk::Launch<double>::pressure(L, d_tiles, 0, nt, parity, d_partials, nullptr, stream));
            LB_CUDA(lbk::Launch<double>::pressure_sum(L, n, d_partials, d_psum, stream));
            if (P)
                LB_CUDA(lbk::Launch<double>::pressure(L, d_tiles, tile_begin(l), tile_end(l) - tile_begin(l), parity,
                                                      nullptr, d_tmp, stream));
        } else {
            const lbk::Lat<float> *L = (const lbk::Lat<float> *)d_lats;
            LB_CUDA(lbk::Launch<float>::pressure(L, d_tiles, 0, nt, parity, d_partials, nullptr, stream));
            LB_CUDA(lbk::Launch<float>::pressure_sum(L, n, d_partials, d_psum, stream));
            if (P)
                LB_CUDA(lbk::Launch<float>::pressure(L, d_tiles, tile_begin(l), tile_end(l) - tile_begin(l), parity,
                                                     nullptr, d_tmp, stream));
        }
        double h[lbk::kPStride];
        LB_CUDA(cudaMemcpyAsync(h, d_psum + (size_t)l * lbk::kPStride, sizeof h, cudaMemcpyDeviceToHost, stream));
        if (P) LB_CUDA(cudaMemcpyAsync(P, d_tmp, 6 * cells * sizeof(double), cudaMemcpyDeviceToHost, stream));
        LB_CUDA(cudaStreamSynchronize(stream));
        if (sums)
            for (int a = 0; a < lbk::kNumPSlots; ++a) sums[a] = h[a];
        return end();
    }

    int get_fields(int l, double *rho, double *mom, double *ubar)
    {
        const size_t cells = (size_t)nx(l) * ny(l);
        int rc = begin();
        if (rc) return rc;
        if ((rc = ensure_tmp(8 * cells))) return rc;
        LB_CUDA(launch_density_obs(parity, tile_begin(l), tile_end(l) - tile_begin(l)));
        LB_CUDA(launch_observe(parity, tile_begin(l), tile_end(l) - tile_begin(l), nullptr, d_tmp, d_tmp + 2 * cells,
                               d_tmp + 6 * cells));
        if (rho) LB_CUDA(cudaMemcpyAsync(rho, d_tmp, 2 * cells * sizeof(double), cudaMemcpyDeviceToHost, stream));
        if (mom)
            LB_CUDA(cudaMemcpyAsync(mom, d_tmp + 2 * cells, 4 * cells * sizeof(double), cudaMemcpyDeviceToHost, stream));
        if (ubar)
            LB_CUDA(cudaMemcpyAsync(ubar, d_tmp + 6 * cells, 2 * cells * sizeof(double), cudaMemcpyDeviceToHost, stream));
        LB_CUDA(cudaStreamSynchronize(stream));
        return end();
    }

    int set_fields(int l, const double *rho, const double *u, bool device_ptrs)
    {
        if (!rho) return fail(LB_EINVAL, "rho is NULL");
        const size_t cells = (size_t)nx(l) * ny(l);
        int rc = begin();
        if (rc) return rc;
        const double *drho = rho, *du = u;
        if (!device_ptrs) {
            if ((rc = ensure_tmp(4 * cells))) return rc;
            LB_CUDA(cudaMemcpyAsync(d_tmp, rho, 2 * cells * sizeof(double), cudaMemcpyHostToDevice, stream));
            drho = d_tmp;
            du = nullptr;
            if (u) {
                LB_CUDA(cudaMemcpyAsync(d_tmp + 2 * cells, u, 2 * cells * sizeof(double), cudaMemcpyHostToDevice,
                                        stream));
                du = d_tmp + 2 * cells;
            }
        }
        if (precision == LB_FP64)
            LB_CUDA(lbk::Launch<double>::init((const lbk::Lat<double> *)d_lats, l, nx(l), ny(l), drho, du, parity, stream));
        else
            LB_CUDA(lbk::Launch<float>::init((const lbk::Lat<float> *)d_lats, l, nx(l), ny(l), drho, du, parity, stream));
        if (!device_ptrs) LB_CUDA(cudaStreamSynchronize(stream));
        return end();
    }

    int get_pops(int l, double *f)
    {
        if (!f) return fail(LB_EINVAL, "f is NULL");
        const size_t cells = (size_t)nx(l) * ny(l);
        int rc = begin();
        if (rc) return rc;
        if ((rc = ensure_tmp(18 * cells))) return rc;
        if (precision == LB_FP64)
            LB_CUDA(lbk::Launch<double>::get_pops((const lbk::Lat<double> *)d_lats, l, nx(l), ny(l), parity, d_tmp, stream));
        else
            LB_CUDA(lbk::Launch<float>::get_pops((const lbk::Lat<float> *)d_lats, l, nx(l), ny(l), parity, d_tmp, stream));
        LB_CUDA(cudaMemcpyAsync(f, d_tmp, 18 * cells * sizeof(double), cudaMemcpyDeviceToHost, stream));
        LB_CUDA(cudaStreamSynchronize(stream));
        return end();
    }

    int set_pops(int l, const double *f)
    {
        if (!f) return fail(LB_EINVAL, "f is NULL");
        const size_t cells = (size_t)nx(l) * ny(l);
        int rc = begin();
        if (rc) return rc;
        if ((rc = ensure_tmp(18 * cells))) return rc;
        LB_CUDA(cudaMemcpyAsync(d_tmp, f, 18 * cells * sizeof(double), cudaMemcpyHostToDevice, stream));
        if (precision == LB_FP64)
            LB_CUDA(lbk::Launch<double>::set_pops((const lbk::Lat<double> *)d_lats, l, nx(l), ny(l), parity, d_tmp, stream));
        else
            LB_CUDA(lbk::Launch<float>::set_pops((const lbk::Lat<float> *)d_lats, l, nx(l), ny(l), parity, d_tmp, stream));
        LB_CUDA(cudaStreamSynchronize(stream));
        return end();
    }

    int set_probe(int l, double cx, double cy, double R)
    {
        if (!is_fin(cx) || !is_fin(cy) || !is_fin(R)) return fail(LB_EINVAL, "non-finite probe");
        int rc = begin();
        if (rc) return rc;
        const int has = R > 0.0 ? 1 : 0;
        const double pr[3] = {cx, cy, R};
        if (precision == LB_FP64) {
            L64[l].has_probe = has;
            std::memcpy(L64[l].probe, pr, sizeof pr);
            LB_CUDA(cudaMemcpyAsync((lbk::Lat<double> *)d_lats + l, &L64[l], sizeof(L64[l]), cudaMemcpyHostToDevice,
                                    stream));
        } else {
            L32[l].has_probe = has;
            std::memcpy(L32[l].probe, pr, sizeof pr);
            LB_CUDA(cudaMemcpyAsync((lbk::Lat<float> *)d_lats + l, &L32[l], sizeof(L32[l]), cudaMemcpyHostToDevice,
                                    stream));
        }
        LB_CUDA(cudaStreamSynchronize(stream));
        return end();
    }
};

namespace {

int engine_create(const lb_params *p, int n, lb_engine **out)
{
    *out = nullptr;
    if (n < 1) return fail(LB_EINVAL, "need at least one lattice");
    for (int i = 0; i < n; ++i) {
        int rc = validate(&p[i], i);
        if (rc) return rc;
        if (p[i].precision != p[0].precision) return fail(LB_EINVAL, "all lattices of a batch need the same precision");
    }
    lb_engine *e = new (std::nothrow) lb_engine();
    if (!e) return fail(LB_ENOMEM, "host allocation failed");
    e->precision = p[0].precision;
    e->n = n;
    e->P.assign(p, p + n);
    auto bail = [&](int rc) {
        delete e;
        return rc;
    };
    if (cudaGetDevice(&e->device) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(LB_ECUDA, "no CUDA device"));
    }
    cudaError_t ce;
    if (p[0].stream) {
        e->stream = (cudaStream_t)p[0].stream;
    } else {
        if ((ce = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(cuda_fail(ce, "cudaStreamCreateWithFlags"));
        e->own_stream = true;
    }

    // layout: per lattice two population copies and the density field
    const size_t rs = e->real_size();
    std::vector<size_t> off_f0(n), off_f1(n), off_r0(n), off_r1(n);
    size_t total = 0;
    for (int l = 0; l < n; ++l) {
        const size_t pitch = align_up((size_t)p[l].nx, 32), plane = pitch * p[l].ny;
        off_f0[l] = total;
        total = align_up(total + 18 * plane * rs, kAlign);
        off_f1[l] = total;
        total = align_up(total + 18 * plane * rs, kAlign);
        off_r0[l] = total;
        total = align_up(total + 2 * plane * rs, kAlign);
        off_r1[l] = total;
        total = align_up(total + 2 * plane * rs, kAlign);
    }
    e->pool_bytes = total;
    if (cudaMalloc(&e->d_pool, total) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(LB_ENOMEM, "cudaMalloc of the lattice state failed"));
    }
    if ((ce = cudaMemsetAsync(e->d_pool, 0, total, e->stream)) != cudaSuccess) return bail(cuda_fail(ce, "cudaMemsetAsync"));

    // tiles in raster order, lattice by lattice
    for (int l = 0; l < n; ++l) {
        const int begin = (int)e->tiles.size();
        for (int y0 = 0; y0 < p[l].ny; y0 += lbk::TY)
            for (int x0 = 0; x0 < p[l].nx; x0 += lbk::TX) e->tiles.push_back(make_int4(l, x0, y0, 0));
        const int end = (int)e->tiles.size();
        char *base = (char *)e->d_pool;
        if (e->precision == LB_FP64) {
            lbk::Lat<double> L;
            fill_lat(L, p[l]);
            L.f[0] = (double *)(base + off_f0[l]);
            L.f[1] = (double *)(base + off_f1[l]);
            L.rho[0] = (double *)(base + off_r0[l]);
            L.rho[1] = (double *)(base + off_r1[l]);
            L.tile_begin = begin;
            L.tile_end = end;
            e->L64.push_back(L);
        } else {
            lbk::Lat<float> L;
            fill_lat(L, p[l]);
            L.f[0] = (float *)(base + off_f0[l]);
            L.f[1] = (float *)(base + off_f1[l]);
            L.rho[0] = (float *)(base + off_r0[l]);
            L.rho[1] = (float *)(base + off_r1[l]);
            L.tile_begin = begin;
            L.tile_end = end;
            e->L32.push_back(L);
        }
    }
    const size_t lat_bytes = e->precision == LB_FP64 ? n * sizeof(lbk::Lat<double>) : n * sizeof(lbk::Lat<float>);
    const void *lat_src = e->precision == LB_FP64 ? (const void *)e->L64.data() : (const void *)e->L32.data();
    if (cudaMalloc(&e->d_lats, lat_bytes) != cudaSuccess ||
        cudaMalloc((void **)&e->d_tiles, e->tiles.size() * sizeof(int4)) != cudaSuccess ||
        cudaMalloc((void **)&e->d_partials, e->tiles.size() * lbk::kAccStride * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&e->d_obs, (size_t)n * lbk::kObsStride * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(LB_ENOMEM, "cudaMalloc of the descriptors failed"));
    }
    // time-step tiles for every supported tile height, and the persistent
    // launch's control block and error word
    for (int ti = 0; ti < 3; ++ti) {
        const int tyv = kTileHeights[ti];
        std::vector<int> counts(n, 0);
        for (int l = 0; l < n; ++l) {
            const size_t before = e->stiles[ti].size();
            for (int y0 = 0; y0 < p[l].ny; y0 += tyv)
                for (int x0 = 0; x0 < p[l].nx; x0 += lbk::TX) e->stiles[ti].push_back(make_int4(l, x0, y0, 0));
            counts[l] = (int)(e->stiles[ti].size() - before);
        }
        if (cudaMalloc((void **)&e->d_stiles[ti], e->stiles[ti].size() * sizeof(int4)) != cudaSuccess ||
            cudaMalloc((void **)&e->d_sntiles[ti], n * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(LB_ENOMEM, "cudaMalloc of the tile lists failed"));
        }
        if ((ce = cudaMemcpyAsync(e->d_stiles[ti], e->stiles[ti].data(), e->stiles[ti].size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, e->stream)) != cudaSuccess ||
            (ce = cudaMemcpyAsync(e->d_sntiles[ti], counts.data(), n * sizeof(int), cudaMemcpyHostToDevice,
                                  e->stream)) != cudaSuccess ||
            (ce = cudaStreamSynchronize(e->stream)) != cudaSuccess)
            return bail(cuda_fail(ce, "tile list upload"));
        e->persist_bps[ti] = e->precision == LB_FP64 ? lbk::Launch<double>::persistent_blocks_per_sm(tyv)
                                                     : lbk::Launch<float>::persistent_blocks_per_sm(tyv);
    }
    if (cudaMalloc(&e->d_ctl, e->ctl_bytes()) != cudaSuccess || cudaMalloc((void **)&e->d_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(LB_ENOMEM, "cudaMalloc of the persistent control block failed"));
    }
    if ((ce = cudaMemsetAsync(e->d_err, 0, sizeof(int), e->stream)) != cudaSuccess) return bail(cuda_fail(ce, "cudaMemsetAsync"));
    {
        int khz = 0;
        cudaDeviceGetAttribute(&e->sm_count, cudaDevAttrMultiProcessorCount, e->device);
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, e->device);
        e->wait_cycles = (long long)(2.0 * (khz > 0 ? khz : 2000000) * 1000.0);   // 2 s
    }
    if ((ce = cudaMemcpyAsync(e->d_lats, lat_src, lat_bytes, cudaMemcpyHostToDevice, e->stream)) != cudaSuccess ||
        (ce = cudaMemcpyAsync(e->d_tiles, e->tiles.data(), e->tiles.size() * sizeof(int4), cudaMemcpyHostToDevice,
                              e->stream)) != cudaSuccess ||
        (ce = cudaStreamSynchronize(e->stream)) != cudaSuccess)
        return bail(cuda_fail(ce, "descriptor upload"));
    if (e->precision == LB_FP32) {
        const int rc = e->build_tma_maps();
        if (rc) return bail(rc);
    }
    // the chains of a batch's step graph (as many as lattices, at most
    // kChains): lattices by node count, each to the group with the fewest
    // nodes so far
    if (n >= 2) {
        const int nc = std::min(n, kChains);
        std::vector<int> order(n), group(n, 0);
        for (int l = 0; l < n; ++l) order[l] = l;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (int64_t)p[a].nx * p[a].ny > (int64_t)p[b].nx * p[b].ny;
        });
        int64_t load[kChains] = {};
        for (int l : order) {
            int g = 0;
            for (int k = 1; k < nc; ++k)
                if (load[k] < load[g]) g = k;
            group[l] = g;
            load[g] += (int64_t)p[l].nx * p[l].ny;
        }
        for (int ti = 0; ti < 3; ++ti) {
            const int tyv = kTileHeights[ti];
            std::vector<int4> list;
            for (int g = 0; g < nc; ++g) {
                e->c_off[ti][g] = (int)list.size();
                for (int pass = 0; pass < 2; ++pass) {
                    for (const int4 &t : e->stiles[ti])
                        if (group[t.x] == g && lbk::tma_box_tile(p[t.x].nx, p[t.x].ny, t.y, t.z, tyv) == (pass == 0))
                            list.push_back(make_int4(t.x, t.y, t.z, pass == 0 ? lbk::kTmaBoxMark : 0));
                    if (pass == 0) e->c_box[ti][g] = (int)list.size() - e->c_off[ti][g];
                }
                e->c_cnt[ti][g] = (int)list.size() - e->c_off[ti][g];
            }
            if (cudaMalloc((void **)&e->d_ctiles[ti], list.size() * sizeof(int4)) != cudaSuccess) {
                cudaGetLastError();
                return bail(fail(LB_ENOMEM, "cudaMalloc of the chain tile lists failed"));
            }
            if ((ce = cudaMemcpyAsync(e->d_ctiles[ti], list.data(), list.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                      e->stream)) != cudaSuccess ||
                (ce = cudaStreamSynchronize(e->stream)) != cudaSuccess)
                return bail(cuda_fail(ce, "chain tile list upload"));
        }
        if ((ce = cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming)) != cudaSuccess)
            return bail(cuda_fail(ce, "cudaEventCreateWithFlags"));
        for (int g = 1; g < nc; ++g)
            if ((ce = cudaStreamCreateWithFlags(&e->aux[g], cudaStreamNonBlocking)) != cudaSuccess ||
                (ce = cudaEventCreateWithFlags(&e->ev_join[g], cudaEventDisableTiming)) != cudaSuccess)
                return bail(cuda_fail(ce, "auxiliary streams of the step graph"));
        e->nchains = nc;
    }
    *out = e;
    return LB_OK;
}

struct SaveHeader {
    char magic[8];
    int32_t precision, nx, ny, pad;
    int64_t t;
    int64_t bytes;
};

}  // namespace

namespace lbk {
void set_last_error(const char *msg) { g_err = msg; }
int validate_params(const lb_params *p, int index) { return validate(p, index); }
}  // namespace lbk

struct lb_handle {
    lb_engine *e;
};
struct lb_batch {
    lb_engine *e;
};

extern "C" {

const char *lb_last_error(void) { return g_err.c_str(); }

int lb_create(const lb_params *p, lb_handle **out)
{
    if (!out) return fail(LB_EINVAL, "out is NULL");
    *out = nullptr;
    lb_engine *e = nullptr;
    int rc = engine_create(p, 1, &e);
    if (rc) return rc;
    lb_handle *h = new (std::nothrow) lb_handle{e};
    if (!h) {
        delete e;
        return fail(LB_ENOMEM, "host allocation failed");
    }
    *out = h;
    return LB_OK;
}

void lb_destroy(lb_handle *h)
{
    if (!h) return;
    delete h->e;
    delete h;
}

#define CHECK_H(h) \
    if (!(h) || !(h)->e) return fail(LB_EINVAL, "handle is NULL")

int lb_set_fields(lb_handle *h, const double *rho, const double *u)
{
    CHECK_H(h);
    int rc = h->e->set_fields(0, rho, u, false);
    if (!rc) h->e->t = 0;
    return rc;
}

int lb_set_fields_device(lb_handle *h, const double *rho, const double *u)
{
    CHECK_H(h);
    int rc = h->e->set_fields(0, rho, u, true);
    if (!rc) h->e->t = 0;
    return rc;
}

int lb_step(lb_handle *h, int64_t n)
{
    CHECK_H(h);
    return h->e->step(n);
}

int lb_synchronize(lb_handle *h)
{
    CHECK_H(h);
    cudaError_t ce = cudaStreamSynchronize(h->e->stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamSynchronize");
    return h->e->check_timeout();
}

int lb_set_config(lb_handle *h, int32_t mode, int32_t tile_height)
{
    CHECK_H(h);
    return h->e->set_config(mode, tile_height);
}

int lb_get_config(const lb_handle *h, int32_t *mode, int32_t *tile_height)
{
    if (!h || !h->e || !mode || !tile_height) return fail(LB_EINVAL, "NULL argument");
    *mode = h->e->mode;
    *tile_height = h->e->ty;
    return LB_OK;
}

int lb_autotune(lb_handle *h, int32_t trial_steps, const char *cache_path, double *best_ms)
{
    CHECK_H(h);
    return h->e->autotune(trial_steps, cache_path, best_ms);
}

int64_t lb_time(const lb_handle *h) { return (h && h->e) ? h->e->t : -1; }

int lb_set_probe(lb_handle *h, double cx, double cy, double R)
{
    CHECK_H(h);
    return h->e->set_probe(0, cx, cy, R);
}

int lb_observables(lb_handle *h, lb_obs *o)
{
    CHECK_H(h);
    if (!o) return fail(LB_EINVAL, "o is NULL");
    return h->e->observables(o);
}

int lb_get_fields(lb_handle *h, double *rho, double *mom, double *ubar)
{
    CHECK_H(h);
    return h->e->get_fields(0, rho, mom, ubar);
}

int lb_pressure_tensor(lb_handle *h, double *P, double sums[6])
{
    CHECK_H(h);
    return h->e->pressure(0, P, sums);
}

int lb_step_vjp(lb_handle *h, const double *w, double *out, double dtheta[5])
{
    CHECK_H(h);
    return h->e->step_vjp(w, out, dtheta);
}

int lb_get_populations(lb_handle *h, double *f)
{
    CHECK_H(h);
    return h->e->get_pops(0, f);
}

int lb_set_populations(lb_handle *h, const double *f, int64_t t)
{
    CHECK_H(h);
    int rc = h->e->set_pops(0, f);
    if (!rc) h->e->t = t;
    return rc;
}

int lb_save(lb_handle *h, void *buf, size_t *len)
{
    CHECK_H(h);
    if (!len) return fail(LB_EINVAL, "len is NULL");
    lb_engine *e = h->e;
    const size_t bytes = e->pop_bytes(0) + e->ref_bytes(0);
    const size_t need = sizeof(SaveHeader) + bytes;
    if (!buf) {
        *len = need;
        return LB_OK;
    }
    if (*len < need) return fail(LB_EINVAL, "checkpoint buffer too small");
    SaveHeader hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, "LBGB300", 8);
    hd.precision = e->precision;
    hd.nx = e->nx(0);
    hd.ny = e->ny(0);
    hd.t = e->t;
    hd.bytes = (int64_t)bytes;
    std::memcpy(buf, &hd, sizeof hd);
    int rc = e->begin();
    if (rc) return rc;
    LB_CUDA(cudaMemcpyAsync((char *)buf + sizeof hd, e->fbuf(0, e->parity), e->pop_bytes(0), cudaMemcpyDeviceToHost,
                            e->stream));
    if (e->ref_bytes(0))
        LB_CUDA(cudaMemcpyAsync((char *)buf + sizeof hd + e->pop_bytes(0), e->rbuf(0, e->parity), e->ref_bytes(0),
                                cudaMemcpyDeviceToHost, e->stream));
    LB_CUDA(cudaStreamSynchronize(e->stream));
    *len = need;
    return e->end();
}

int lb_load(lb_handle *h, const void *buf, size_t len)
{
    CHECK_H(h);
    if (!buf || len < sizeof(SaveHeader)) return fail(LB_EINVAL, "checkpoint buffer too small");
    lb_engine *e = h->e;
    SaveHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    const size_t bytes = e->pop_bytes(0) + e->ref_bytes(0);
    if (std::memcmp(hd.magic, "LBGB300", 8) != 0 || hd.precision != e->precision || hd.nx != e->nx(0) ||
        hd.ny != e->ny(0) || (size_t)hd.bytes != bytes || len < sizeof hd + bytes)
        return fail(LB_EINVAL, "checkpoint does not match this lattice");
    int rc = e->begin();
    if (rc) return rc;
    LB_CUDA(cudaMemcpyAsync(e->fbuf(0, e->parity), (const char *)buf + sizeof hd, e->pop_bytes(0),
                            cudaMemcpyHostToDevice, e->stream));
    if (e->ref_bytes(0))
        LB_CUDA(cudaMemcpyAsync(e->rbuf(0, e->parity), (const char *)buf + sizeof hd + e->pop_bytes(0), e->ref_bytes(0),
                                cudaMemcpyHostToDevice, e->stream));
    LB_CUDA(cudaStreamSynchronize(e->stream));
    e->t = hd.t;
    return e->end();
}

int lb_profile(lb_handle *h, int32_t nsteps, void *flush_buf, size_t flush_bytes, double ms[3])
{
    CHECK_H(h);
    return h->e->profile(nsteps, flush_buf, flush_bytes, ms);
}

int lb_grad(lb_handle *h, int64_t nsteps, int32_t ckpt_every, int32_t objective, double *J, double dJ[5])
{
    CHECK_H(h);
    return h->e->grad(nsteps, ckpt_every, objective, J, dJ);
}

int lb_batch_create(const lb_params *p, int32_t n, lb_batch **out)
{
    if (!out) return fail(LB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!p) return fail(LB_EINVAL, "params is NULL");
    lb_engine *e = nullptr;
    int rc = engine_create(p, n, &e);
    if (rc) return rc;
    lb_batch *b = new (std::nothrow) lb_batch{e};
    if (!b) {
        delete e;
        return fail(LB_ENOMEM, "host allocation failed");
    }
    *out = b;
    return LB_OK;
}

void lb_batch_destroy(lb_batch *b)
{
    if (!b) return;
    delete b->e;
    delete b;
}

#define CHECK_B(b, i)                                                           \
    if (!(b) || !(b)->e) return fail(LB_EINVAL, "batch is NULL");               \
    if ((i) < 0 || (i) >= (b)->e->n) return fail(LB_EINVAL, "lattice index out of range")

int lb_batch_size(const lb_batch *b) { return (b && b->e) ? b->e->n : -1; }

int lb_batch_set_fields(lb_batch *b, int32_t i, const double *rho, const double *u)
{
    CHECK_B(b, i);
    return b->e->set_fields(i, rho, u, false);
}

int lb_batch_step(lb_batch *b, int64_t n)
{
    CHECK_B(b, 0);
    return b->e->step(n);
}

int lb_batch_synchronize(lb_batch *b)
{
    CHECK_B(b, 0);
    cudaError_t ce = cudaStreamSynchronize(b->e->stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamSynchronize");
    return b->e->check_timeout();
}

int lb_batch_set_config(lb_batch *b, int32_t mode, int32_t tile_height)
{
    CHECK_B(b, 0);
    return b->e->set_config(mode, tile_height);
}

int lb_batch_get_config(const lb_batch *b, int32_t *mode, int32_t *tile_height)
{
    if (!b || !b->e || !mode || !tile_height) return fail(LB_EINVAL, "NULL argument");
    *mode = b->e->mode;
    *tile_height = b->e->ty;
    return LB_OK;
}

int lb_batch_autotune(lb_batch *b, int32_t trial_steps, const char *cache_path, double *best_ms)
{
    CHECK_B(b, 0);
    return b->e->autotune(trial_steps, cache_path, best_ms);
}

int lb_batch_set_wait_limit(lb_batch *b, double seconds, int32_t drop_tile)
{
    CHECK_B(b, 0);
    if (!(seconds > 0.0) || !std::isfinite(seconds)) return fail(LB_EINVAL, "wait limit must be finite and > 0");
    int khz = 0;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, b->e->device);
    b->e->wait_cycles = (long long)(seconds * (khz > 0 ? khz : 2000000) * 1000.0);
    b->e->drop_tile = drop_tile < 0 ? -1 : drop_tile;
    b->e->drop_graph();
    return LB_OK;
}

int lb_batch_set_probe(lb_batch *b, int32_t i, double cx, double cy, double R)
{
    CHECK_B(b, i);
    return b->e->set_probe(i, cx, cy, R);
}

int lb_batch_observables(lb_batch *b, lb_obs *o)
{
    CHECK_B(b, 0);
    if (!o) return fail(LB_EINVAL, "o is NULL");
    return b->e->observables(o);
}

int lb_batch_get_fields(lb_batch *b, int32_t i, double *rho, double *mom, double *ubar)
{
    CHECK_B(b, i);
    return b->e->get_fields(i, rho, mom, ubar);
}

int lb_batch_pressure_tensor(lb_batch *b, int32_t i, double *P, double sums[6])
{
    CHECK_B(b, i);
    return b->e->pressure(i, P, sums);
}

int lb_batch_profile(lb_batch *b, int32_t nsteps, void *flush_buf, size_t flush_bytes, double ms[3])
{
    CHECK_B(b, 0);
    return b->e->profile(nsteps, flush_buf, flush_bytes, ms);
}

}  // extern "C"

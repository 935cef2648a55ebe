// lb_tma.cu -- the FP32 one-pass time step with each tile's populations and
// reference densities, halo included, brought into shared memory by the
// tensor memory accelerator (cp.async.bulk.tensor, completion on an mbarrier)
// instead of per-thread loads.  The explicit FP32 arithmetic of lb_vops.cuh,
// in the same order as fused_tile, so the results are the same bit for bit:
// the densities of the staged nodes are the sums of Eq. (6) over the boxed
// populations, then the forces of Eqs. (8), (9), the collision of Eqs. (1),
// (2), (5) and the push streaming of collide_site.
//
// Box of a tile (x0, y0) of 32 x TY nodes: columns x0 - 4 .. x0 + 35 (the
// D2Q25 halo needs 2; 4 keep the x offset a multiple of 16 bytes), rows
// y0 - 2 .. y0 + TY + 1, all 18 population planes; a second box holds the 2
// reference-density planes.  Parts of the box beyond the lattice are filled
// with zeros by the copy and not used: the halo slots there (across a
// periodic edge, or wall ghost rows) are formed as in fused_tile.  The
// caller launches this kernel over the tiles that box_tile accepts and the
// plain one-pass kernel over the others (ragged tiles, lattices smaller than
// the box), so neither carries the other's registers.
#include "lb_kernels.cuh"
#include "lb_launch.h"

namespace lbk {

namespace {

template <int TYv>
struct TmaBox {
    static constexpr int H = TYv + 2 * HALO;
    static constexpr int kPop = kTmaBoxW * H * 18;   // floats
    static constexpr int kRef = kTmaBoxW * H * 2;
    static constexpr int kStage = kPop + kRef;
    static constexpr unsigned kBytes = (unsigned)kStage * 4u;
    static_assert((kPop * 4) % 128 == 0 && (kStage * 4) % 128 == 0, "stage buffers stay 128-byte aligned");
};

// Resident blocks per SM the kernel is compiled for: as the plain one-pass
// kernel, unless the staging buffer leaves room for fewer.
template <int TYv>
constexpr int kTmaMinBlocks = (225 * 1024) / (TmaBox<TYv>::kBytes + 8 * 1024) < kCollideMinBlocks<float, TYv>
                                  ? (225 * 1024) / (TmaBox<TYv>::kBytes + 8 * 1024)
                                  : kCollideMinBlocks<float, TYv>;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of phase `phase` of *bar.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned phase, long long limit)
{
    const long long start = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - start > limit) return false;
    return true;
}

// Bring the box at (x, y, z) of the tensor into L2 (no shared memory, no
// completion to wait for).
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int x, int y, int z)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(map), "r"(x), "r"(y), "r"(z)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Staged density and psi of the tile and its halo as (species A, species B)
// pairs per node, so that one 64-bit shared load serves both species.
template <int TYv>
struct PairSmem {
    float2 sr[TYv + 2 * HALO][SW];
    float2 sp[TYv + 2 * HALO][SW];
    Lat<float> L;   // descriptor copy: stores to the populations cannot alias it
};

// The pair planes as collide_site reads them (the interface of SplitStage):
// both species' forces of Eqs. (8), (9) and rho_k g, their densities, and
// the densities a push re-references with, each as an (A, B) pair.
template <int SHv>
struct PairStage {
    const float2 (*sr)[SW];
    const float2 (*sp)[SW];
    __device__ __forceinline__ float2 density2(int cy, int cx) const { return sr[cy][cx]; }
    // Eq. (8) + Eq. (9) + rho_k g, the operations of force_at on each lane
    __device__ __forceinline__ void force2(const Lat<float> &L, int cx, int cy, float2 &Fx, float2 &Fy) const
    {
        auto at_psi = [&](int dy, int dx) { return sp[cy + dy][cx + dx]; };
        auto at_rho = [&](int dy, int dx) { return sr[cy + dy][cx + dx]; };
        float2 msx, msy, s3x, s3y;
        vq25c<float2>(at_psi, L.cw, p25f, msx, msy);
        vq9<float2>(at_rho, s3x, s3y);   // lane j: sums over species j's density
        // each species is pushed by the other's density sum
        vforce<float2>(sp[cy][cx], sr[cy][cx], msx, msy, vswap(s3x), vswap(s3y), L.GAB, L.g[0], L.g[1], Fx, Fy);
    }
    template <int EX, int EY>
    __device__ __forceinline__ float2 dest(int cx, int cy) const
    {
        return sr[cy + EY][cx + EX];
    }
};

// Staged slot (sx, sy) of the h-th position of the halo ring: two rows above,
// two below, then the two columns on each side of the tile's rows.
template <int TYv>
__device__ __forceinline__ void ring_slot(int h, int &sx, int &sy)
{
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
}

// The slot's node lies beyond the lattice (across a periodic edge, or a wall
// ghost row): not in the box's lattice part.
__device__ __forceinline__ bool slot_outside(const Lat<float> &G, int4 t, int sx, int sy)
{
    const int gx = t.y + sx - HALO, gy = t.z + sy - HALO;
    return gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny;
}

// fused_tile with the tile's and the halo's populations and reference
// densities read from the box (pop: [18][H][40], ref: [2][H][40]).  The tile
// is full.  Halo slots beyond the lattice were staged by the caller.
template <int TYv>
__device__ __forceinline__ void fused_tile_box(const Lat<float> *__restrict__ lats, int4 t, int parity,
                                               PairSmem<TYv> &sm, const float *__restrict__ pop,
                                               const float *__restrict__ ref)
{
    constexpr int SHv = TYv + 2 * HALO, H = SHv, W = kTmaBoxW;
    const Lat<float> &G = lats[t.x];
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int i = tid; i < (int)(sizeof(Lat<float>) / 4); i += TX * TYv)
        reinterpret_cast<uint32_t *>(&sm.L)[i] = reinterpret_cast<const uint32_t *>(&G)[i];
    // staged slot (sx, sy) is box column sx + 2, row sy; its densities are
    // the sums of node_density.  The node's own density and force-free moments from one read of its
    // populations, then the densities of the halo ring
    const int x = t.y + threadIdx.x, y = t.z + threadIdx.y;
    const int cx = threadIdx.x + HALO, cy = threadIdx.y + HALO;
    const size_t c = (size_t)y * G.pitch + x;
    // the node's own populations stay in the box: collide_site reads them there
    const float *own = pop + cy * W + cx + 2;
    float fk[2][9], Rn[2];
    NodeMoments nm;
    {
        float2 v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = make_float2(own[i * H * W], own[(9 + i) * H * W]);
        const float2 R2 = make_float2(ref[cy * W + cx + 2], ref[(H + cy) * W + cx + 2]);
        const float2 rn = vadd(R2, vzeroth<float2>(v));
        Rn[0] = R2.x;
        Rn[1] = R2.y;
        G.rho[parity ^ 1][c] = rn.x;
        G.rho[parity ^ 1][G.plane + c] = rn.y;
        sm.sr[cy][cx] = rn;
        sm.sp[cy][cx] = make_float2(psi_of<float>(rn.x), psi_of<float>(rn.y));
        node_moments(v, rn, R2, nm);
    }
    // both species' densities of a ring slot
    auto slot_density = [&](int sx, int sy) {
        float2 v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i)
            v[i] = make_float2(pop[(i * H + sy) * W + sx + 2], pop[((9 + i) * H + sy) * W + sx + 2]);
        return vadd(make_float2(ref[sy * W + sx + 2], ref[(H + sy) * W + sx + 2]), vzeroth<float2>(v));
    };
    constexpr int kRing = 4 * SW + 4 * TYv;
    for (int h = tid; h < kRing; h += TX * TYv) {
        int sx, sy;
        ring_slot<TYv>(h, sx, sy);
        if (slot_outside(G, t, sx, sy)) continue;
        const float2 r = slot_density(sx, sy);
        sm.sr[sy][sx] = r;
        sm.sp[sy][sx] = make_float2(psi_of<float>(r.x), psi_of<float>(r.y));
    }
    __syncthreads();
    const bool inner = t.y >= 1 && t.y + TX + 1 <= sm.L.nx && t.z >= 1 && t.z + TYv + 1 <= sm.L.ny;
    const PairStage<SHv> sg{sm.sr, sm.sp};
    if (inner) collide_site<float, true, true>(sm.L, G.f[parity ^ 1], sg, fk, Rn, x, y, cx, cy, own, H * W, &nm);
    else collide_site<float, false, true>(sm.L, G.f[parity ^ 1], sg, fk, Rn, x, y, cx, cy, own, H * W, &nm);
}

// One block per tile: thread 0 starts the two copies, every thread waits
// (bounded) on the mbarrier, then the tile is computed from the box.  A tile
// box_tile rejects is a caller error: it sets *err = 2 and is skipped.
template <int TYv>
__global__ void __launch_bounds__(TX *TYv, kTmaMinBlocks<TYv>)
    k_fused_tma(const Lat<float> *__restrict__ lats, const int4 *__restrict__ tiles, int tile_offset, int parity,
                const TmaMaps *__restrict__ maps, int *err, long long wait_cycles, int drop_tile, int n_tiles,
                int ahead, int wave)
{
    using B = TmaBox<TYv>;
    constexpr int ti = TYv == 2 ? 0 : (TYv == 4 ? 1 : 2);
    extern __shared__ __align__(128) float box[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ PairSmem<TYv> sm;
    // the tile is full and its lattice holds a whole box (so its maps exist):
    // the host marked it so when it sorted the list (tma_box_tile), which
    // keeps the lattice's descriptor off the way to the copy.  A tile without
    // the mark starts no copy and no load and leaves with *err = 2 where a
    // failed wait would (block-uniform, no early branch in the prologue)
    const int4 t = tiles[tile_offset + blockIdx.x];
    const bool good = t.w == kTmaBoxMark;
    const int tid = threadIdx.y * TX + threadIdx.x;
    // the boxes of the tile `ahead` blocks later (about one wave of resident
    // blocks) into L2, so that its copies find them there; a block of the
    // first wave issues it once its own box has landed, so that it does not
    // compete with the first wave's own copies
    const bool first_wave = (int)blockIdx.x < wave;
    auto prefetch_ahead = [&]() {
        if (ahead > 0 && (int)blockIdx.x + ahead < n_tiles) {
            const int4 tn = tiles[tile_offset + blockIdx.x + ahead];
            tma_prefetch_3d(&maps[tn.x].pop[ti][parity], tn.y - 4, tn.z - HALO, 0);
            tma_prefetch_3d(&maps[tn.x].ref[ti][parity], tn.y - 4, tn.z - HALO, 0);
        }
    };
    // the copy of drop_tile (a test hook) is never started: its wait runs out
    const bool issued = good && tile_offset + (int)blockIdx.x != drop_tile;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (issued) {
            mbar_expect_tx(&bar, B::kBytes);
            tma_load_3d(box, &maps[t.x].pop[ti][parity], t.y - 4, t.z - HALO, 0, &bar);
            tma_load_3d(box + B::kPop, &maps[t.x].ref[ti][parity], t.y - 4, t.z - HALO, 0, &bar);
        }
        if (good && !first_wave) prefetch_ahead();
    }
    // halo slots beyond the lattice load their nodes directly (wrapped, or
    // wall ghost rows): done while the copy is in flight
    {
        const Lat<float> &G = lats[t.x];
        if (good && (t.y == 0 || t.y + TX + HALO > G.nx || t.z < HALO || t.z + TYv + HALO > G.ny)) {
            constexpr int kRing = 4 * SW + 4 * TYv;
            for (int h = tid; h < kRing; h += TX * TYv) {
                int sx, sy;
                ring_slot<TYv>(h, sx, sy);
                if (slot_outside(G, t, sx, sy)) {
                    float rA, rB;
                    slot_densities<float, false>(G, t, parity, sx, sy, rA, rB);
                    sm.sr[sy][sx] = make_float2(rA, rB);
                    sm.sp[sy][sx] = make_float2(psi_of<float>(rA), psi_of<float>(rB));
                }
            }
        }
    }
    __syncthreads();   // the barrier is initialised before anyone waits on it
    const bool ok = good && mbar_wait(&bar, 0, wait_cycles);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            atomicExch(err, good ? 1 : 2);
            // let a copy still in flight land before the block ends (bounded
            // too, by at least 2^31 clocks, ~1 s)
            if (issued) mbar_wait(&bar, 0, wait_cycles > (1ll << 31) ? wait_cycles : (1ll << 31));
        }
        return;
    }
    if (tid == 0 && first_wave) prefetch_ahead();
    fused_tile_box<TYv>(lats, t, parity, sm, box, box + B::kPop);
}

// Distance, in quarters of a wave of resident blocks, between a tile and the
// tile whose boxes it prefetches into L2 (0: none).  Half a wave to a wave
// measured alike (a 4096^2 step 3 % shorter than without the prefetch);
// beyond it the boxes are prefetched too early.
constexpr int kPrefetchQuarterWaves = 3;

template <int TYv>
struct TmaKernel {
    static constexpr size_t kSmem = TmaBox<TYv>::kBytes;
    static int grid_wave;   // resident blocks on the device
    static cudaError_t prepare()
    {
        cudaError_t e = cudaFuncSetAttribute(k_fused_tma<TYv>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        int dev = 0, sms = 0, occ = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_tma<TYv>, TX * TYv, kSmem);
        if (e == cudaSuccess) grid_wave = sms * occ;
        return e;
    }
    static cudaError_t launch(const Lat<float> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                              const TmaMaps *maps, int *err, long long wait_cycles, int drop_tile, cudaStream_t s)
    {
        k_fused_tma<TYv><<<n_tiles, dim3(TX, TYv), kSmem, s>>>(lats, tiles, tile_offset, parity, maps, err, wait_cycles,
                                                               drop_tile, n_tiles,
                                                               kPrefetchQuarterWaves * grid_wave / 4, grid_wave);
        return cudaGetLastError();
    }
};
template <int TYv>
int TmaKernel<TYv>::grid_wave = 0;

}  // namespace

cudaError_t prepare_fused_tma()
{
    cudaError_t e = TmaKernel<2>::prepare();
    if (e == cudaSuccess) e = TmaKernel<4>::prepare();
    if (e == cudaSuccess) e = TmaKernel<8>::prepare();
    return e;
}

cudaError_t launch_fused_tma(const Lat<float> *lats, const int4 *tiles, int tile_offset, int n_tiles, int parity,
                             const TmaMaps *maps, int *err, long long wait_cycles, int drop_tile, int ty, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    switch (ty) {
    case 2: return TmaKernel<2>::launch(lats, tiles, tile_offset, n_tiles, parity, maps, err, wait_cycles, drop_tile, s);
    case 4: return TmaKernel<4>::launch(lats, tiles, tile_offset, n_tiles, parity, maps, err, wait_cycles, drop_tile, s);
    case 8: return TmaKernel<8>::launch(lats, tiles, tile_offset, n_tiles, parity, maps, err, wait_cycles, drop_tile, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbk

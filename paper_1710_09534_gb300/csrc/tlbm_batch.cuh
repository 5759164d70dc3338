// Batched execution: many lattices of different sizes advanced together.
//
// Each member lattice is described on the device by a LatDesc (its buffers,
// geometry, parameters and row-segment length).  One step of the batch is
//   k_batch_interior: a persistent kernel whose blocks take tiles (member,
//                     strip, segment) from a shared counter until the tile
//                     list is exhausted, running the same tile code as the
//                     single-lattice fused kernel;
//   k_batch_wall:     a grid-stride loop over the concatenated near-wall
//                     lists of all members.
// Tile and wall counts live in device memory, so one captured CUDA graph of a
// pair of steps stays valid when the membership changes.
#pragma once
#include "tlbm_kernels.cuh"

namespace tlb {

template <typename R>
struct LatDesc {
    const void* buf[2];  // distribution buffers; steps of parity p read buf[p], write buf[p ^ 1]
    void* cu;
    const uint8_t* cls;
    Geo g;
    Prm<R> P;
    int rows;  // row-segment length of this member's tiles
};

struct TileItem {
    int lat, bx, by;
};

struct WallItem {
    int lat;
    uint32_t packed;  // (y << 16) | x
};

struct BatchCounters {
    int n_tiles, n_wall;
    int next[2];  // tile counters of the two step parities (reset before each launch)
};

template <typename S, typename R, int BLOCK, bool PREFETCH, int MINB, bool MRT>
__global__ void __launch_bounds__(BLOCK, MINB)
k_batch_interior(const LatDesc<R>* __restrict__ descs, const TileItem* __restrict__ items,
                 BatchCounters* __restrict__ ctr, int parity)
{
    __shared__ ColRings<R, BLOCK> sh;
    constexpr bool kStash = kStashPops && std::is_same<R, float>::value && !MRT;
    __shared__ PopStash<R, kStash ? BLOCK : 1> stash;
    __shared__ Prm<R> Ps;
    __shared__ int item_s;
    static_assert(sizeof(Prm<R>) % sizeof(R) == 0, "params are whole words");
    constexpr int kWords = (int)(sizeof(Prm<R>) / sizeof(R));
    const int n = ctr->n_tiles;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(&ctr->next[parity], 1);
        __syncthreads();
        const int it = item_s;
        if (it >= n) break;
        const TileItem ti = items[it];
        const LatDesc<R>* d = descs + ti.lat;
        for (int i = threadIdx.x; i < kWords; i += BLOCK)
            reinterpret_cast<R*>(&Ps)[i] = reinterpret_cast<const R*>(&d->P)[i];
        __syncthreads();
        const Geo g = d->g;
        // members with equal densities and viscosities take the uniform-property
        // update, as they do when stepped alone (the branch is uniform per tile)
        auto* st = reinterpret_cast<PopStash<R, BLOCK>*>(&stash);  // used only when kStash
        if (Ps.uni != R(0))
            interior_tile<S, R, BLOCK, PREFETCH, MRT, true, kStash>((const S*)d->buf[parity], (S*)d->buf[parity ^ 1],
                                                                    (CuT<S>*)d->cu, d->cls, g, Ps, ti.bx, ti.by,
                                                                    d->rows, sh, st);
        else
            interior_tile<S, R, BLOCK, PREFETCH, MRT, false, kStash>((const S*)d->buf[parity], (S*)d->buf[parity ^ 1],
                                                                     (CuT<S>*)d->cu, d->cls, g, Ps, ti.bx, ti.by,
                                                                     d->rows, sh, st);
        __syncthreads();  // rings, parameters and item_s are reused by the next tile
    }
}

template <typename S, typename R, bool MRT>
__global__ void __launch_bounds__(128)
k_batch_wall(const LatDesc<R>* __restrict__ descs, const WallItem* __restrict__ items,
             const BatchCounters* __restrict__ ctr, int parity)
{
    const int n = ctr->n_wall;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const WallItem wi = items[i];
        const LatDesc<R>* d = descs + wi.lat;
        wall_node<S, R, MRT>((const S*)d->buf[parity], (S*)d->buf[parity ^ 1], (CuT<S>*)d->cu, d->cls, d->g, d->P,
                        wi.packed);
    }
}

}  // namespace tlb

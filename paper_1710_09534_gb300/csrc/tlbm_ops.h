// Host-side launch table of one storage precision (internal to the library).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include "tlbm_device.cuh"

namespace tlb {

struct Ops {
    size_t elem;     // bytes per stored distribution scalar
    int ndist;       // planes of `elem` bytes per distribution buffer
    size_t cu_elem;  // bytes per scalar of the c_i u planes
    // one time step A -> B = interior tiles (fused kernel) + near-wall list
    cudaError_t (*interior)(const void* fA, void* fB, void* cu, const uint8_t* cls, const Geo& g,
                            const Prm<double>& P, cudaStream_t s);
    cudaError_t (*wall)(const void* fA, void* fB, void* cu, const uint8_t* cls, const uint32_t* list,
                        int nlist, const Geo& g, const Prm<double>& P, cudaStream_t s);
    cudaError_t (*init)(void* fA, void* cu, const uint8_t* cls, const double* c1, const double* c2,
                        const double* ux, const double* uy, const double* p, const Geo& g,
                        const Prm<double>& P, cudaStream_t s);
    cudaError_t (*read)(const void* fA, const uint8_t* cls, double* out, uint32_t mask, const Geo& g,
                        const Prm<double>& P, cudaStream_t s);
    // contact-line diagnostic of component comp on the wall row (FP64):
    // wallc[nx], colh[nx] scratch, out[4*max_drops], *count
    cudaError_t (*contact)(const void* fA, const uint8_t* cls, int comp, double* wallc, double* colh,
                           double* out, int max_drops, int* count, const Geo& g, cudaStream_t s);
    // film thickness above solid node (x, y_top) of the order-parameter sum
    // selected by comps (FP64), into *out
    cudaError_t (*film)(const void* fA, const uint8_t* cls, int x, int y_top, int comps, double* out, const Geo& g,
                        cudaStream_t s);
    // batched step: persistent interior kernel (variant 0: 64-thread blocks,
    // 1: 128-thread blocks) over the tile list on s, the near-wall loop on ws
    // (the caller orders ws after the previous step and s's next step after ws)
    cudaError_t (*batch_step)(const void* descs, const void* tiles, const void* walls, void* ctr, int parity,
                              int variant, int grid_interior, int grid_wall, cudaStream_t s, cudaStream_t ws);
    // resident blocks per SM of the persistent interior kernel of a variant
    int (*batch_blocks_per_sm)(int variant);
    size_t desc_size;  // bytes of one device lattice descriptor
    void (*fill_desc)(void* dst, const void* buf0, const void* buf1, void* cu, const uint8_t* cls, const Geo& g,
                      const Prm<double>& P, int rows);
    // FP64 mass totals into out[4] via nparts block partials in part[4*nparts]
    cudaError_t (*mass)(const void* fA, const uint8_t* cls, double* part, int nparts, double* out,
                        const Geo& g, cudaStream_t s);
    // set-up of rows y0 .. y1-1 from dense FP64 rows (see k_init)
    cudaError_t (*init_rows)(void* fA, void* cu, const uint8_t* cls, const double* c1, const double* c2,
                             const double* ux, const double* uy, const double* p, const Geo& g,
                             const Prm<double>& P, int y0, int y1, int y_b, int rows, cudaStream_t s);
    // In-place (AA-pattern) step of parity odd = 0/1 on the one buffer f:
    // csum_ip writes c_1, c_2 into the planes cpl (2 planes of relem bytes),
    // interior_ip the fused interior update, wall_ip the lid nodes (lid = 1)
    // or the other near-wall nodes (lid = 0); swap_ip streams the layout an
    // even step leaves into the usual one.
    size_t relem;
    cudaError_t (*csum_ip)(const void* f, void* cpl, const uint8_t* cls, const Geo& g, int odd, cudaStream_t s);
    cudaError_t (*interior_ip)(void* f, void* cu, const void* cpl, const uint8_t* cls, const Geo& g,
                               const Prm<double>& P, int odd, cudaStream_t s);
    cudaError_t (*wall_ip)(void* f, void* cu, const void* cpl, const uint8_t* cls, const uint32_t* list, int nlist,
                           const Geo& g, const Prm<double>& P, int odd, int lid, cudaStream_t s);
    cudaError_t (*swap_ip)(void* f, const uint8_t* cls, const Geo& g, cudaStream_t s);
};

// Storage precisions (the TLB_FP64 .. TLB_BF16 values of the C ABI):
// bytes per distribution scalar, planes of that size per buffer, bytes per
// c_i u scalar.
inline size_t elem_for(int precision) { return precision == 0 ? 8 : (precision == 1 ? 4 : 2); }
inline int ndist_for(int precision) { return precision == 0 ? 27 : (precision == 1 ? 29 : 33); }
inline size_t cu_elem_for(int precision) { return precision == 0 ? 8 : 4; }

const Ops& ops_f64();
const Ops& ops_f32();
const Ops& ops_f16();
const Ops& ops_bf16();
const Ops& ops_f64_mrt();
const Ops& ops_f32_mrt();
const Ops& ops_f16_mrt();
const Ops& ops_bf16_mrt();

// launch table of a storage precision and collision model
inline const Ops& ops_for(int precision, bool mrt)
{
    switch (precision) {
    case 0: return mrt ? ops_f64_mrt() : ops_f64();
    case 1: return mrt ? ops_f32_mrt() : ops_f32();
    case 2: return mrt ? ops_f16_mrt() : ops_f16();
    default: return mrt ? ops_bf16_mrt() : ops_bf16();
    }
}

// Fused interior kernel: threads per block (one column each, 4 of them halo)
// and rows marched per block, per precision.
#ifndef TLB_BLOCK64
#define TLB_BLOCK64 128
#endif
#ifndef TLB_ROWS64
#define TLB_ROWS64 16
#endif
#ifndef TLB_BLOCK32
#define TLB_BLOCK32 128
#endif
#ifndef TLB_ROWS32
#define TLB_ROWS32 16
#endif
#ifndef TLB_MINB64
#define TLB_MINB64 3
#endif
#ifndef TLB_MINB32
#define TLB_MINB32 5
#endif
#ifndef TLB_PREFETCH32
#define TLB_PREFETCH32 1
#endif
// the FP32-arithmetic MRT update keeps two 9-moment vectors per distribution
// live: at 5 blocks per SM (96 registers) it spills, at 4 (128) it does not
#ifndef TLB_MINB32_MRT
#define TLB_MINB32_MRT 4
#endif
constexpr int kBlock64 = TLB_BLOCK64, kRows64 = TLB_ROWS64, kMinB64 = TLB_MINB64;
// FP32 storage with the one-row-ahead population loads holds about 20 more
// registers per thread: 4 blocks per SM
#ifndef TLB_MINB_F32
#define TLB_MINB_F32 4
#endif
constexpr int kBlock32 = TLB_BLOCK32, kRows32 = TLB_ROWS32, kMinB32 = TLB_MINB32, kMinB32Mrt = TLB_MINB32_MRT;
constexpr int kMinBF32 = TLB_MINB_F32;
constexpr bool kPrefetch32 = TLB_PREFETCH32 != 0;


}  // namespace tlb

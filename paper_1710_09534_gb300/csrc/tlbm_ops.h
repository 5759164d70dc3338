// Host-side launch table of one storage precision (internal to the library).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include "tlbm_device.cuh"

namespace tlb {

struct Ops {
    size_t elem;  // bytes per stored scalar
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
    // FP64 mass totals into out[4] via nparts block partials in part[4*nparts]
    cudaError_t (*mass)(const void* fA, const uint8_t* cls, double* part, int nparts, double* out,
                        const Geo& g, cudaStream_t s);
};

const Ops& ops_f64();
const Ops& ops_f32();

// Fused interior kernel: threads per block (one column each, 4 of them halo)
// and rows marched per block, per precision.
constexpr int kBlock64 = 64, kRows64 = 64;
constexpr int kBlock32 = 64, kRows32 = 64;

}  // namespace tlb

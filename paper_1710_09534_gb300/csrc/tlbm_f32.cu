// FP32 storage, FP32 arithmetic.
#include "tlbm_ops_impl.cuh"

namespace tlb {
const Ops& ops_f32() { return OpsImpl<float, float, kTileX32, kTileY32>::table(); }
}  // namespace tlb

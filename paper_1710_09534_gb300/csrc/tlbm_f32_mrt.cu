// FP32 storage, FP32 arithmetic, MRT collision.
#include "tlbm_ops_impl.cuh"

namespace tlb {
const Ops& ops_f32_mrt() { return OpsImpl<float, float, kBlock32, kRows32, kPrefetch32, kMinB32Mrt, true>::table(); }
}  // namespace tlb

// FP16 storage (shifted, scaled), FP32 arithmetic, MRT collision.
#include "tlbm_ops_impl.cuh"

namespace tlb {
const Ops& ops_f16_mrt() { return OpsImpl<__half, float, kBlock32, kRows32, kPrefetch32, kMinB32Mrt, true>::table(); }
}  // namespace tlb

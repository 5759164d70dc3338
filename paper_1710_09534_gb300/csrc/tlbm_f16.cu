// FP16 storage (shifted, scaled), FP32 arithmetic, BGK collision.
#include "tlbm_ops_impl.cuh"

namespace tlb {
const Ops& ops_f16() { return OpsImpl<__half, float, kBlock32, kRows32, kPrefetch32, kMinB32, false>::table(); }
}  // namespace tlb

// BF16 storage (shifted), FP32 arithmetic, MRT collision.
#include "tlbm_ops_impl.cuh"

namespace tlb {
const Ops& ops_bf16_mrt() { return OpsImpl<__nv_bfloat16, float, kBlock32, kRows32, kPrefetch32, kMinB32Mrt, true>::table(); }
}  // namespace tlb

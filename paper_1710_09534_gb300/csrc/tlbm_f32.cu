// FP32 storage, FP32 arithmetic, BGK collision.
#include "tlbm_ops_impl.cuh"

namespace tlb {
const Ops& ops_f32() { return OpsImpl<float, float, kBlock32, kRows32, kPrefetch32, kMinBF32, false>::table(); }
}  // namespace tlb

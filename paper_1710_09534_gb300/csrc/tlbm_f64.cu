// FP64 storage, FP64 arithmetic.
#include "tlbm_ops_impl.cuh"

namespace tlb {
const Ops& ops_f64() { return OpsImpl<double, double, kTileX64, kTileY64>::table(); }
}  // namespace tlb

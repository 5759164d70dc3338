// FP64 storage, FP64 arithmetic, MRT collision.
#include "tlbm_ops_impl.cuh"

namespace tlb {
const Ops& ops_f64_mrt() { return OpsImpl<double, double, kBlock64, kRows64, false, kMinB64, true>::table(); }
}  // namespace tlb

// FP64 storage, FP64 arithmetic, BGK collision.
#include "tlbm_ops_impl.cuh"

namespace tlb {
const Ops& ops_f64() { return OpsImpl<double, double, kBlock64, kRows64, false, kMinB64, false>::table(); }
}  // namespace tlb

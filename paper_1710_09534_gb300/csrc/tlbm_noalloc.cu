// tlb_diagnostics_noalloc: the FP64 mass/non-finite reduction of
// tlb_diagnostics, for callers that cannot allocate device memory at the
// point where they need it -- for example code that runs inside a fixed
// memory arena it does not own, or a real-time loop that must not pay for
// (or synchronize on) an allocation.  It reads the lattice state from the
// caller's workspace, writes the result to a caller-provided device buffer,
// and keeps its block partial sums in a fixed static device array instead of
// any allocated scratch.  It calls no cudaMalloc/cudaFree and no allocating
// library routine.
#include <cstdio>
#include <mutex>

#include "tlbm.h"
#include "tlbm_internal.h"
#include "tlbm_ops.h"

namespace {

// One partial row (4 doubles) per block of kNodesPerPart nodes.
constexpr long long kNodesPerPart = 16384;
constexpr int kMaxParts = 1024;  // 1024 rows x 4 doubles = 32 KiB of scratch
constexpr long long kMaxNodes = kNodesPerPart * kMaxParts;  // 16,777,216 nodes (4096^2)

// Shared by every call on a device and kept until the process exits; each
// call overwrites the rows it reads, so nothing has to start at zero.
static __device__ __align__(256) double g_partials[kMaxParts * 4];

std::mutex g_mu;
double* g_addr[256] = {};  // device address of g_partials, per device ordinal

// Device address of g_partials on `device` (which must be current).  The
// host-side symbol is only a stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress.
int scratch_address(int device, double** out)
{
    if (device < 0 || device >= 256) return tlb::set_error(TLB_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the static scratch failed: %s",
                     cudaGetErrorString(e));
            return tlb::set_error(TLB_ECUDA, msg);
        }
        g_addr[device] = (double*)p;
    }
    *out = g_addr[device];
    return TLB_OK;
}

}  // namespace

extern "C" int tlb_diagnostics_noalloc(tlb_lattice* lat, double* dev_out)
{
    tlb::LatticeView v;
    int rc = tlb::lattice_view(lat, &v);
    if (rc) return rc;
    if (!dev_out) return tlb::set_error(TLB_EINVAL, "dev_out is null");
    const long long n = (long long)v.geo.nx * v.geo.ny;
    if (n > kMaxNodes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "lattice of %lld nodes exceeds the %lld-node limit of the static scratch "
                 "(use tlb_diagnostics)", n, kMaxNodes);
        return tlb::set_error(TLB_EINVAL, msg);
    }
    double* part = nullptr;
    if ((rc = scratch_address(v.device, &part))) return rc;
    const int nparts = (int)((n + kNodesPerPart - 1) / kNodesPerPart);
    // the lattice's own reduction kernels (partials, then the fixed-order final sum)
    const cudaError_t e = v.ops->mass(v.dist, v.cls, part, nparts, dev_out, v.geo, v.stream);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "launch failed: %s", cudaGetErrorString(e));
        return tlb::set_error(TLB_ECUDA, msg);
    }
    return tlb::clear_error();
}

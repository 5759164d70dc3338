// Internal accessors shared between the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <vector>
#include "tlbm.h"
#include "tlbm_device.cuh"
#include "tlbm_ops.h"

namespace tlb {

// Byte offsets of the regions of one lattice's workspace.
struct Layout {
    int pitch = 0;
    int64_t plane = 0;  // elements
    int64_t fA = 0, fB = 0, cu = 0, cls = 0, list = 0, part = 0, diag = 0, contact = 0, total = 0;
    bool inplace = false;  // one distribution buffer (fB unused) and the order-parameter planes cpl
    int64_t cpl = 0, cpl_bytes = 0;
};

}  // namespace tlb

// Host handle of one lattice (opaque to callers).
struct tlb_lattice {
    int nx = 0, ny = 0, precision = 0, device = 0;
    int32_t edge[4] = {0, 0, 0, 0};
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    // The near-wall kernel of a step runs on `side`, concurrently with the
    // interior kernel on `stream` (they read the same state and write disjoint
    // (node, slot) pairs): `fork` orders it after the previous step, `join`
    // orders the next step after it.
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    char* ws = nullptr;
    tlb::Layout lay;
    const tlb::Ops* ops = nullptr;
    tlb::Geo geo{};
    tlb::Prm<double> prm{};
    int cur = 0;  // which of the two distribution buffers holds the state
    bool have_params = false, have_fields = false;
    std::vector<uint8_t> mask;    // host copy of the solid mask
    std::vector<uint8_t> cls;     // host copy of the node classes (pitched)
    int64_t nlist = 0;
    std::vector<uint32_t> hlist;  // host copy of the near-wall list
    tlb_batch* batch = nullptr;   // batch this lattice belongs to, if any
    // optional per-kernel timing: per step, events around the interior launch
    // (on `stream`) and around the near-wall launch (on `side`)
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    double prof_ms[2] = {0, 0};
    int64_t prof_n[2] = {0, 0};

    void* bufA() { return ws + (cur == 0 ? lay.fA : lay.fB); }
    void* bufB() { return lay.inplace ? nullptr : ws + (cur == 0 ? lay.fB : lay.fA); }
    void* cpl() { return ws + lay.cpl; }
    void* cu() { return ws + lay.cu; }
    const uint8_t* dcls() { return (const uint8_t*)(ws + lay.cls); }
    const uint32_t* dlist() { return (const uint32_t*)(ws + lay.list); }
    int64_t n() const { return (int64_t)nx * ny; }
};

namespace tlb {

// Read-only view of a lattice's current state inside the caller's workspace.
struct LatticeView {
    const void* dist;      // current distribution buffer
    const uint8_t* cls;    // node classes
    Geo geo;
    int precision;
    const Ops* ops;        // launch table of the lattice's precision
    int device;
    cudaStream_t stream;
};

// Fills *v (and makes the lattice's device current); TLB_E* code on failure.
int lattice_view(tlb_lattice* lat, LatticeView* v);

// A member lattice's geometry, parameters or buffers changed outside the
// batch: its descriptors and work lists must be rebuilt before the next step.
void batch_member_changed(tlb_batch* B);
// Wait for the batch stream (a member's own-stream calls must not overtake
// batch steps still queued on it); TLB_OK for a lattice outside any batch.
int batch_sync(tlb_batch* B);

// Record an error message for tlb_last_error() and return `code`.
int set_error(int code, const char* msg);
int clear_error();

}  // namespace tlb

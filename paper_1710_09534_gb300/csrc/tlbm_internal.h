// Internal accessors shared between the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include "tlbm.h"
#include "tlbm_device.cuh"

namespace tlb {

// Read-only view of a lattice's current state inside the caller's workspace.
struct LatticeView {
    const void* dist;      // current distribution buffer (27 planes)
    const uint8_t* cls;    // node classes
    Geo geo;
    int precision;
    int device;
    cudaStream_t stream;
};

// Fills *v (and makes the lattice's device current); TLB_E* code on failure.
int lattice_view(tlb_lattice* lat, LatticeView* v);

// Record an error message for tlb_last_error() and return `code`.
int set_error(int code, const char* msg);
int clear_error();

}  // namespace tlb

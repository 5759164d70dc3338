// Fused interior update with the order-parameter rows staged in shared memory
// by the bulk-copy engine (FP32 and 16-bit storage).
//
// The column-marching tile of k_step_interior needs, per iteration, the 18
// order-parameter populations (plus the rest populations' lo parts) of the row
// it enters, to sum c_1, c_2 (Eq. 13a), and two iterations later the same
// populations again for the collision of that row.  Here one thread of the
// block's first warp issues, kPrefetch iterations ahead, one cp.async.bulk copy
// per plane of the row segment (one lane per plane) into a ring of
// shared-memory slots, completing on an mbarrier per slot; the threads wait on the slot's phase and read the row
// from shared memory for both uses.  The loads leave the threads' critical
// path and their registers, and the DRAM traffic of a row is in flight while
// the rows before it are computed.
//
// Every wait is bounded: a wait that runs out sets *status (a device int the
// host reads), the block stops after its next barrier, and the producer thread
// waits (again bounded) for the copies it still has in flight before exiting.
#pragma once
#include "tlbm_kernels.cuh"

namespace tlb {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// one arrival that also announces `bytes` of transactions for the phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of `parity` to complete, giving up after ~2^20 polls
// (far beyond any copy's latency).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    for (int i = 0; i < (1 << 20); i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// order earlier generic-proxy accesses to shared memory before async-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory ring of staged rows.  A slot holds one row segment of NC
// columns starting at global column a0 (a multiple of 8):
//   FP32:   20 float planes: f^1_0..8, f^2_0..8, then the lo parts of f^1_0, f^2_0
//   16-bit: 16 16-bit planes f^1_1..8, f^2_1..8, then 4 float planes:
//           f^1_0 hi, f^2_0 hi, f^1_0 lo, f^2_0 lo
template <typename S, int BLOCK, int PF>
struct StagedRing {
    static constexpr bool k16 = Store<S>::k16;
    static constexpr int NC = BLOCK + 8;
    // Row j is issued after the first barrier of iteration j - PF, summed at
    // iteration j and read again by the update at j + 2; its slot is reissued
    // (for row j + kSlots) after the first barrier of iteration j + 3, when
    // every thread has finished the update of iteration j + 2.
    static constexpr int kSlots = PF + 3;
    static constexpr int kSlotBytes = k16 ? (16 * NC * 2 + 4 * NC * 4) : (20 * NC * 4);
    static constexpr int kBytes = kSlots * kSlotBytes;
    static_assert(kSlotBytes % 16 == 0 && (16 * NC * 2) % 16 == 0, "16-byte aligned planes");
};

template <typename S, typename R, int BLOCK, int PF>
struct StagedRows {
    using Ring = StagedRing<S, BLOCK, PF>;
    static constexpr int NC = Ring::NC, kSlots = Ring::kSlots;
    const S* __restrict__ f;
    long long PL;
    unsigned char* slots;  // dynamic shared memory, kSlots * kSlotBytes
    uint64_t* bars;        // kSlots mbarriers
    int* abort_flag;       // shared
    int* status;           // device status word
    int pitch, ny, y0, y1, dir, iters, a0, col;  // col: this thread's staged column
    bool periodic_y;
    int issued = -1;  // last iteration whose row was issued (producer thread)

    __device__ __forceinline__ int row_of(int j) const { return dir > 0 ? y0 - 2 + j : y1 + 1 - j; }

    // producer (warp 0): stage the row that iteration j will sum; lane 0
    // arms the slot's barrier, then one lane per plane issues its copy
    __device__ __forceinline__ void issue(int j)
    {
        if (threadIdx.x >= 32 || j >= iters) return;
        const int lane = threadIdx.x;
        unsigned char* slot = slots + (j % kSlots) * Ring::kSlotBytes;
        uint64_t* bar = bars + (j % kSlots);
        int y = row_of(j);
        bool valid = true;
        if (y < 0 || y >= ny) {
            if (periodic_y) y = y < 0 ? y + ny : y - ny;
            else valid = false;
        }
        const int cs = a0 > 0 ? a0 : 0;
        const int ce = (a0 + NC < pitch) ? a0 + NC : pitch;
        const int ncol = ce - cs;
        if (lane == 0) {
            issued = j;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, valid ? (uint32_t)(ncol * (Ring::k16 ? 16 * 2 + 4 * 4 : 20 * 4)) : 0u);
        }
        __syncwarp();
        if (!valid || lane >= 20) return;
        fence_proxy_async_smem();
        const long long rowoff = (long long)y * pitch + cs;
        if constexpr (Ring::k16) {
            if (lane < 16) {
                const int q = lane < 8 ? lane + 1 : lane + 2;
                bulk_g2s(slot + (lane * NC + (cs - a0)) * 2,
                         reinterpret_cast<const unsigned short*>(f) + q * PL + rowoff, (uint32_t)(ncol * 2), bar);
            } else {
                const int j2 = lane - 16;
                bulk_g2s(slot + 32 * NC + (j2 * NC + (cs - a0)) * 4, rest_region(f, PL) + j2 * PL + rowoff,
                         (uint32_t)(ncol * 4), bar);
            }
        } else {
            const int q = lane < 18 ? lane : 27 + (lane - 18);
            bulk_g2s(slot + (lane * NC + (cs - a0)) * 4, f + q * PL + rowoff, (uint32_t)(ncol * 4), bar);
        }
    }

    __device__ __forceinline__ void prologue()
    {
        for (int j = 0; j < PF; j++) issue(j);
    }
    __device__ __forceinline__ void begin(int it) { issue(it + PF); }

    __device__ __forceinline__ const unsigned char* slot_of(int j) const
    {
        return slots + (j % kSlots) * Ring::kSlotBytes;
    }
    // population q (0..17) of this thread's column in the slot of iteration j
    __device__ __forceinline__ R spop(const unsigned char* slot, int q) const
    {
        if constexpr (Ring::k16) {
            if (q == 0 || q == 9)
                return R(reinterpret_cast<const float*>(slot + 32 * NC)[(q == 9 ? NC : 0) + col]);
            const int m = q < 9 ? q - 1 : q - 2;
            constexpr float inv = 1.0f / float(1 << Store<S>::kScaleExp);
            return R(dec16(S{}, reinterpret_cast<const unsigned short*>(slot)[m * NC + col]) * inv);
        } else {
            return R(reinterpret_cast<const float*>(slot)[q * NC + col]);
        }
    }
    __device__ __forceinline__ R slo(const unsigned char* slot, int i) const
    {
        if constexpr (Ring::k16) return R(reinterpret_cast<const float*>(slot + 32 * NC)[(2 + i) * NC + col]);
        else return R(reinterpret_cast<const float*>(slot)[(18 + i) * NC + col]);
    }

    // c_1, c_2 of the entered row at this thread's column (inside: not a
    // periodic image, so the column is in the staged segment)
    __device__ __forceinline__ void c_at(int it, long long o, bool inside, R& a, R& b)
    {
        if (!inside) {
            order_params<R>(f, PL, o, a, b);
            return;
        }
        if (!mbar_wait_bounded(bars + (it % kSlots), (uint32_t)((it / kSlots) & 1))) {
            atomicExch(status, 1);
            *abort_flag = 1;
        }
        const unsigned char* slot = slot_of(it);
        R v[18];
#pragma unroll
        for (int k = 0; k < 18; k++) v[k] = spop(slot, k);
        v[0] += slo(slot, 0);
        v[9] += slo(slot, 1);
        a = sum9(v);
        b = sum9(v + 9);
    }
    __device__ __forceinline__ bool aborted() const { return *abort_flag != 0; }

    // the updated row of iteration it was entered (and waited for) at it - 2
    template <int K>
    __device__ __forceinline__ void pop(int it, long long, R& f1k, R& f2k) const
    {
        const unsigned char* slot = slot_of(it - 2);
        f1k = spop(slot, K);
        f2k = spop(slot, 9 + K);
    }
    __device__ __forceinline__ void lo(int it, long long, R& l1, R& l2) const
    {
        const unsigned char* slot = slot_of(it - 2);
        l1 = slo(slot, 0);
        l2 = slo(slot, 1);
    }
    // after the loop: on an early stop (at iteration it, whose wait ran out),
    // drain the copies still in flight
    __device__ __forceinline__ void finish(int it)
    {
        if (threadIdx.x != 0) return;
        for (int j = it; j <= issued; j++)
            if (!mbar_wait_bounded(bars + (j % kSlots), (uint32_t)((j / kSlots) & 1))) atomicExch(status, 2);
    }
};

template <typename S, typename R, int BLOCK, int ROWS, int PF, int MINB, bool MRT>
__global__ void __launch_bounds__(BLOCK, MINB)
k_step_interior_staged(const S* __restrict__ fA, S* __restrict__ fB, CuT<S>* __restrict__ cu,
                       const uint8_t* __restrict__ cls, Geo g, Prm<R> P, int* __restrict__ status)
{
    using Ring = StagedRing<S, BLOCK, PF>;
    extern __shared__ __align__(128) unsigned char staged[];
    __shared__ TileRings<R, BLOCK> sh;
    __shared__ __align__(8) uint64_t bars[Ring::kSlots];
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        for (int s = 0; s < Ring::kSlots; s++) mbar_init(&bars[s], 1);
        abort_flag = 0;
        mbar_init_fence();
    }
    __syncthreads();
    const int bx = blockIdx.x, by = blockIdx.y;
    const int x0 = bx * (BLOCK - 4);
    const int y0 = by * ROWS;
    const int y1 = min(y0 + ROWS, g.ny);
    StagedRows<S, R, BLOCK, PF> src;
    src.f = fA;
    src.PL = g.plane;
    src.slots = staged;
    src.bars = bars;
    src.abort_flag = &abort_flag;
    src.status = status;
    src.pitch = g.pitch;
    src.ny = g.ny;
    src.y0 = y0;
    src.y1 = y1;
    src.dir = (by & 1) ? -1 : 1;
    src.iters = (y1 - y0) + 4;
    src.a0 = ((x0 - 2) >> 3) << 3;  // floor to a multiple of 8 (x0 - 2 >= -2)
    src.col = (x0 - 2 + (int)threadIdx.x) - src.a0;
    src.periodic_y = g.edge[2] == EDGE_PERIODIC;
    src.prologue();
    interior_tile<S, R, BLOCK, true, MRT>(fA, fB, cu, cls, g, P, bx, by, ROWS, sh, src);
}

}  // namespace tlb

// Launchers of one precision; included by tlbm_f64.cu and tlbm_f32.cu.
#pragma once
#include "tlbm_batch.cuh"
#include "tlbm_inplace.cuh"
#include "tlbm_kernels.cuh"
#include "tlbm_ops.h"

namespace tlb {

template <typename R>
inline Prm<R> cast_prm(const Prm<double>& d)
{
    Prm<R> r;
    for (int i = 0; i < 3; i++) {
        r.lam[i] = R(d.lam[i]);
        r.rho[i] = R(d.rho[i]);
        r.nu[i] = R(d.nu[i]);
    }
    for (int i = 0; i < 2; i++) {
        r.k34Dlam[i] = R(d.k34Dlam[i]);
        r.eta[i] = R(d.eta[i]);
        r.inv_tau[i] = R(d.inv_tau[i]);
        r.omt[i] = R(d.omt[i]);
        r.src_f[i] = R(d.src_f[i]);
        r.e0[i] = R(d.e0[i]);
        r.drho[i] = R(d.drho[i]);
        r.dnu[i] = R(d.dnu[i]);
        r.aM[i] = R(d.aM[i]);
        for (int c = 0; c < 2; c++) {
            r.aw[i][c] = R(d.aw[i][c]);
            r.bw[i][c] = R(d.bw[i][c]);
            r.sw[i][c] = R(d.sw[i][c]);
        }
    }
    r.lamT = R(d.lamT);
    r.two_lamT = R(d.two_lamT);
    r.k12D = R(d.k12D);
    r.k34D = R(d.k34D);
    r.k4D = R(d.k4D);
    r.l3_l1 = R(d.l3_l1);
    r.l3_l2 = R(d.l3_l2);
    r.cos12 = R(d.cos12);
    r.cos13 = R(d.cos13);
    r.cos23 = R(d.cos23);
    r.gx = R(d.gx);
    r.gy = R(d.gy);
    r.lid_u = R(d.lid_u);
    r.mrt = R(d.mrt);
    r.mrt_s_f = R(d.mrt_s_f);
    r.mrt_s_g = R(d.mrt_s_g);
    r.uni = R(d.uni);
    r.inv_rho3 = R(d.inv_rho3);
    r.inv_taug3 = R(d.inv_taug3);
    r.omtg3 = R(d.omtg3);
    r.kG3 = R(d.kG3);
    for (int c = 0; c < 2; c++) {
        r.Rw3[c] = R(d.Rw3[c]);
        r.Kw3[c] = R(d.Kw3[c]);
    }
    r.p3tg3 = R(d.p3tg3);
    r.rg3x = R(d.rg3x);
    r.rg3y = R(d.rg3y);
    for (int i = 0; i < 2; i++) {
        r.Kl[i] = R(d.Kl[i]);
        r.K34l6[i] = R(d.K34l6[i]);
        r.drho12[i] = R(d.drho12[i]);
        r.aM6[i] = R(d.aM6[i]);
        r.k3tau[i] = R(d.k3tau[i]);
        r.kq[i] = R(d.kq[i]);
        r.ks[i] = R(d.ks[i]);
        r.K3w3[i] = R(d.K3w3[i]);
        r.qa[i][0] = R(d.qa[i][0]);
        r.qa[i][1] = R(d.qa[i][1]);
    }
    r.Kt = R(d.Kt);
    return r;
}

// Streaming multiprocessors of the current device (queried once per process).
inline int sm_count()
{
    static int n = 0;
    if (n <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
    }
    return n;
}

// Row-segment length of a single-lattice interior launch: `rows`, halved (down
// to 4) while the grid would not fill every SM with `per_sm` resident blocks,
// so that a small lattice still spreads over the chip (the halo work per node
// grows, but idle SMs cost more).
#ifndef TLB_ADAPTIVE_ROWS
#define TLB_ADAPTIVE_ROWS 1
#endif
// one_wave (the FP64 two-buffer interior kernel): a lattice large enough for
// more than one wave of blocks gets segments long enough that the whole grid
// is resident at once, so that the halo rows' c sums and chemical potentials
// (FP64 arithmetic, the kernel's bound) are repeated on fewer rows.  GB300:
// FP64 2048^2 interior kernel 1.929 -> 1.911 ms, 1024x2048 cylinder impact
// within +-3%.  FP32 and 16-bit storage (latency-bound) lose the dynamic
// balancing of several waves: the cylinder impact ran 12% (FP32) and 10%
// (FP16) slower, so they keep short segments; the in-place kernels too.
#ifndef TLB_ONE_WAVE
#define TLB_ONE_WAVE 1
#endif
inline int rows_for(const Geo& g, int tx, int rows, int per_sm, bool one_wave = false)
{
    if (!TLB_ADAPTIVE_ROWS) return rows;
    const int strips = (g.nx + tx - 1) / tx;
    if (TLB_ONE_WAVE && one_wave) {
        const long long segs = (long long)sm_count() * per_sm / strips;
        if (segs >= 1) {
            const int r = (int)((g.ny + segs - 1) / segs);
            if (r > rows) return r;
        }
    }
    while (rows > 4 && (long long)strips * ((g.ny + rows - 1) / rows) < (long long)sm_count() * per_sm) rows /= 2;
    return rows;
}

// Resident blocks per SM of the FP64 BGK uniform-property interior kernel,
// which needs fewer registers than the general one: at 4 (128 registers, no
// spills) it measured slower than at 3 (GB300, 2048^2: 1.913 -> 1.947 ms).
#ifndef TLB_MINB64_UNI
#define TLB_MINB64_UNI 3
#endif

template <typename S, typename R, int BLOCK, int ROWS, bool PREFETCH, int MINB, bool MRT>
struct OpsImpl {
    static constexpr int kMinBUni = std::is_same<R, double>::value && !MRT ? TLB_MINB64_UNI : MINB;
    static cudaError_t interior(const void* fA, void* fB, void* cu, const uint8_t* cls, const Geo& g,
                                const Prm<double>& Pd, cudaStream_t s)
    {
        const Prm<R> P = cast_prm<R>(Pd);
        constexpr int TX = BLOCK - 4;
        constexpr bool kOneWave = std::is_same<R, double>::value;
        // equal densities and viscosities: the uniform-property update
        if (Pd.uni != 0.0) {
            const int rows = rows_for(g, TX, ROWS, kMinBUni, kOneWave);
            dim3 grid((g.nx + TX - 1) / TX, (g.ny + rows - 1) / rows);
            k_step_interior<S, R, BLOCK, ROWS, PREFETCH, kMinBUni, MRT, true><<<grid, BLOCK, 0, s>>>(
                (const S*)fA, (S*)fB, (CuT<S>*)cu, cls, g, P, rows);
        } else {
            const int rows = rows_for(g, TX, ROWS, MINB, kOneWave);
            dim3 grid((g.nx + TX - 1) / TX, (g.ny + rows - 1) / rows);
            k_step_interior<S, R, BLOCK, ROWS, PREFETCH, MINB, MRT, false><<<grid, BLOCK, 0, s>>>(
                (const S*)fA, (S*)fB, (CuT<S>*)cu, cls, g, P, rows);
        }
        return cudaGetLastError();
    }
    static cudaError_t wall(const void* fA, void* fB, void* cu, const uint8_t* cls, const uint32_t* list,
                            int nlist, const Geo& g, const Prm<double>& Pd, cudaStream_t s)
    {
        const Prm<R> P = cast_prm<R>(Pd);
        if (nlist > 0)
            k_step_wall<S, R, MRT><<<(nlist + 127) / 128, 128, 0, s>>>((const S*)fA, (S*)fB, (CuT<S>*)cu, cls, list,
                                                                   nlist, g, P);
        return cudaGetLastError();
    }
    static cudaError_t init(void* fA, void* cu, const uint8_t* cls, const double* c1, const double* c2,
                            const double* ux, const double* uy, const double* p, const Geo& g,
                            const Prm<double>& Pd, cudaStream_t s)
    {
        const Prm<R> P = cast_prm<R>(Pd);
        dim3 grid((g.nx + 127) / 128, g.ny);
        k_init<S, R><<<grid, 128, 0, s>>>((S*)fA, (CuT<S>*)cu, cls, c1, c2, ux, uy, p, g, P, 0, 0, g.ny);
        return cudaGetLastError();
    }
    static cudaError_t read(const void* fA, const uint8_t* cls, double* out, uint32_t mask, const Geo& g,
                            const Prm<double>& Pd, cudaStream_t s)
    {
        const Prm<R> P = cast_prm<R>(Pd);
        dim3 grid((g.nx + 127) / 128, g.ny);
        k_read_fields<S, R><<<grid, 128, 0, s>>>((const S*)fA, cls, out, mask, g, P);
        return cudaGetLastError();
    }
    static cudaError_t mass(const void* fA, const uint8_t* cls, double* part, int nparts, double* out,
                            const Geo& g, cudaStream_t s)
    {
        k_mass_partials<S, R><<<nparts, 256, 0, s>>>((const S*)fA, cls, part, g);
        k_mass_final<<<1, 256, 0, s>>>(part, nparts, out);
        return cudaGetLastError();
    }
    static cudaError_t contact(const void* fA, const uint8_t* cls, int comp, double* wallc, double* colh,
                               double* out, int max_drops, int* count, const Geo& g, cudaStream_t s)
    {
        k_contact_columns<S><<<(g.nx + 127) / 128, 128, 0, s>>>((const S*)fA, cls, comp, wallc, colh, g);
        k_contact_scan<<<1, 32, 0, s>>>(wallc, colh, g.nx, out, max_drops, count);
        return cudaGetLastError();
    }
    static cudaError_t film(const void* fA, const uint8_t* cls, int x, int y_top, int comps, double* out,
                            const Geo& g, cudaStream_t s)
    {
        k_film<S><<<1, 32, 0, s>>>((const S*)fA, cls, x, y_top, comps, out, g);
        return cudaGetLastError();
    }
    // the two block shapes the batch tuner chooses between
    static constexpr int kMinB64 = std::is_same<R, float>::value ? 8 : 6;
    static cudaError_t batch_step(const void* descs, const void* tiles, const void* walls, void* ctr, int parity,
                                  int variant, int grid_interior, int grid_wall, cudaStream_t s, cudaStream_t ws)
    {
        BatchCounters* c = (BatchCounters*)ctr;
        cudaError_t e = cudaMemsetAsync(&c->next[parity], 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        if (variant == 0)
            k_batch_interior<S, R, 64, PREFETCH, kMinB64, MRT><<<grid_interior, 64, 0, s>>>(
                (const LatDesc<R>*)descs, (const TileItem*)tiles, c, parity);
        else
            k_batch_interior<S, R, 128, PREFETCH, MINB, MRT><<<grid_interior, 128, 0, s>>>(
                (const LatDesc<R>*)descs, (const TileItem*)tiles, c, parity);
        k_batch_wall<S, R, MRT><<<grid_wall, 128, 0, ws>>>((const LatDesc<R>*)descs, (const WallItem*)walls, c, parity);
        return cudaGetLastError();
    }
    static int batch_blocks_per_sm(int variant)
    {
        int n = 0;
        if (variant == 0)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_interior<S, R, 64, PREFETCH, kMinB64, MRT>, 64, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_interior<S, R, 128, PREFETCH, MINB, MRT>, 128, 0);
        return n;
    }
    static void fill_desc(void* dst, const void* buf0, const void* buf1, void* cu, const uint8_t* cls, const Geo& g,
                          const Prm<double>& P, int rows)
    {
        LatDesc<R>* d = (LatDesc<R>*)dst;
        d->buf[0] = buf0;
        d->buf[1] = buf1;
        d->cu = cu;
        d->cls = cls;
        d->g = g;
        d->P = cast_prm<R>(P);
        d->rows = rows;
    }
    static cudaError_t init_rows(void* fA, void* cu, const uint8_t* cls, const double* c1, const double* c2,
                                 const double* ux, const double* uy, const double* p, const Geo& g,
                                 const Prm<double>& Pd, int y0, int y1, int y_b, int rows, cudaStream_t s)
    {
        const Prm<R> P = cast_prm<R>(Pd);
        if (y1 <= y0) return cudaSuccess;
        dim3 grid((g.nx + 127) / 128, y1 - y0);
        k_init<S, R><<<grid, 128, 0, s>>>((S*)fA, (CuT<S>*)cu, cls, c1, c2, ux, uy, p, g, P, y0, y_b, rows);
        return cudaGetLastError();
    }
    static cudaError_t csum_ip(const void* f, void* cpl, const uint8_t* cls, const Geo& g, int odd, cudaStream_t s)
    {
        dim3 grid((g.pitch + 127) / 128, g.ny);
        if (odd) k_csum<S, R, true><<<grid, 128, 0, s>>>((const S*)f, (R*)cpl, cls, g);
        else k_csum<S, R, false><<<grid, 128, 0, s>>>((const S*)f, (R*)cpl, cls, g);
        return cudaGetLastError();
    }
    // resident blocks of the in-place interior kernel per step parity: its
    // FP32 form holds all 18 order-parameter populations at once; at 5 blocks
    // (96 registers) the odd (gathering) form spills a few words, and is still
    // faster than at 4 blocks (GB300, 2048^2: FP32 13.0 -> 14.1, FP16 13.6 ->
    // 15.1 G node updates/s with both parities at 5)
#ifndef TLB_IP_MINB_EVEN
#define TLB_IP_MINB_EVEN 5
#endif
#ifndef TLB_IP_MINB_ODD
#define TLB_IP_MINB_ODD 5
#endif
    // 16-bit storage with the whole next read set loaded one iteration ahead
    // (TLB_PIPE_IP16) runs at 4 blocks (GB300, 2048^2: 16.3 -> 17.2 G node
    // updates/s; at 5 blocks it spills and gains 1%)
#ifndef TLB_IP_MINB16
#define TLB_IP_MINB16 4
#endif
    static constexpr int kMinBIpEven =
        Store<S>::k16 && kPipeIp16 ? TLB_IP_MINB16 : (std::is_same<R, float>::value ? TLB_IP_MINB_EVEN : MINB);
    static constexpr int kMinBIpOdd =
        Store<S>::k16 && kPipeIp16 ? TLB_IP_MINB16 : (std::is_same<R, float>::value ? TLB_IP_MINB_ODD : MINB);
    template <bool UNI, bool ODD>
    static void launch_interior_ip(void* f, void* cu, const void* cpl, const uint8_t* cls, const Geo& g,
                                   const Prm<R>& P, cudaStream_t s)
    {
        constexpr int TX = BLOCK - 4;
        constexpr int kMinB = ODD ? kMinBIpOdd : kMinBIpEven;
        const int rows = rows_for(g, TX, ROWS, kMinB);
        dim3 grid((g.nx + TX - 1) / TX, (g.ny + rows - 1) / rows);
        k_step_interior_ip<S, R, BLOCK, ROWS, PREFETCH, kMinB, MRT, UNI, ODD><<<grid, BLOCK, 0, s>>>(
            (S*)f, (CuT<S>*)cu, (const R*)cpl, cls, g, P, rows);
    }
    static cudaError_t interior_ip(void* f, void* cu, const void* cpl, const uint8_t* cls, const Geo& g,
                                   const Prm<double>& Pd, int odd, cudaStream_t s)
    {
        const Prm<R> P = cast_prm<R>(Pd);
        if (Pd.uni != 0.0) {
            if (odd) launch_interior_ip<true, true>(f, cu, cpl, cls, g, P, s);
            else launch_interior_ip<true, false>(f, cu, cpl, cls, g, P, s);
        } else {
            if (odd) launch_interior_ip<false, true>(f, cu, cpl, cls, g, P, s);
            else launch_interior_ip<false, false>(f, cu, cpl, cls, g, P, s);
        }
        return cudaGetLastError();
    }
    static cudaError_t wall_ip(void* f, void* cu, const void* cpl, const uint8_t* cls, const uint32_t* list,
                               int nlist, const Geo& g, const Prm<double>& Pd, int odd, int lid, cudaStream_t s)
    {
        const Prm<R> P = cast_prm<R>(Pd);
        if (nlist <= 0) return cudaSuccess;
        const int blocks = (nlist + 127) / 128;
        if (odd)
            k_step_wall_ip<S, R, MRT, true><<<blocks, 128, 0, s>>>((S*)f, (CuT<S>*)cu, (const R*)cpl, cls, list, nlist,
                                                                  g, P, lid);
        else
            k_step_wall_ip<S, R, MRT, false><<<blocks, 128, 0, s>>>((S*)f, (CuT<S>*)cu, (const R*)cpl, cls, list,
                                                                   nlist, g, P, lid);
        return cudaGetLastError();
    }
    static cudaError_t swap_ip(void* f, const uint8_t* cls, const Geo& g, cudaStream_t s)
    {
        dim3 grid((g.nx + 127) / 128, g.ny);
        k_swap<S><<<grid, 128, 0, s>>>((S*)f, cls, g);
        return cudaGetLastError();
    }
    static const Ops& table()
    {
        static const Ops t{sizeof(S), Store<S>::kPlanes, sizeof(CuT<S>), &interior, &wall, &init, &read, &contact, &film, &batch_step,
                          &batch_blocks_per_sm, sizeof(LatDesc<R>), &fill_desc, &mass, &init_rows, sizeof(R),
                          &csum_ip, &interior_ip, &wall_ip, &swap_ip};
        return t;
    }
};

}  // namespace tlb

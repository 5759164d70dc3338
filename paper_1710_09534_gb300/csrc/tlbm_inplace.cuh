// In-place streaming (the AA pattern): one distribution buffer instead of two.
//
// Step parity EVEN (ODD = false): node x reads its pre-collision populations
// from its own slots k and writes each post-collision f'_k into its own slot
// k-bar.  Step parity ODD: node x reads f_k from slot k-bar of x - e_k, where
// the even step left it (or from its own slot k when x - e_k is a wall, the
// half-way bounce-back of Eq. 44), and writes f'_k into slot k of x + e_k (or
// into its own slot k-bar on a wall link).  After an odd step the buffer is
// back in the layout of the two-buffer update (slot k of x holds the
// pre-collision f_k(x)); an even step that ends a call is followed by
// k_swap, the plain streaming of that layout.
//
// In both parities a node reads and writes one and the same set of
// locations, which no other node touches, so the update is race-free with
// plain loads, provided that the populations of an opposite pair are both
// read before either is written (collide_all_inplace).  The order parameters
// are the one non-local input (the radius-2 stencils of Eqs. 8, 20a, 20b): a
// neighbour's sum would race with that neighbour's own update, so k_csum
// writes c_1, c_2 of every node to two planes first and the update reads them
// from there.
#pragma once
#include "tlbm_kernels.cuh"

namespace tlb {

// Where the pre-collision population of direction k of node (x, y) lives in
// the in-place layout: element offset and slot (0..8 within a distribution),
// or nowhere (a population arriving from beyond a lid edge is zero).
template <bool ODD>
__device__ __forceinline__ bool src_ip(const Geo& g, const uint8_t* __restrict__ cls, int k, int x, int y,
                                       long long o, long long& off, int& slot)
{
    off = o;
    slot = k;
    if (!ODD || k == 0) return true;
    long long s_off = 0;
    const int s = site_of(g, cls, x - ex(k), y - ey(k), s_off);
    if (fluidlike(s)) {
        off = s_off;
        slot = opp(k);
        return true;
    }
    return s == ST_WET || s == ST_NEUTRAL;  // bounce-back: own slot k
}

// c_1, c_2 of every node (zero on solid nodes and row padding) into planes
// cpl[0], cpl[PL] (Eq. 13a with the sum order of order_params).
template <typename S, typename R, bool ODD>
__global__ void k_csum(const S* __restrict__ f, R* __restrict__ cpl, const uint8_t* __restrict__ cls, Geo g)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= g.pitch) return;
    const long long PL = g.plane;
    const long long o = (long long)y * g.pitch + x;
    R c1 = R(0), c2 = R(0);
    const uint8_t c = x < g.nx ? cls[o] : uint8_t(ST_NEUTRAL);
    if (fluidlike(c & CLS_KIND_MASK)) {
        R v[18];
        if (ODD && (c & CLS_INTERIOR)) {
            // no wall within reach: the plain (periodically wrapped) neighbours
            const PushOffsets po(g, x, y);
            static_for<0, 9>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                const long long s = K == 0 ? o : po.template dest<opp(K)>();
                v[K] = ld_pop<R>(f, opp(K), PL, s);
                v[9 + K] = ld_pop<R>(f, 9 + opp(K), PL, s);
            });
        } else {
#pragma unroll
            for (int k = 0; k < 9; k++) {
                long long off;
                int slot;
                const bool has = src_ip<ODD>(g, cls, k, x, y, o, off, slot);
                v[k] = has ? ld_pop<R>(f, slot, PL, off) : R(0);
                v[9 + k] = has ? ld_pop<R>(f, 9 + slot, PL, off) : R(0);
            }
        }
        if constexpr (Store<S>::kLo) {
            v[0] += ld_lo<R>(f, 0, PL, o);
            v[9] += ld_lo<R>(f, 1, PL, o);
        }
        c1 = sum9(v);
        c2 = sum9(v + 9);
    }
    cpl[o] = c1;
    cpl[PL + o] = c2;
}

// 16-bit storage: the whole read set of the next iteration's update node (8
// pair words, 4 FP32 rest parts, 9 g values, 4 c_i u values) loaded one
// iteration ahead, as stored, and decoded when consumed.  Safe in place: a
// node's read set is written by that node's own update only.
#ifndef TLB_PIPE_IP16
#define TLB_PIPE_IP16 1
#endif
constexpr bool kPipeIp16 = TLB_PIPE_IP16 != 0;

struct RawIpNode {
    unsigned w[8];
    float r[2], l[2], cu[4];
    unsigned short gq[9];
};

// ---------------------------------------------------------------------------
// Interior tile, in place: the marching scheme of interior_tile with c read
// from the planes and the parity's addressing.  Interior nodes have no wall
// within radius 2, so no bounce-back arises here.
// ---------------------------------------------------------------------------
template <typename S, typename R, int BLOCK, bool PREFETCH, bool MRT, bool UNI, bool ODD>
__device__ __forceinline__ void interior_tile_ip(S* f, CuT<S>* __restrict__ cu, const R* __restrict__ cpl,
                                                 const uint8_t* __restrict__ cls, const Geo& g, const Prm<R>& P,
                                                 int bx, int by, int rows, ColRings<R, BLOCK>& sh)
{
    const long long PL = g.plane;
    const int t = threadIdx.x;
    const int x0 = bx * (BLOCK - 4);
    const int xs = x0 - 2 + t;
    int xw = xs;
    bool col_in = xs < g.nx + 2;
    if (xs < 0 || xs >= g.nx) {
        if (g.edge[0] == EDGE_PERIODIC) xw = xs < 0 ? xs + g.nx : xs - g.nx;
        else col_in = false;
    }
    const bool updater = t >= 2 && t < BLOCK - 2 && xs < g.nx;
    const int y0 = by * rows;
    const int y1 = min(y0 + rows, g.ny);
    const int dir = (by & 1) ? -1 : 1;
    const int iters = (y1 - y0) + 4;
    // this column's c and mu histories (as in interior_tile)
    R ca[3] = {R(0), R(0), R(0)}, cb[3] = {R(0), R(0), R(0)};
    R ma[3] = {R(0), R(0), R(0)}, mb[3] = {R(0), R(0), R(0)};
    constexpr bool PIP = kPipeIp16 && Store<S>::k16 && PREFETCH && !MRT;
    RawIpNode nr;
    // the read set of node (xs, yr) in this parity's layout, as stored
    auto load_raw = [&](int yr) {
        const long long o2 = (long long)yr * g.pitch + xs;
        const PushOffsets p2(g, xs, yr);
        const unsigned* wp = reinterpret_cast<const unsigned*>(f);
        const unsigned short* hp = reinterpret_cast<const unsigned short*>(f);
        const float* rp = rest_region(f, PL);
        static_for<1, 9>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            constexpr int q = ODD ? opp(K) : K;
            const long long sK = ODD ? p2.template dest<opp(K)>() : o2;
            nr.w[K - 1] = ld_any<false>(wp + (long long)(q - 1) * PL + sK);
        });
#pragma unroll
        for (int i = 0; i < 2; i++) {
            nr.r[i] = ld_any<false>(rp + i * PL + o2);
            nr.l[i] = ld_any<false>(rp + (2 + i) * PL + o2);
        }
        static_for<0, 9>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            const long long sK = (ODD && K != 0) ? p2.template dest<opp(K)>() : o2;
            nr.gq[K] = ld_any<false>(hp + idx16(18 + (ODD ? opp(K) : K), PL, sK));
        });
#pragma unroll
        for (int q = 0; q < 4; q++) nr.cu[q] = float(cu[q * PL + o2]);
    };

    for (int it = 0; it < iters; it++) {
        const int yc = dir > 0 ? y0 - 2 + it : y1 + 1 - it;
        const int ym = yc - dir;
        const int yu = yc - 2 * dir;
        // the update node's loads are issued before its node class is known
        // (see interior_tile); all their addresses are inside the lattice
        const bool in_rows = updater && it >= 4;
        const long long ou = in_rows ? (long long)yu * g.pitch + xs : 0;
        const bool upd = in_rows && (cls[ou] & CLS_INTERIOR) != 0;
        R gv[9], cp[4];
        PushOffsets po(g, in_rows ? xs : 0, in_rows ? yu : 0);
        // g of direction k: own slot k (even) or slot k-bar of x - e_k (odd)
        auto load_g = [&]() {
            static_for<0, 9>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                gv[K] = ODD ? ld_pop<R, false>(f, 18 + opp(K), PL, K == 0 ? ou : po.template dest<opp(K)>())
                            : ld_pop<R, false>(f, 18 + K, PL, ou);
            });
#pragma unroll
            for (int q = 0; q < 4; q++) cp[q] = R(cu[q * PL + ou]);
        };
        // With FP32 arithmetic all 18 order-parameter populations are read
        // before the collision, and with PREFETCH already here, so that their
        // latency overlaps the shared-memory phases: plain loads cannot be
        // moved past the stores of earlier directions, so reading them pair by
        // pair would expose one load latency per pair.  (FP64 keeps the pairs:
        // its registers are the tighter limit.)
        constexpr bool kPre = std::is_same<R, float>::value;
        R f1[9], f2[9];
        auto load_f = [&](auto kc, R& f1k, R& f2k) {
            constexpr int K = decltype(kc)::value;
            const long long s = (ODD && K != 0) ? po.template dest<opp(K)>() : ou;
            constexpr int q = ODD ? opp(K) : K;
            if constexpr (q == 0) {
                f1k = ld_pop<R, false>(f, 0, PL, s);
                f2k = ld_pop<R, false>(f, 9, PL, s);
            } else {
                ld_pair<R, false>(f, q, PL, s, f1k, f2k);
            }
        };
        auto load_all_f = [&]() {
            static_for<0, 9>([&](auto kc) { load_f(kc, f1[decltype(kc)::value], f2[decltype(kc)::value]); });
        };
        R pl[2] = {R(0), R(0)};
        if constexpr (PIP) {
            if constexpr (Store<S>::k16) {
                // decode this iteration's read set, then issue the next one's
                constexpr float inv = 1.0f / float(1 << Store<S>::kScaleExp);
#pragma unroll
                for (int k = 1; k < 9; k++) {
                    const float2 v = dec16x2(S{}, nr.w[k - 1]);
                    f1[k] = R(v.x * inv);
                    f2[k] = R(v.y * inv);
                }
                f1[0] = R(nr.r[0]);
                f2[0] = R(nr.r[1]);
                pl[0] = R(nr.l[0]);
                pl[1] = R(nr.l[1]);
#pragma unroll
                for (int k = 0; k < 9; k++) gv[k] = R(dec16(S{}, nr.gq[k]) * inv);
#pragma unroll
                for (int q = 0; q < 4; q++) cp[q] = R(nr.cu[q]);
                if (updater && it + 1 >= 4 && it + 1 < iters) load_raw(yu + dir);
            }
        } else if (PREFETCH && in_rows) {
            load_g();
            if constexpr (kPre) load_all_f();
        }
        // 1) c of row yc from the planes
        {
            int yw = yc;
            bool in = col_in && yc < g.ny + 2;
            if (yc < 0 || yc >= g.ny) {
                if (g.edge[2] == EDGE_PERIODIC) yw = yc < 0 ? yc + g.ny : yc - g.ny;
                else in = false;
            }
            R a = R(0), b = R(0);
            if (in) {
                const long long oc = (long long)yw * g.pitch + xw;
                a = __ldg(cpl + oc);
                b = __ldg(cpl + PL + oc);
            }
            ca[2] = ca[1];
            ca[1] = ca[0];
            ca[0] = a;
            cb[2] = cb[1];
            cb[1] = cb[0];
            cb[0] = b;
            if (it >= 2) {
                const int sl = (ym + 9) % 3;
                sh.put_ad(sl, t, fma(R(4), ca[1], ca[0] + ca[2]), fma(R(4), cb[1], cb[0] + cb[2]),
                          dir > 0 ? ca[0] - ca[2] : ca[2] - ca[0], dir > 0 ? cb[0] - cb[2] : cb[2] - cb[0]);
            }
        }
        __syncthreads();
        // 2) mu of row ym (Eq. 8 with Eq. 20b)
        if (it >= 2 && t >= 1 && t < BLOCK - 1) {
            const int sl = (ym + 9) % 3;
            const auto al = sh.a(sl, t - 1), ar = sh.a(sl, t + 1);
            const R lap1 = fma(R(4), fma(R(-5), ca[1], ca[0] + ca[2]), al.x + ar.x);
            const R lap2 = fma(R(4), fma(R(-5), cb[1], cb[0] + cb[2]), al.y + ar.y);
            R mu1, mu2;
            chem_pot(P, ca[1], cb[1], lap1, lap2, mu1, mu2);
            ma[2] = ma[1];
            ma[1] = ma[0];
            ma[0] = mu1;
            mb[2] = mb[1];
            mb[1] = mb[0];
            mb[0] = mu2;
            if constexpr (!UNI) {
                sh.put_m(t, fma(R(4), ma[1], ma[0] + ma[2]), fma(R(4), mb[1], mb[0] + mb[2]));
            }
        }
        // only the general update's M is written in phase 2 and read in phase
        // 3 of the same iteration; the rings of A and D need the one barrier
        // above per iteration (uniform update without this one, GB300, 2048^2:
        // FP32 14.21 -> 14.29, FP16 17.57 -> 17.66 G node updates/s)
        if constexpr (!UNI) __syncthreads();
        // 3) update of row yu
        if (!upd) continue;
        Macro<R> m;
        {
            const int su = (yu + 9) % 3;
            m.c1 = ca[2];
            m.c2 = cb[2];
            m.mu1 = ma[1];
            m.mu2 = mb[1];
            const auto al = sh.a(su, t - 1), ar = sh.a(su, t + 1);
            const auto dl = sh.d(su, t - 1), dc = sh.d(su, t), dr = sh.d(su, t + 1);
            m.g1x = ar.x - al.x;
            m.g2x = ar.y - al.y;
            m.g1y = fma(R(4), dc.x, dl.x + dr.x);
            m.g2y = fma(R(4), dc.y, dl.y + dr.y);
            if constexpr (UNI) {
                m.lm1 = m.lm2 = R(0);
            } else {
                const auto ml = sh.m(t - 1), mr = sh.m(t + 1);
                m.lm1 = fma(R(4), fma(R(-5), ma[1], ma[0] + ma[2]), ml.x + mr.x);
                m.lm2 = fma(R(4), fma(R(-5), mb[1], mb[0] + mb[2]), ml.y + mr.y);
            }
            m.rho = UNI ? P.rho[2] : density(P, m.c1, m.c2);
        }
        if (!PREFETCH) load_g();
        Hydro<R> h;
        hydro_from_g<UNI>(P, m, gv, h);
        const R c1ux = m.c1 * h.ux, c1uy = m.c1 * h.uy, c2ux = m.c2 * h.ux, c2uy = m.c2 * h.uy;
        cu[0 * PL + ou] = CuT<S>(c1ux);
        cu[1 * PL + ou] = CuT<S>(c1uy);
        cu[2 * PL + ou] = CuT<S>(c2ux);
        cu[3 * PL + ou] = CuT<S>(c2uy);
        if constexpr (kPre) {
            if (!PREFETCH) load_all_f();
        }
        CollideOf<MRT, R, UNI> col;
        col.build(P, m, h, c1ux - cp[0], c1uy - cp[1], c2ux - cp[2], c2uy - cp[3]);
        collide_all_inplace<S, R>(col, gv,
            [&](auto kc, R& f1k, R& f2k) {
                if constexpr (kPre) {
                    f1k = f1[decltype(kc)::value];
                    f2k = f2[decltype(kc)::value];
                } else {
                    load_f(kc, f1k, f2k);
                }
            },
            [&](R& l1, R& l2) {
                if constexpr (PIP) {
                    l1 = pl[0];
                    l2 = pl[1];
                } else {
                    l1 = ld_lo<R, false>(f, 0, PL, ou);
                    l2 = ld_lo<R, false>(f, 1, PL, ou);
                }
            },
            [&](auto kc, auto o1, auto o2, auto og) {
                constexpr int K = decltype(kc)::value;
                const long long d = (ODD && K != 0) ? po.template dest<K>() : ou;
                constexpr int q = ODD ? K : opp(K);
                st_three(f, q, PL, d, o1, o2, og);
            },
            [&](R l1, R l2) {
                st_lo(f, 0, PL, ou, l1);
                st_lo(f, 1, PL, ou, l2);
            });
    }
}

template <typename S, typename R, int BLOCK, int ROWS, bool PREFETCH, int MINB, bool MRT, bool UNI, bool ODD>
__global__ void __launch_bounds__(BLOCK, MINB)
k_step_interior_ip(S* f, CuT<S>* __restrict__ cu, const R* __restrict__ cpl, const uint8_t* __restrict__ cls,
                   Geo g, Prm<R> P, int rows)
{
    __shared__ ColRings<R, BLOCK> sh;
    interior_tile_ip<S, R, BLOCK, PREFETCH, MRT, UNI, ODD>(f, cu, cpl, cls, g, P, blockIdx.x, blockIdx.y, rows, sh);
}

// ---------------------------------------------------------------------------
// Near-wall and lid nodes, in place.  Lid nodes (Eq. 51 reads the
// pre-collision state of the node below, which the same step updates) run in
// a launch of their own before the others: LID selects which kind a launch
// takes.
// ---------------------------------------------------------------------------
template <bool ODD, typename S, typename V1, typename V2, typename VG>
__device__ __forceinline__ void store_ip(const Geo& g, const uint8_t* __restrict__ cls, S* f, int K, int x, int y,
                                         long long o, V1 o1, V2 o2, VG og)
{
    const long long PL = g.plane;
    long long d = o;
    int q = opp(K);  // even: own slot k-bar
    if (ODD && K != 0) {
        const int s = site_of(g, cls, x + ex(K), y + ey(K), d);
        if (fluidlike(s)) {
            q = K;
        } else {
            d = o;  // wall: bounce back into own slot k-bar (Eq. 44)
            if (s == ST_VOID) {  // leaves through the lid; nothing comes in
                o1 = V1{};
                o2 = V2{};
                og = VG{};
            }
        }
    }
    st_three(f, q, PL, d, o1, o2, og);
}

template <typename S, typename R, bool MRT, bool ODD>
__device__ __forceinline__ void wall_node_ip(S* f, CuT<S>* __restrict__ cu, const R* __restrict__ cpl,
                                             const uint8_t* __restrict__ cls, const Geo& g, const Prm<R>& P,
                                             uint32_t packed, bool lid)
{
    const int x = (int)(packed & 0xffffu), y = (int)(packed >> 16);
    const long long PL = g.plane;
    const long long o = (long long)y * g.pitch + x;
    const int kind = cls[o] & CLS_KIND_MASK;
    if ((kind == ST_LID) != lid) return;
    PlaneFetch<R> fetch{cpl, PL};
    // pre-collision population of distribution base (0, 9, 18), direction k,
    // of node (xn, yn)
    auto pop = [&](int base, int k, int xn, int yn, long long on) {
        long long off;
        int slot;
        return src_ip<ODD>(g, cls, k, xn, yn, on, off, slot) ? ld_pop<R, false>(f, base + slot, PL, off) : R(0);
    };
    auto store = [&](auto kc, auto o1, auto o2, auto og) { store_ip<ODD>(g, cls, f, decltype(kc)::value, x, y, o, o1, o2, og); };
    auto store_lo = [&](R l1, R l2) {
        st_lo(f, 0, PL, o, l1);
        st_lo(f, 1, PL, o, l2);
    };

    if (kind == ST_FLUID) {
        Macro<R> m;
        window_macros(g, cls, P, x, y, fetch, m);
        R gv[9];
#pragma unroll
        for (int k = 0; k < 9; k++) gv[k] = pop(18, k, x, y, o);
        Hydro<R> h;
        hydro_from_g(P, m, gv, h);
        const R c1ux = m.c1 * h.ux, c1uy = m.c1 * h.uy, c2ux = m.c2 * h.ux, c2uy = m.c2 * h.uy;
        const R d1x = c1ux - R(cu[0 * PL + o]), d1y = c1uy - R(cu[1 * PL + o]);
        const R d2x = c2ux - R(cu[2 * PL + o]), d2y = c2uy - R(cu[3 * PL + o]);
        cu[0 * PL + o] = CuT<S>(c1ux);
        cu[1 * PL + o] = CuT<S>(c1uy);
        cu[2 * PL + o] = CuT<S>(c2ux);
        cu[3 * PL + o] = CuT<S>(c2uy);
        CollideOf<MRT, R> col;
        col.build(P, m, h, d1x, d1y, d2x, d2y);
        collide_all_inplace<S, R>(col, gv,
            [&](auto kc, R& f1k, R& f2k) {
                constexpr int K = decltype(kc)::value;
                f1k = pop(0, K, x, y, o);
                f2k = pop(9, K, x, y, o);
            },
            [&](R& l1, R& l2) {
                l1 = ld_lo<R, false>(f, 0, PL, o);
                l2 = ld_lo<R, false>(f, 1, PL, o);
            },
            store, store_lo);
    } else if (kind == ST_LID) {
        // x_f is the node below; x_u takes its macros and gradients, u = (U0, 0)
        const long long of = o - g.pitch;
        Macro<R> m;
        window_macros(g, cls, P, x, y - 1, fetch, m);
        R gf[9];
#pragma unroll
        for (int k = 0; k < 9; k++) gf[k] = pop(18, k, x, y - 1, of);
        Hydro<R> hf;
        hydro_from_g(P, m, gf, hf);
        Hydro<R> h = hf;
        h.ux = P.lid_u;
        h.uy = R(0);
        h.usq = P.lid_u * P.lid_u;
        const R c1ux = m.c1 * h.ux, c2ux = m.c2 * h.ux;
        const R d1x = c1ux - R(cu[0 * PL + o]), d1y = R(0) - R(cu[1 * PL + o]);
        const R d2x = c2ux - R(cu[2 * PL + o]), d2y = R(0) - R(cu[3 * PL + o]);
        cu[0 * PL + o] = CuT<S>(c1ux);
        cu[1 * PL + o] = CuT<S>(0);
        cu[2 * PL + o] = CuT<S>(c2ux);
        cu[3 * PL + o] = CuT<S>(0);
        CollideOf<MRT, R> col;
        col.build(P, m, h, d1x, d1y, d2x, d2y);
        // Eq. 51: f(x_u) = f^eq(x_u) + [f(x_f) - f^eq(x_f)], for f^1, f^2 and g
        R gu[9], f1u[9], f2u[9];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            R e1u, e2u, egu, e1f, e2f, egf;
            equilibria(k, P, m.c1, m.c2, m.mu1, m.mu2, m.rho, hf.p, h.ux, h.uy, e1u, e2u, egu);
            equilibria(k, P, m.c1, m.c2, m.mu1, m.mu2, m.rho, hf.p, hf.ux, hf.uy, e1f, e2f, egf);
            R ff1 = pop(0, k, x, y - 1, of), ff2 = pop(9, k, x, y - 1, of);
            if constexpr (Store<S>::kLo) {
                if (k == 0) {
                    ff1 += ld_lo<R, false>(f, 0, PL, of);
                    ff2 += ld_lo<R, false>(f, 1, PL, of);
                }
            }
            f1u[k] = e1u + (ff1 - e1f);
            f2u[k] = e2u + (ff2 - e2f);
            gu[k] = egu + (gf[k] - egf);
        }
        collide_all_inplace<S, R>(col, gu,
            [&](auto kc, R& f1k, R& f2k) {
                constexpr int K = decltype(kc)::value;
                f1k = f1u[K];
                f2k = f2u[K];
            },
            [&](R& l1, R& l2) {
                l1 = R(0);
                l2 = R(0);
            },
            store, store_lo);
    }
}

template <typename S, typename R, bool MRT, bool ODD>
__global__ void __launch_bounds__(128)
k_step_wall_ip(S* f, CuT<S>* __restrict__ cu, const R* __restrict__ cpl, const uint8_t* __restrict__ cls,
               const uint32_t* __restrict__ list, int nlist, Geo g, Prm<R> P, int lid)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nlist) return;
    wall_node_ip<S, R, MRT, ODD>(f, cu, cpl, cls, g, P, list[t], lid != 0);
}

// ---------------------------------------------------------------------------
// Streaming of the even-step layout into the two-buffer layout, in place:
// slot k-bar of x (f'_k of x) and slot k of x + e_k (f'_{k-bar} of x + e_k)
// trade places, each pair taken by the node whose link to the other is one
// of +x, +y, (1, 1), (-1, 1).  A wall link keeps the bounced-back value
// where it is (Eq. 44); a lid link empties the slot (nothing enters from
// beyond the lid).  Rest populations do not move.
// ---------------------------------------------------------------------------
template <typename S>
__global__ void k_swap(S* f, const uint8_t* __restrict__ cls, Geo g)
{
    using E = typename std::conditional<Store<S>::k16, unsigned short, S>::type;  // raw element
    E* e = reinterpret_cast<E*>(f);
    // element index of moving population q of node n (16-bit: the paired layout)
    auto at = [&](int q, long long n) -> long long {
        if constexpr (Store<S>::k16) return idx16(q, g.plane, n);
        else return q * g.plane + n;
    };
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= g.nx) return;
    const long long o = (long long)y * g.pitch + x;
    if (!fluidlike(cls[o] & CLS_KIND_MASK)) return;
    static_for<1, 9>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        constexpr int KB = opp(K);
        long long d = 0;
        const int s = site_of(g, cls, x + ex(K), y + ey(K), d);
        if (fluidlike(s)) {
            if constexpr (K == 1 || K == 2 || K == 5 || K == 6) {
#pragma unroll
                for (int b = 0; b < 27; b += 9) {
                    const E a = e[at(b + KB, o)];
                    e[at(b + KB, o)] = e[at(b + K, d)];
                    e[at(b + K, d)] = a;
                }
            }
        } else if (s == ST_VOID) {
#pragma unroll
            for (int b = 0; b < 27; b += 9) e[at(b + KB, o)] = E(0);
        }
    });
}

}  // namespace tlb

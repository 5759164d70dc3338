// Kernels of one time step and of set-up / read-out, templated on the storage
// type S and the arithmetic type R (double/double or float/float).
//
//   k_step_interior  fused stencil + collide + push for every node whose
//                    5x5 neighbourhood is plain fluid (no wall, no lid):
//                    c_1, c_2 on the tile plus a radius-2 halo from the local
//                    sums of the pre-collision f (push streaming keeps them
//                    local), mu_1, mu_2 on the tile plus radius 1 in shared
//                    memory, then the per-node update.
//   k_step_wall      the same update for the compacted list of the other
//                    fluid nodes, with the ghost rules of Eqs. 42-43,
//                    bounce-back (Eq. 44) and the lid (Eqs. 51-53).
//   k_init, k_read_fields, k_mass_partials/k_mass_final
#pragma once
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include "tlbm_device.cuh"

namespace tlb {

template <int K, int N, typename F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (K < N) {
        f(std::integral_constant<int, K>{});
        static_for<K + 1, N>(f);
    }
}

template <typename S>
__device__ __forceinline__ double to_d(S v) { return (double)v; }

// c_i = sum_k f^i_k (Eq. 13a): the eight moving populations first, the rest
// population last, so that the large term is rounded once.
template <typename R>
__device__ __forceinline__ R sum9(const R* v)
{
    return v[0] + (((v[1] + v[2]) + (v[3] + v[4])) + ((v[5] + v[6]) + (v[7] + v[8])));
}
// The same with the moving populations in units of 2^SE (v[0] in plain units).
template <int SE, typename R>
__device__ __forceinline__ R sum9s(const R* v)
{
    if constexpr (SE == 0) {
        return sum9(v);
    } else {
        const R m = ((v[1] + v[2]) + (v[3] + v[4])) + ((v[5] + v[6]) + (v[7] + v[8]));
        return fma(R(1.0 / double(1 << SE)), m, v[0]);
    }
}

// Storage formats of the distributions (template parameter S):
//   double  27 FP64 planes (q = 0..8 f^1_k, 9..17 f^2_k, 18..26 g_k).
//   float   27 FP32 planes, plus the rest populations f^1_0, f^2_0 kept as
//           unevaluated float pairs hi + lo (hi in planes 0/9, lo in planes
//           27/28), so that the per-node update conserves sum_k f^i_k
//           (Eq. 1a conserves c_i) without ever rounding the O(1) rest value
//           (see collide_all).
//   __half, __nv_bfloat16
//           the 25 other populations as 16-bit values after subtracting their
//           equilibrium at rest (u = 0, mu = 0, p = 0), which is zero for every
//           one of them in this model (Eq. 2a: f^{i,eq}_k, k != 0, is
//           proportional to mu_i and u; Eq. 2b: g^eq is pressure-based), and
//           (FP16) scaled by 2^kF16ScaleExp so that small populations stay normal
//           numbers; the rest populations, whose equilibrium at rest is c_i
//           itself, stay FP32 pairs.  Layout: 8 planes of 32-bit words, word
//           k-1 of a node holding f^1_k (low half) and f^2_k (high half) for
//           k = 1..8 (both stream to the same node, so one 32-bit access moves
//           both); 9 16-bit planes g_0..g_8; then 4 FP32 planes: f^1_0 hi,
//           f^2_0 hi, f^1_0 lo, f^2_0 lo.
// The c_i u planes of Eq. 19 are FP64 with FP64 storage and FP32 otherwise.
template <typename S>
struct Store {
    static constexpr bool k16 = std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value;
    static constexpr bool kLo = !std::is_same<S, double>::value;
    static constexpr int kPlanes = std::is_same<S, double>::value ? 27 : (k16 ? 33 : 29);  // in units of S
    static constexpr int kScaleExp = std::is_same<S, __half>::value ? kF16ScaleExp : 0;
    using Cu = typename std::conditional<std::is_same<S, double>::value, double, float>::type;
    using R = typename std::conditional<std::is_same<S, double>::value, double, float>::type;
};
template <typename S>
using CuT = typename Store<S>::Cu;

__device__ __forceinline__ float dec16(__half, unsigned short b) { return __half2float(__ushort_as_half(b)); }
__device__ __forceinline__ float dec16(__nv_bfloat16, unsigned short b) { return __uint_as_float((unsigned)b << 16); }
__device__ __forceinline__ unsigned short enc16(__half, float v) { return __half_as_ushort(__float2half_rn(v)); }
__device__ __forceinline__ unsigned short enc16(__nv_bfloat16, float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
// A 32-bit pair word (low half, high half) decoded to two floats, and two
// floats encoded into one, by the packed conversions (one rounding per value,
// the same as enc16 of each).
__device__ __forceinline__ float2 dec16x2(__half, unsigned w)
{
    __half2 h;
    memcpy(&h, &w, sizeof w);
    return __half22float2(h);
}
__device__ __forceinline__ float2 dec16x2(__nv_bfloat16, unsigned w)
{
    __nv_bfloat162 h;
    memcpy(&h, &w, sizeof w);
    return __bfloat1622float2(h);
}
__device__ __forceinline__ unsigned enc16x2(__half, float lo, float hi)
{
    const __half2 h = __floats2half2_rn(lo, hi);
    unsigned w;
    memcpy(&w, &h, sizeof w);
    return w;
}
__device__ __forceinline__ unsigned enc16x2(__nv_bfloat16, float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    unsigned w;
    memcpy(&w, &h, sizeof w);
    return w;
}

// FP32 region of a 16-bit buffer (after the 16 + 9 16-bit planes)
template <typename S>
__device__ __forceinline__ const float* rest_region(const S* f, long long PL)
{
    return reinterpret_cast<const float*>(f + 25 * PL);
}
template <typename S>
__device__ __forceinline__ float* rest_region(S* f, long long PL)
{
    return reinterpret_cast<float*>(f + 25 * PL);
}
// 16-bit element index of moving population q (1..8, 10..26) of node o in a
// 16-bit buffer: f^1_k, f^2_k share 32-bit word k-1 of the node, g_k follow
__device__ __forceinline__ long long idx16(int q, long long PL, long long o)
{
    if (q < 9) return (long long)(q - 1) * 2 * PL + 2 * o;
    if (q < 18) return (long long)(q - 10) * 2 * PL + 2 * o + 1;
    return 16 * PL + (long long)(q - 18) * PL + o;
}

// Load through the read-only path (NC: the buffer is not written during the
// kernel) or a plain coherent load (the in-place update writes what it reads).
template <bool NC, typename T>
__device__ __forceinline__ T ld_any(const T* p)
{
    if constexpr (NC) return __ldg(p);
    else return *p;
}

// Population q (0..26) of node offset o, as the arithmetic type R (for the
// rest populations of the paired formats: the hi part).  RAW: a 16-bit
// population in the units it is stored in (FP16: 2^kF16ScaleExp times its
// value), so that an update working in those units skips the scaling.
template <typename R, bool NC = true, bool RAW = false, typename S>
__device__ __forceinline__ R ld_pop(const S* __restrict__ f, int q, long long PL, long long o)
{
    if constexpr (Store<S>::k16) {
        if (q == 0 || q == 9) return R(ld_any<NC>(rest_region(f, PL) + (q == 9 ? PL : 0) + o));
        const float v = dec16(S{}, ld_any<NC>(reinterpret_cast<const unsigned short*>(f) + idx16(q, PL, o)));
        if constexpr (RAW) return R(v);
        constexpr float inv = 1.0f / float(1 << Store<S>::kScaleExp);
        return R(v * inv);
    } else {
        return R(ld_any<NC>(f + q * PL + o));
    }
}

// A 16-bit population already encoded (the bits as stored).
struct Bits16 {
    unsigned short b;
};
// f^1_k (low half) and f^2_k (high half) of a node already encoded into the
// 32-bit word of a 16-bit buffer.
struct Pair16 {
    unsigned w;
};
// lo part of rest population i (0: f^1_0, 1: f^2_0); zero for FP64
template <typename R, bool NC = true, typename S>
__device__ __forceinline__ R ld_lo(const S* __restrict__ f, int i, long long PL, long long o)
{
    if constexpr (Store<S>::k16) return R(ld_any<NC>(rest_region(f, PL) + (2 + i) * PL + o));
    else if constexpr (Store<S>::kLo) return R(ld_any<NC>(f + (27 + i) * PL + o));
    else return R(0);
}
// The value population q takes once stored (16-bit formats round; others keep it)
template <typename S, typename R>
__device__ __forceinline__ R as_stored(int q, R v)
{
    if constexpr (Store<S>::k16) {
        if (q == 0 || q == 9) return v;
        constexpr float sc = float(1 << Store<S>::kScaleExp), inv = 1.0f / sc;
        return R(dec16(S{}, enc16(S{}, float(v) * sc)) * inv);
    } else {
        return v;
    }
}
template <typename S, typename R>
__device__ __forceinline__ void st_pop(S* __restrict__ f, int q, long long PL, long long o, R v)
{
    if constexpr (std::is_same<R, Bits16>::value) {
        static_assert(Store<S>::k16, "encoded values belong to a 16-bit format");
        reinterpret_cast<unsigned short*>(f)[idx16(q, PL, o)] = v.b;
    } else if constexpr (Store<S>::k16) {
        if (q == 0 || q == 9) {
            rest_region(f, PL)[(q == 9 ? PL : 0) + o] = float(v);
        } else {
            constexpr float sc = float(1 << Store<S>::kScaleExp);
            reinterpret_cast<unsigned short*>(f)[idx16(q, PL, o)] = enc16(S{}, float(v) * sc);
        }
    } else {
        f[q * PL + o] = S(v);
    }
}
template <typename S, typename R>
__device__ __forceinline__ void st_lo(S* __restrict__ f, int i, long long PL, long long o, R v)
{
    if constexpr (Store<S>::k16) rest_region(f, PL)[(2 + i) * PL + o] = float(v);
    else if constexpr (Store<S>::kLo) f[(27 + i) * PL + o] = S(v);
}
// f^1_k and f^2_k (k = 1..8) of node o; with 16-bit storage one 32-bit load
// (RAW as for ld_pop).
template <typename R, bool NC = true, bool RAW = false, typename S>
__device__ __forceinline__ void ld_pair(const S* __restrict__ f, int k, long long PL, long long o, R& f1k, R& f2k)
{
    if constexpr (Store<S>::k16) {
        const unsigned w = ld_any<NC>(reinterpret_cast<const unsigned*>(f) + (long long)(k - 1) * PL + o);
        constexpr float inv = RAW ? 1.0f : 1.0f / float(1 << Store<S>::kScaleExp);
        const float2 v = dec16x2(S{}, w);
        f1k = R(v.x * inv);
        f2k = R(v.y * inv);
    } else {
        f1k = ld_pop<R, NC>(f, k, PL, o);
        f2k = ld_pop<R, NC>(f, 9 + k, PL, o);
    }
}
// The populations k of f^1, f^2 and g pushed to node d: values of the
// arithmetic type or, for 16-bit storage, Bits16 already encoded (the f^1_k,
// f^2_k pair of a 16-bit buffer goes out as one 32-bit store).
template <typename S, typename V1, typename V2, typename VG>
__device__ __forceinline__ void st_three(S* __restrict__ f, int k, long long PL, long long d, V1 o1, V2 o2, VG og)
{
    if constexpr (std::is_same<V1, Pair16>::value) {
        static_assert(Store<S>::k16 && std::is_same<V2, Pair16>::value, "a pair word goes to a 16-bit buffer");
        reinterpret_cast<unsigned*>(f)[(long long)(k - 1) * PL + d] = o1.w;  // k != 0: rest values are not pairs
        st_pop(f, 18 + k, PL, d, og);
    } else {
        if constexpr (Store<S>::k16 && std::is_same<V1, Bits16>::value && std::is_same<V2, Bits16>::value) {
            if (k != 0) {
                reinterpret_cast<unsigned*>(f)[(long long)(k - 1) * PL + d] = (unsigned)o1.b | ((unsigned)o2.b << 16);
                st_pop(f, 18 + k, PL, d, og);
                return;
            }
        }
        st_pop(f, k, PL, d, o1);
        st_pop(f, 9 + k, PL, d, o2);
        st_pop(f, 18 + k, PL, d, og);
    }
}

// c_i = sum_k f^i_k of node o for i = 1, 2 (rest population hi + lo)
template <typename R, typename S>
__device__ __forceinline__ void order_params(const S* __restrict__ f, long long PL, long long o, R& c1, R& c2)
{
    R v[18];
#pragma unroll
    for (int k = 0; k < 18; k++) v[k] = ld_pop<R>(f, k, PL, o);
    if constexpr (Store<S>::kLo) {
        v[0] += ld_lo<R>(f, 0, PL, o);
        v[9] += ld_lo<R>(f, 1, PL, o);
    }
    c1 = sum9(v);
    c2 = sum9(v + 9);
}

// Error-free transformation of a sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Rest pair (hi + lo) plus a small FP32 increment d, renormalised: TwoSum
// keeps the rounding of hi + d, which joins lo.
__device__ __forceinline__ void rest_add(float hi, float lo, float d, float& nhi, float& nlo)
{
    float s, e;
    two_sum(hi, d, s, e);
    const float t = e + lo;
    nhi = s + t;
    nlo = t - (nhi - s);
}

// All nine directions of one node.  load(kc, f1k, f2k) fetches the
// pre-collision order-parameter populations of direction kc (for kc = 0 the
// hi part), load_lo(f1lo, f2lo) the lo parts of the rest populations (FP32
// and 16-bit storage), store(kc, o1, o2, og) streams the post-collision triple
// and store_lo(o1lo, o2lo) the rest lo parts.  With paired rest populations
// the new rest population is the old one plus sum_k (f_k - o'_k) over the
// eight moving directions (o'_k as stored), so the stored sum_k f'^i_k equals
// the stored sum_k f^i_k (Eq. 1a conserves c_i; sum_k f^eq_k = c_i,
// sum_k F_k = 0) up to the FP32 rounding of those small differences and
// their sum -- none where f_k and o'_k are within a factor 2 of each other
// (Sterbenz), which covers near-equilibrium nodes, and exact for 16-bit
// storage -- while the O(1) rest value itself is never rounded; FP64 uses the
// direct form.
//
// SE: the moving populations (and g_0) are passed in and produced in units of
// 2^SE (SE = kF16ScaleExp when the update works in the units of FP16
// storage, 0 otherwise).  With 16-bit storage the outputs are encoded once
// here and handed to `store` as Bits16; the rest pair sees the decoded
// (stored) values, so the mass bookkeeping is unchanged.
template <typename S, typename R, int SE = 0, bool UNI, typename Load, typename LoadLo, typename St, typename StLo>
__device__ __forceinline__ void collide_all(const Collider<R, UNI>& col, const R gv[9], Load load, LoadLo load_lo,
                                            St store, StLo store_lo)
{
    constexpr bool ff = Store<S>::kLo;
    constexpr bool k16 = Store<S>::k16;
    static_assert(SE == 0 || (k16 && SE == Store<S>::kScaleExp), "scaled units are those of FP16 storage");
    // encode a value for 16-bit storage (in the units of the values)
    auto enc = [](R v) -> Bits16 {
        if constexpr (k16) {
            constexpr float sc = SE ? 1.0f : float(1 << Store<S>::kScaleExp);
            return Bits16{enc16(S{}, float(v) * sc)};
        } else {
            return Bits16{0};
        }
    };
    R d1 = R(0), d2 = R(0);  // sum_k (f_k - o'_k) over the moving directions
    // the directions go in opposite pairs (k, k-bar), which share most of
    // their arithmetic; both inputs of a pair are read before either output
    // is written (the in-place update relies on it)
    static_for<0, 4>([&](auto pc) {
        constexpr int K = pair_dir(decltype(pc)::value);
        constexpr int KB = opp(K);
        std::integral_constant<int, K> kc;
        std::integral_constant<int, KB> kbc;
        R a1, a2, b1, b2, oa1, oa2, oag, ob1, ob2, obg;
        load(kc, a1, a2);
        load(kbc, b1, b2);
        col.template pair<K>(a1, a2, gv[K], b1, b2, gv[KB], oa1, oa2, oag, ob1, ob2, obg);
        if constexpr (k16) {
            // f^1_k, f^2_k of each direction encoded into their pair word at once
            constexpr float sc = SE ? 1.0f : float(1 << Store<S>::kScaleExp);
            constexpr float inv = SE ? 1.0f : 1.0f / float(1 << Store<S>::kScaleExp);
            const Pair16 pa{enc16x2(S{}, float(oa1) * sc, float(oa2) * sc)};
            const Pair16 pb{enc16x2(S{}, float(ob1) * sc, float(ob2) * sc)};
            const float2 da = dec16x2(S{}, pa.w), db = dec16x2(S{}, pb.w);
            d1 += (a1 - R(da.x * inv)) + (b1 - R(db.x * inv));
            d2 += (a2 - R(da.y * inv)) + (b2 - R(db.y * inv));
            store(kc, pa, pa, enc(oag));
            store(kbc, pb, pb, enc(obg));
        } else {
            if constexpr (ff) {
                d1 += (a1 - oa1) + (b1 - ob1);
                d2 += (a2 - oa2) + (b2 - ob2);
            }
            store(kc, oa1, oa2, oag);
            store(kbc, ob1, ob2, obg);
        }
    });
    if constexpr (SE != 0) {
        constexpr R inv = R(1.0 / double(1 << SE));
        d1 *= inv;
        d2 *= inv;
    }
    std::integral_constant<int, 0> k0;
    R f10, f20, o1, o2, og;
    load(k0, f10, f20);
    if constexpr (ff) {
        R l1, l2;
        load_lo(l1, l2);
        // the collision sees the rest population as hi + lo
        col.post0(f10 + l1, f20 + l2, gv[0], o1, o2, og);
        R h1, h2, lo1, lo2;
        rest_add(f10, l1, d1, h1, lo1);
        rest_add(f20, l2, d2, h2, lo2);
        if constexpr (k16) store(k0, h1, h2, enc(og));
        else store(k0, h1, h2, og);
        store_lo(lo1, lo2);
    } else {
        col.post0(f10, f20, gv[0], o1, o2, og);
        store(k0, o1, o2, og);
    }
}

// The same contract with the MRT collision: the nine populations of each
// distribution are relaxed together in moment space, so all are loaded first
// (in plain units: SE = 0).
template <typename S, typename R, int SE = 0, typename Load, typename LoadLo, typename St, typename StLo>
__device__ __forceinline__ void collide_all(const MrtNode<R>& col, const R gv[9], Load load, LoadLo load_lo,
                                            St store, StLo store_lo)
{
    static_assert(SE == 0, "the MRT update works in plain units");
    constexpr bool ff = Store<S>::kLo;
    R f1[9], f2[9], o1[9], o2[9], og[9];
    static_for<0, 9>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        load(kc, f1[K], f2[K]);
    });
    const R h10 = f1[0], h20 = f2[0];
    R l1 = R(0), l2 = R(0);
    if constexpr (ff) {
        load_lo(l1, l2);
        f1[0] += l1;
        f2[0] += l2;
    }
    col.apply(f1, f2, gv, o1, o2, og);
#pragma unroll
    for (int k = 1; k < 9; k++) {
        o1[k] = as_stored<S>(k, o1[k]);
        o2[k] = as_stored<S>(9 + k, o2[k]);
    }
    if constexpr (ff) {
        R d1 = R(0), d2 = R(0);
#pragma unroll
        for (int k = 1; k < 9; k++) {
            d1 += f1[k] - o1[k];
            d2 += f2[k] - o2[k];
        }
        R hh1, hh2, lo1, lo2;
        rest_add(h10, l1, d1, hh1, lo1);
        rest_add(h20, l2, d2, hh2, lo2);
        store(std::integral_constant<int, 0>{}, hh1, hh2, og[0]);
        store_lo(lo1, lo2);
    } else {
        store(std::integral_constant<int, 0>{}, o1[0], o2[0], og[0]);
    }
    static_for<1, 9>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        store(kc, o1[K], o2[K], og[K]);
    });
}

// In-place form of the BGK collide_all: the post-collision populations of
// direction k land in the location the input of direction k-bar came from
// (and vice versa); collide_all already reads both inputs of an opposite pair
// before it writes either output.
template <typename S, typename R, bool UNI, typename Load, typename LoadLo, typename St, typename StLo>
__device__ __forceinline__ void collide_all_inplace(const Collider<R, UNI>& col, const R gv[9], Load load,
                                                    LoadLo load_lo, St store, StLo store_lo)
{
    collide_all<S, R>(col, gv, load, load_lo, store, store_lo);
}
// MRT already reads all nine populations before writing any.
template <typename S, typename R, typename Load, typename LoadLo, typename St, typename StLo>
__device__ __forceinline__ void collide_all_inplace(const MrtNode<R>& col, const R gv[9], Load load, LoadLo load_lo,
                                                    St store, StLo store_lo)
{
    collide_all<S, R>(col, gv, load, load_lo, store, store_lo);
}

// Per-node collision data of the BGK (MRT = false) or MRT update; UNI: the
// uniform-property form of the BGK update.
template <bool MRT, typename R, bool UNI = false>
using CollideOf = typename std::conditional<MRT, MrtNode<R>, Collider<R, UNI>>::type;

// Destinations of the push from an interior node (x, y): the neighbouring
// columns and rows, wrapped on a periodic axis (interior nodes never reach a
// non-periodic edge), so that each direction costs one add.
struct PushOffsets {
    int col[3];        // x - 1, x, x + 1 (wrapped)
    long long row[3];  // (y - 1, y, y + 1) * pitch (wrapped)
    __device__ __forceinline__ PushOffsets(const Geo& g, int x, int y)
    {
        col[0] = x > 0 ? x - 1 : g.nx - 1;
        col[1] = x;
        col[2] = x < g.nx - 1 ? x + 1 : 0;
        row[0] = (long long)(y > 0 ? y - 1 : g.ny - 1) * g.pitch;
        row[1] = (long long)y * g.pitch;
        row[2] = (long long)(y < g.ny - 1 ? y + 1 : 0) * g.pitch;
    }
    template <int K>
    __device__ __forceinline__ long long dest() const { return row[1 + ey(K)] + col[1 + ex(K)]; }
};

// ---------------------------------------------------------------------------
// K1: fused interior update, marching along a strip of columns.
//
// A block of BLOCK threads owns one column each: columns x0-2 .. x0+BLOCK-3
// of which the middle TX = BLOCK-4 are updated, over the `rows` rows of its
// segment.  Even segments march up, odd segments down, so that two adjacent
// segments read the two halo rows they share at about the same time (both
// at their start or both at their end) and the second read hits L2.  The
// iteration that reaches row r computes
//   c1, c2 of row r         (sum of the 18 order-parameter populations)
//   mu1, mu2 of row r - dir (needs c rows r - 2 dir .. r)
//   update of row r - 2 dir (needs c and mu rows around it)
// with each column's recent c and mu kept by its own thread and the column
// sums its neighbours need in shared memory (ColRings), so each order
// parameter is summed once per node (plus a 4-column, 4-row halo per block)
// and no c or mu array ever reaches HBM.
// ---------------------------------------------------------------------------

// Column sums of the two-buffer interior tile.  For one row r of an order
// parameter c and each column j of the strip:
//   A_j = c(j, r-1) + 4 c(j, r) + c(j, r+1),   D_j = c(j, r+1) - c(j, r-1),
// from which the scaled stencils of Eq. 20 at (j, r) need only the two
// neighbouring columns:
//   12 d_x c = A_{j+1} - A_{j-1},   12 d_y c = D_{j-1} + 4 D_j + D_{j+1},
//   6 lap c  = A_{j-1} + A_{j+1} + 4 (c(j, r-1) + c(j, r+1) - 5 c(j, r)).
// Each thread forms them for its own column from the c values it summed
// itself (kept in registers), so every stencil costs a few operations per
// node and the 3x3 neighbourhood is never gathered.  A and D of row r live in
// slot (r + 9) % 3: written in phase 1 of one iteration, read in phase 2 of
// that iteration (after its barrier) and in phase 3 of the next, and replaced
// in phase 1 two iterations after that, which follows the barrier every
// thread passes only once it has finished the last read.  M: the A of mu for
// the row being updated (the general update's lap mu), written and read in
// the same iteration, so the general update needs a second barrier.
// The two order parameters' sums of a column share one 2-vector, so a thread
// writes A (or D) of both in one shared store and reads them in one load.
template <typename R>
struct Vec2T;
template <>
struct Vec2T<float> {
    using type = float2;
};
template <>
struct Vec2T<double> {
    using type = double2;
};

template <typename R, int BLOCK>
struct ColRings {
    using V = typename Vec2T<R>::type;
    V A[3][BLOCK], D[3][BLOCK], M[BLOCK];  // (.x, .y) = order parameter 1, 2
    __device__ __forceinline__ void put_ad(int sl, int j, R a1, R a2, R d1, R d2)
    {
        A[sl][j] = V{a1, a2};
        D[sl][j] = V{d1, d2};
    }
    __device__ __forceinline__ void put_m(int j, R m1, R m2) { M[j] = V{m1, m2}; }
    __device__ __forceinline__ V a(int sl, int j) const { return A[sl][j]; }
    __device__ __forceinline__ V d(int sl, int j) const { return D[sl][j]; }
    __device__ __forceinline__ V m(int j) const { return M[j]; }
};

// Per-thread copy of the 18 order-parameter populations (and the two rest lo
// parts) that phase 1 reads for the c sums of a row, kept until the same
// thread updates that row two iterations later (row r in slot (r + 9) % 3).
// The 20 values of a column and row sit in five 4-vectors, in the order the
// collision reads them: vector p holds f^1, f^2 of direction pair_dir(p) and
// of its opposite, vector 4 the rest populations and their lo parts; one
// shared store or load moves four values (FP32 arithmetic only).  With the
// 2-vector column sums: 39 shared-memory instructions per node fewer than one
// per value; GB300, 2048^2, FP32 storage 19.91 -> 20.01, BF16 26.95 -> 27.20
// G node updates/s, FP16 and FP64 unchanged.
template <typename R, int BLOCK>
struct PopStash {
    float4 v[3][5][BLOCK];
};
__host__ __device__ constexpr int stash_vec(int k)
{
    int p = 4;
    for (int i = 0; i < 4; i++)
        if (pair_dir(i) == k || opp(pair_dir(i)) == k) p = i;
    return k == 0 ? 4 : p;
}
__host__ __device__ constexpr bool stash_hi(int k) { return k != 0 && pair_dir(stash_vec(k)) != k; }
static_assert(stash_vec(0) == 4 && stash_vec(1) == 0 && stash_vec(3) == 0 && stash_vec(6) == 3 && stash_hi(6) &&
                  !stash_hi(8) && stash_hi(4) && !stash_hi(2),
              "stash slots follow the collision's direction pairs");
// Used by the FP32-arithmetic BGK interior kernels (single lattices and
// batches): 5% faster FP32 and 2% faster FP16 on the 2048^2 lattice than
// re-reading the populations through the cache.
#ifndef TLB_STASH32
#define TLB_STASH32 1
#endif
constexpr bool kStashPops = TLB_STASH32 != 0;
// FP32 storage loads the order-parameter populations of the next c row one
// iteration ahead (register double buffering, at 4 blocks per SM): GB300,
// 2048^2, 18.6 -> 19.8 G node updates/s; 16-bit storage, with half the bytes
// per load, measured slower with it (22.8 -> 22.5 at 5 blocks, 20.2 at 4).
#ifndef TLB_PIPE32
#define TLB_PIPE32 1
#endif
constexpr bool kPipeRows = TLB_PIPE32 != 0;
// 16-bit storage: the same one-row-ahead loads, kept as the words loaded (8
// pair words and 4 FP32 rest parts, 12 registers) and decoded when consumed:
// GB300, 2048^2, 5 blocks per SM: FP16 23.0 -> 25.4, BF16 24.0 -> 26.5 G node
// updates/s (at 4 blocks per SM 24.2).
#ifndef TLB_PIPE16R
#define TLB_PIPE16R 1
#endif
constexpr bool kPipeRows16 = TLB_PIPE16R != 0;
// With the one-row-ahead loads, the g populations and c_i u of the next
// iteration's update row are loaded one iteration ahead as well (as stored,
// 13 registers): 16-bit storage, GB300, 2048^2, 5 blocks per SM: FP16 25.3 ->
// 26.1, BF16 26.6 -> 27.2 G node updates/s.
#ifndef TLB_PIPEG16
#define TLB_PIPEG16 1
#endif
constexpr bool kPipeG16 = TLB_PIPEG16 != 0;
// (FP32 storage, at 4 blocks per SM: 19.9 -> 19.4, so off there)
#ifndef TLB_PIPEG32
#define TLB_PIPEG32 0
#endif
constexpr bool kPipeG32 = TLB_PIPEG32 != 0;

// One row of the order-parameter populations of a 16-bit buffer as loaded.
struct Raw16Row {
    unsigned w[8];
    float r[2], l[2];
};

// One tile: strip bx (columns bx*(BLOCK-4) .. +BLOCK-5), segment by (rows
// by*rows .. +rows-1, marching up for even by and down for odd by).
template <typename S, typename R, int BLOCK, bool PREFETCH, bool MRT, bool UNI = false, bool STASH = false>
__device__ __forceinline__ void interior_tile(const S* __restrict__ fA, S* __restrict__ fB, CuT<S>* __restrict__ cu,
                                              const uint8_t* __restrict__ cls, const Geo& g, const Prm<R>& P,
                                              int bx, int by, int rows, ColRings<R, BLOCK>& sh,
                                              PopStash<R, BLOCK>* stash = nullptr)
{
    const long long PL = g.plane;
    const int t = threadIdx.x;
    // the BGK update of FP16 storage works in the units the populations are
    // stored in (2^kF16ScaleExp times their value)
    constexpr int SE = (Store<S>::k16 && !MRT) ? Store<S>::kScaleExp : 0;
    const int x0 = bx * (BLOCK - 4);
    const int xs = x0 - 2 + t;  // this thread's column, in [-2, nx + BLOCK]
    // wrapped column (periodic x) and whether it holds data at all; only
    // columns -2 .. nx+1 are ever read
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
    // this column's c of rows yc, yc - dir, yc - 2 dir and mu of rows ym,
    // ym - dir, ym - 2 dir (index 0 the newest)
    R ca[3] = {R(0), R(0), R(0)}, cb[3] = {R(0), R(0), R(0)};
    R ma[3] = {R(0), R(0), R(0)}, mb[3] = {R(0), R(0), R(0)};
    // PIPE: the 18 order-parameter populations (and the two rest lo parts) of
    // the next iteration's c row are loaded one iteration ahead, so that their
    // memory latency overlaps a whole iteration instead of stalling phase 1
    constexpr bool PIPE = STASH && kPipeRows && std::is_same<S, float>::value;
    auto load_c_row = [&](int ycr, R (&v)[18], R (&l)[2]) {
        int yw = ycr;
        bool in = col_in && ycr < g.ny + 2;
        if (ycr < 0 || ycr >= g.ny) {
            if (g.edge[2] == EDGE_PERIODIC) yw = ycr < 0 ? ycr + g.ny : ycr - g.ny;
            else in = false;
        }
        if (in) {
            const long long oc = (long long)yw * g.pitch + xw;
            v[0] = ld_pop<R>(fA, 0, PL, oc);
            v[9] = ld_pop<R>(fA, 9, PL, oc);
#pragma unroll
            for (int k = 1; k < 9; k++) ld_pair<R, true, SE != 0>(fA, k, PL, oc, v[k], v[9 + k]);
            l[0] = ld_lo<R>(fA, 0, PL, oc);
            l[1] = ld_lo<R>(fA, 1, PL, oc);
        } else {
#pragma unroll
            for (int k = 0; k < 18; k++) v[k] = R(0);
            l[0] = l[1] = R(0);
        }
    };
    R nv[18], nl[2];
    if constexpr (PIPE) load_c_row(dir > 0 ? y0 - 2 : y1 + 1, nv, nl);
    constexpr bool PIPE16 = STASH && kPipeRows16 && Store<S>::k16;
    auto load_raw_row = [&](int ycr, Raw16Row& q) {
        int yw = ycr;
        bool in = col_in && ycr < g.ny + 2;
        if (ycr < 0 || ycr >= g.ny) {
            if (g.edge[2] == EDGE_PERIODIC) yw = ycr < 0 ? ycr + g.ny : ycr - g.ny;
            else in = false;
        }
        if (in) {
            const long long oc = (long long)yw * g.pitch + xw;
            const unsigned* wp = reinterpret_cast<const unsigned*>(fA);
#pragma unroll
            for (int k = 0; k < 8; k++) q.w[k] = __ldg(wp + (long long)k * PL + oc);
            const float* rp = rest_region(fA, PL);
#pragma unroll
            for (int i = 0; i < 2; i++) {
                q.r[i] = __ldg(rp + i * PL + oc);
                q.l[i] = __ldg(rp + (2 + i) * PL + oc);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) q.w[k] = 0u;
            q.r[0] = q.r[1] = q.l[0] = q.l[1] = 0.0f;
        }
    };
    Raw16Row nq;
    if constexpr (PIPE16) load_raw_row(dir > 0 ? y0 - 2 : y1 + 1, nq);
    constexpr bool PIPEG = ((PIPE16 && kPipeG16) || (PIPE && kPipeG32)) && PREFETCH;
    typename std::conditional<Store<S>::k16, unsigned short, S>::type ngr[9];
    CuT<S> ncp[4];

    for (int it = 0; it < iters; it++) {
        const int yc = dir > 0 ? y0 - 2 + it : y1 + 1 - it;  // c row of this iteration
        const int ym = yc - dir;                              // mu row
        const int yu = yc - 2 * dir;                          // updated row
        R cv[18], cl[2];
        if constexpr (PIPE) {
#pragma unroll
            for (int k = 0; k < 18; k++) cv[k] = nv[k];
            cl[0] = nl[0];
            cl[1] = nl[1];
            if (it + 1 < iters) load_c_row(yc + dir, nv, nl);
        }
        if constexpr (PIPE16) {
            // decode this iteration's row, then issue the next one's loads
            if constexpr (Store<S>::k16) {
                constexpr float inv = SE != 0 ? 1.0f : 1.0f / float(1 << Store<S>::kScaleExp);
                cv[0] = R(nq.r[0]);
                cv[9] = R(nq.r[1]);
#pragma unroll
                for (int k = 1; k < 9; k++) {
                    const float2 v = dec16x2(S{}, nq.w[k - 1]);
                    cv[k] = R(v.x * inv);
                    cv[9 + k] = R(v.y * inv);
                }
                cl[0] = R(nq.l[0]);
                cl[1] = R(nq.l[1]);
            }
            if (it + 1 < iters) load_raw_row(yc + dir, nq);
        }
        // the update node (row yu of this column, if any): its g and c_i u
        // are the first touches of HBM, issued before its node class is
        // known (the load of the class is consumed only in phase 3, so its
        // latency overlaps phases 1 and 2; a node that is not interior was
        // read for nothing)
        const bool in_rows = updater && it >= 4;
        const long long ou = in_rows ? (long long)yu * g.pitch + xs : 0;
        const bool upd = in_rows && (cls[ou] & CLS_INTERIOR) != 0;
        R gv[9], cp[4];
        if constexpr (PIPEG) {
            if constexpr (Store<S>::k16) {
                constexpr float inv = SE != 0 ? 1.0f : 1.0f / float(1 << Store<S>::kScaleExp);
#pragma unroll
                for (int k = 0; k < 9; k++) gv[k] = R(dec16(S{}, ngr[k]) * inv);
            } else {
#pragma unroll
                for (int k = 0; k < 9; k++) gv[k] = R(ngr[k]);
            }
#pragma unroll
            for (int q = 0; q < 4; q++) cp[q] = R(ncp[q]);
            // the next iteration's update row (yu + dir), if it has one
            if (updater && it + 1 >= 4 && it + 1 < iters) {
                const long long on = (long long)(yu + dir) * g.pitch + xs;
                if constexpr (Store<S>::k16) {
                    const unsigned short* gp = reinterpret_cast<const unsigned short*>(fA);
#pragma unroll
                    for (int k = 0; k < 9; k++) ngr[k] = __ldg(gp + idx16(18 + k, PL, on));
                } else {
#pragma unroll
                    for (int k = 0; k < 9; k++) ngr[k] = __ldg(fA + (18 + k) * PL + on);
                }
#pragma unroll
                for (int q = 0; q < 4; q++) ncp[q] = __ldg(&cu[q * PL + on]);
            }
        } else if (PREFETCH && in_rows) {
#pragma unroll
            for (int k = 0; k < 9; k++) gv[k] = ld_pop<R, true, SE != 0>(fA, 18 + k, PL, ou);
#pragma unroll
            for (int q = 0; q < 4; q++) cp[q] = R(cu[q * PL + ou]);
        }
        // 1) c of row yc (Eq. 13a); column sums of row ym
        {
            int yw = yc;
            bool in = col_in && yc < g.ny + 2;
            if (yc < 0 || yc >= g.ny) {
                if (g.edge[2] == EDGE_PERIODIC) yw = yc < 0 ? yc + g.ny : yc - g.ny;
                else in = false;
            }
            R a = R(0), b = R(0);
            if (PIPE || PIPE16 || in) {
                const long long oc = (long long)yw * g.pitch + xw;
                if constexpr (STASH) {
                    R v[18], l1, l2;
                    if constexpr (PIPE || PIPE16) {
#pragma unroll
                        for (int k = 0; k < 18; k++) v[k] = cv[k];
                        l1 = cl[0];
                        l2 = cl[1];
                    } else {
                        v[0] = ld_pop<R>(fA, 0, PL, oc);
                        v[9] = ld_pop<R>(fA, 9, PL, oc);
#pragma unroll
                        for (int k = 1; k < 9; k++) ld_pair<R, true, SE != 0>(fA, k, PL, oc, v[k], v[9 + k]);
                        l1 = ld_lo<R>(fA, 0, PL, oc);
                        l2 = ld_lo<R>(fA, 1, PL, oc);
                    }
                    float4(&st)[5][BLOCK] = stash->v[(yc + 9) % 3];
                    static_for<0, 4>([&](auto pc) {
                        constexpr int K = pair_dir(decltype(pc)::value), KB = opp(K);
                        st[decltype(pc)::value][t] = make_float4(v[K], v[9 + K], v[KB], v[9 + KB]);
                    });
                    st[4][t] = make_float4(v[0], v[9], l1, l2);
                    v[0] += l1;
                    v[9] += l2;
                    a = sum9s<SE>(v);
                    b = sum9s<SE>(v + 9);
                } else {
                    order_params<R>(fA, PL, oc, a, b);
                }
            }
            ca[2] = ca[1];
            ca[1] = ca[0];
            ca[0] = a;
            cb[2] = cb[1];
            cb[1] = cb[0];
            cb[0] = b;
            if (it >= 2) {
                // row ym = yc - dir: its rows ym - 1, ym + 1 are ca[0], ca[2]
                // in the order of the march
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
                // column sums of mu for row yu = ym - dir (the general update's lap mu)
                sh.put_m(t, fma(R(4), ma[1], ma[0] + ma[2]), fma(R(4), mb[1], mb[0] + mb[2]));
            }
        }
        // (only the general update's M needs this barrier; the rings of A and
        // D need one per iteration.  Without it in the uniform update, GB300,
        // 2048^2: FP16 27.15 -> 26.75, BF16 27.17 -> 26.77 G node updates/s,
        // FP32 unchanged: the warps of a block drifting apart cost more than
        // the barrier)
        __syncthreads();
        // 3) update of row yu
        if (!upd) continue;
        Macro<R> m;
        {
            // c(yu) = ca[2]; mu(yu) = ma[1] (mu rows yu + dir, yu - dir: ma[0], ma[2])
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
                m.lm1 = m.lm2 = R(0);  // F_a vanishes with equal densities
            } else {
                const auto ml = sh.m(t - 1), mr = sh.m(t + 1);
                m.lm1 = fma(R(4), fma(R(-5), ma[1], ma[0] + ma[2]), ml.x + mr.x);
                m.lm2 = fma(R(4), fma(R(-5), mb[1], mb[0] + mb[2]), ml.y + mr.y);
            }
            m.rho = UNI ? P.rho[2] : density(P, m.c1, m.c2);
        }
        if (!PREFETCH) {
#pragma unroll
            for (int k = 0; k < 9; k++) gv[k] = ld_pop<R, true, SE != 0>(fA, 18 + k, PL, ou);
#pragma unroll
            for (int q = 0; q < 4; q++) cp[q] = R(cu[q * PL + ou]);
        }
        Hydro<R> h;
        hydro_from_g<UNI, SE>(P, m, gv, h);
        // Eq. 19: d/dt (c_i u) against the stored product of the previous step
        const R c1ux = m.c1 * h.ux, c1uy = m.c1 * h.uy, c2ux = m.c2 * h.ux, c2uy = m.c2 * h.uy;
        cu[0 * PL + ou] = CuT<S>(c1ux);
        cu[1 * PL + ou] = CuT<S>(c1uy);
        cu[2 * PL + ou] = CuT<S>(c2ux);
        cu[3 * PL + ou] = CuT<S>(c2uy);
        CollideOf<MRT, R, UNI> col;
        col.template build<SE>(P, m, h, c1ux - cp[0], c1uy - cp[1], c2ux - cp[2], c2uy - cp[3]);
        const PushOffsets po(g, xs, yu);
        const int su = (yu + 9) % 3;
        collide_all<S, R, SE>(col, gv,
            [&](auto kc, R& f1k, R& f2k) {
                constexpr int K = decltype(kc)::value;
                if constexpr (STASH) {
                    const float4 sv = stash->v[su][stash_vec(K)][t];
                    f1k = stash_hi(K) ? sv.z : sv.x;
                    f2k = stash_hi(K) ? sv.w : sv.y;
                } else {
                    if constexpr (K == 0) {
                        f1k = ld_pop<R>(fA, 0, PL, ou);
                        f2k = ld_pop<R>(fA, 9, PL, ou);
                    } else {
                        ld_pair<R, true, SE != 0>(fA, K, PL, ou, f1k, f2k);
                    }
                }
            },
            [&](R& l1, R& l2) {
                if constexpr (STASH) {
                    const float4 sv = stash->v[su][4][t];
                    l1 = sv.z;
                    l2 = sv.w;
                } else {
                    l1 = ld_lo<R>(fA, 0, PL, ou);
                    l2 = ld_lo<R>(fA, 1, PL, ou);
                }
            },
            [&](auto kc, auto o1, auto o2, auto og) {
                constexpr int K = decltype(kc)::value;
                const long long d = (K == 0) ? ou : po.template dest<K>();
                st_three(fB, K, PL, d, o1, o2, og);
            },
            [&](R l1, R l2) {
                st_lo(fB, 0, PL, ou, l1);
                st_lo(fB, 1, PL, ou, l2);
            });
    }
}

template <typename S, typename R, int BLOCK, int ROWS, bool PREFETCH, int MINB, bool MRT, bool UNI>
__global__ void __launch_bounds__(BLOCK, MINB)
k_step_interior(const S* __restrict__ fA, S* __restrict__ fB, CuT<S>* __restrict__ cu,
                const uint8_t* __restrict__ cls, Geo g, Prm<R> P, int rows)
{
    __shared__ ColRings<R, BLOCK> sh;
    if constexpr (kStashPops && std::is_same<R, float>::value && !MRT) {
        __shared__ PopStash<R, BLOCK> stash;
        interior_tile<S, R, BLOCK, PREFETCH, MRT, UNI, true>(fA, fB, cu, cls, g, P, blockIdx.x, blockIdx.y, rows, sh,
                                                            &stash);
    } else {
        interior_tile<S, R, BLOCK, PREFETCH, MRT, UNI>(fA, fB, cu, cls, g, P, blockIdx.x, blockIdx.y, rows, sh);
    }
}

// ---------------------------------------------------------------------------
// Generic per-node macros with the wall rules (5x5 window of c, 3x3 of mu).
// CF(off, c1, c2) fetches the order parameters of an inside node.
// ---------------------------------------------------------------------------
template <typename R, typename CF>
__device__ __forceinline__ void window_macros(const Geo& g, const uint8_t* __restrict__ cls, const Prm<R>& P,
                                              int x, int y, CF cf, Macro<R>& m)
{
    R wc1[5][5], wc2[5][5];
    int wk[5][5];
#pragma unroll
    for (int j = 0; j < 5; j++) {
#pragma unroll
        for (int i = 0; i < 5; i++) {
            long long off = 0;
            const int s = site_of(g, cls, x + i - 2, y + j - 2, off);
            wk[j][i] = s;
            R a = R(0), b = R(0);
            if (s == ST_FLUID) cf(off, a, b);
            wc1[j][i] = a;
            wc2[j][i] = b;
        }
    }
    // lid row: c is that of the node below (Eqs. 51-53 reading)
#pragma unroll
    for (int j = 1; j < 5; j++) {
#pragma unroll
        for (int i = 0; i < 5; i++) {
            if (wk[j][i] == ST_LID) {
                wc1[j][i] = wc1[j - 1][i];
                wc2[j][i] = wc2[j - 1][i];
            }
        }
    }
    // mu on the 3x3 around the node (Eq. 8), wetting ghosts of Eq. 42
    R wm1[3][3], wm2[3][3];
#pragma unroll
    for (int j = 1; j < 4; j++) {
#pragma unroll
        for (int i = 1; i < 4; i++) {
            R mu1 = R(0), mu2 = R(0);
            if (wk[j][i] == ST_FLUID) {
                const R cc1 = wc1[j][i], cc2 = wc2[j][i];
                R o1, o2;
                wet_offset(P, cc1, cc2, o1, o2);
                R v1[9], v2[9];
                v1[0] = cc1;
                v2[0] = cc2;
#pragma unroll
                for (int k = 1; k < 9; k++) {
                    const int s = wk[j + ey(k)][i + ex(k)];
                    if (fluidlike(s)) {
                        v1[k] = wc1[j + ey(k)][i + ex(k)];
                        v2[k] = wc2[j + ey(k)][i + ex(k)];
                    } else if (s == ST_WET) {
                        v1[k] = cc1 + o1;
                        v2[k] = cc2 + o2;
                    } else {
                        v1[k] = cc1;
                        v2[k] = cc2;
                    }
                }
                chem_pot(P, cc1, cc2, lap9s(v1), lap9s(v2), mu1, mu2);
            }
            wm1[j - 1][i - 1] = mu1;
            wm2[j - 1][i - 1] = mu2;
        }
    }
#pragma unroll
    for (int j = 1; j < 3; j++) {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            if (wk[j + 1][i + 1] == ST_LID) {
                wm1[j][i] = wm1[j - 1][i];
                wm2[j][i] = wm2[j - 1][i];
            }
        }
    }
    // gradients at the centre with symmetric ghosts (Eq. 43)
    R v1[9], v2[9], w1[9], w2[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const int s = k == 0 ? ST_FLUID : wk[2 + ey(k)][2 + ex(k)];
        const bool use = fluidlike(s);
        v1[k] = use ? wc1[2 + ey(k)][2 + ex(k)] : wc1[2][2];
        v2[k] = use ? wc2[2 + ey(k)][2 + ex(k)] : wc2[2][2];
        w1[k] = use ? wm1[1 + ey(k)][1 + ex(k)] : wm1[1][1];
        w2[k] = use ? wm2[1 + ey(k)][1 + ex(k)] : wm2[1][1];
    }
    m.c1 = wc1[2][2];
    m.c2 = wc2[2][2];
    m.mu1 = wm1[1][1];
    m.mu2 = wm2[1][1];
    grad9s(v1, m.g1x, m.g1y);
    grad9s(v2, m.g2x, m.g2y);
    m.lm1 = lap9s(w1);
    m.lm2 = lap9s(w2);
    m.rho = density(P, m.c1, m.c2);
}

template <typename S, typename R>
struct DistFetch {
    const S* f;
    long long PL;
    __device__ __forceinline__ void operator()(long long off, R& a, R& b) const
    {
        order_params<R>(f, PL, off, a, b);
    }
};

// c_1, c_2 from dense FP64 row arrays holding rows y_b .. y_b + rows - 1 of
// the lattice (y_b may be negative; rows outside 0 .. ny-1 hold the wrapped
// rows of a periodic y axis); the whole lattice is y_b = 0, rows = ny.
template <typename R>
struct FieldFetch {
    const double* c1;
    const double* c2;
    int nx, pitch, ny, y_b, rows;
    __device__ __forceinline__ void operator()(long long off, R& a, R& b) const
    {
        const long long y = off / pitch, x = off - y * pitch;
        long long r = y - y_b;
        if (r < 0) r += ny;
        if (r >= rows) r -= ny;
        a = R(c1[r * nx + x]);
        b = R(c2[r * nx + x]);
    }
};

// c_1, c_2 from the two order-parameter planes of the in-place update
template <typename R>
struct PlaneFetch {
    const R* c;  // c_1 plane, then c_2 plane (pitched)
    long long PL;
    __device__ __forceinline__ void operator()(long long off, R& a, R& b) const
    {
        a = c[off];
        b = c[PL + off];
    }
};

// Push of one post-collision triple along direction K from node (x, y) with
// the wall rules: into a fluid node, back into slot K-bar on a solid link
// (Eq. 44), or out through the lid.
template <int K, typename S, typename V1, typename V2, typename VG>
__device__ __forceinline__ void push_wall(const Geo& g, const uint8_t* __restrict__ cls, S* __restrict__ fB,
                                          int x, int y, long long o, V1 o1, V2 o2, VG og)
{
    const long long PL = g.plane;
    if constexpr (K == 0) {
        st_pop(fB, 0, PL, o, o1);
        st_pop(fB, 9, PL, o, o2);
        st_pop(fB, 18, PL, o, og);
        return;
    }
    long long d = 0;
    const int s = site_of(g, cls, x + ex(K), y + ey(K), d);
    if (fluidlike(s)) {
        st_three(fB, K, PL, d, o1, o2, og);
    } else if (s == ST_WET || s == ST_NEUTRAL) {
        st_three(fB, opp(K), PL, o, o1, o2, og);
    }
}

// ---------------------------------------------------------------------------
// K2: near-wall and lid nodes from the compacted list.
// ---------------------------------------------------------------------------
template <typename S, typename R, bool MRT>
__device__ __forceinline__ void wall_node(const S* __restrict__ fA, S* __restrict__ fB, CuT<S>* __restrict__ cu,
                                          const uint8_t* __restrict__ cls, const Geo& g, const Prm<R>& P,
                                          uint32_t packed)
{
    const int x = (int)(packed & 0xffffu), y = (int)(packed >> 16);
    const long long PL = g.plane;
    const long long o = (long long)y * g.pitch + x;
    const int kind = cls[o] & CLS_KIND_MASK;
    DistFetch<S, R> fetch{fA, PL};

    if (kind == ST_FLUID) {
        Macro<R> m;
        window_macros(g, cls, P, x, y, fetch, m);
        R gv[9];
#pragma unroll
        for (int k = 0; k < 9; k++) gv[k] = ld_pop<R>(fA, 18 + k, PL, o);
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
        collide_all<S, R>(col, gv,
            [&](auto kc, R& f1k, R& f2k) {
                constexpr int K = decltype(kc)::value;
                f1k = ld_pop<R>(fA, K, PL, o);
                f2k = ld_pop<R>(fA, 9 + K, PL, o);
            },
            [&](R& l1, R& l2) {
                l1 = ld_lo<R>(fA, 0, PL, o);
                l2 = ld_lo<R>(fA, 1, PL, o);
            },
            [&](auto kc, auto o1, auto o2, auto og) {
                constexpr int K = decltype(kc)::value;
                push_wall<K>(g, cls, fB, x, y, o, o1, o2, og);
            },
            [&](R l1, R l2) {
                st_lo(fB, 0, PL, o, l1);
                st_lo(fB, 1, PL, o, l2);
            });
    } else if (kind == ST_LID) {
        // x_f is the node below; x_u takes its macros and gradients, u = (U0, 0)
        const long long of = o - g.pitch;
        Macro<R> m;
        window_macros(g, cls, P, x, y - 1, fetch, m);
        R gf[9];
#pragma unroll
        for (int k = 0; k < 9; k++) gf[k] = ld_pop<R>(fA, 18 + k, PL, of);
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
            R ff1 = ld_pop<R>(fA, k, PL, of), ff2 = ld_pop<R>(fA, 9 + k, PL, of);
            if constexpr (Store<S>::kLo) {
                if (k == 0) {
                    ff1 += ld_lo<R>(fA, 0, PL, of);
                    ff2 += ld_lo<R>(fA, 1, PL, of);
                }
            }
            f1u[k] = e1u + (ff1 - e1f);
            f2u[k] = e2u + (ff2 - e2f);
            gu[k] = egu + (gf[k] - egf);
        }
        collide_all<S, R>(col, gu,
            [&](auto kc, R& f1k, R& f2k) {
                constexpr int K = decltype(kc)::value;
                f1k = f1u[K];
                f2k = f2u[K];
            },
            [&](R& l1, R& l2) {
                l1 = R(0);
                l2 = R(0);
            },
            [&](auto kc, auto o1, auto o2, auto og) {
                constexpr int K = decltype(kc)::value;
                push_wall<K>(g, cls, fB, x, y, o, o1, o2, og);
                // slots fed from beyond the lid receive nothing: keep them zero
                if constexpr (ey(K) == -1) {
                    long long dummy = 0;
                    if (site_of(g, cls, x - ex(K), y + 1, dummy) == ST_VOID) {
                        st_pop(fB, K, PL, o, R(0));
                        st_pop(fB, 9 + K, PL, o, R(0));
                        st_pop(fB, 18 + K, PL, o, R(0));
                    }
                }
            },
            [&](R l1, R l2) {
                st_lo(fB, 0, PL, o, l1);
                st_lo(fB, 1, PL, o, l2);
            });
    }
}

template <typename S, typename R, bool MRT>
__global__ void __launch_bounds__(128)
k_step_wall(const S* __restrict__ fA, S* __restrict__ fB, CuT<S>* __restrict__ cu,
            const uint8_t* __restrict__ cls, const uint32_t* __restrict__ list, int nlist, Geo g, Prm<R> P)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nlist) return;
    wall_node<S, R, MRT>(fA, fB, cu, cls, g, P, list[t]);
}

// ---------------------------------------------------------------------------
// Set-up: f = f^eq(c, mu(c), u), g = g^eq(p, rho(c), u), cu = c u, for rows
// y0 .. y0 + gridDim.y - 1.  ux, uy, p are dense FP64 rows from y0 on; c1, c2
// dense FP64 rows y_b .. y_b + rows - 1 (wrapped), which must cover the
// radius-2 window of every updated row (radius 3 around a lid row, whose
// window is centred on the row below).  The whole lattice: y0 = y_b = 0,
// rows = ny.
// ---------------------------------------------------------------------------
template <typename S, typename R>
__global__ void k_init(S* __restrict__ fA, CuT<S>* __restrict__ cu, const uint8_t* __restrict__ cls,
                       const double* __restrict__ c1, const double* __restrict__ c2,
                       const double* __restrict__ ux, const double* __restrict__ uy,
                       const double* __restrict__ p, Geo g, Prm<R> P, int y0, int y_b, int rows)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y;
    if (x >= g.nx) return;
    const long long PL = g.plane;
    const long long o = (long long)y * g.pitch + x;
    const long long n = (long long)blockIdx.y * g.nx + x;  // ux, uy, p hold rows y0 ..
    const int kind = cls[o] & CLS_KIND_MASK;
    st_lo(fA, 0, PL, o, R(0));
    st_lo(fA, 1, PL, o, R(0));
    if (!fluidlike(kind)) {
        for (int q = 0; q < 27; q++) st_pop(fA, q, PL, o, R(0));
        for (int q = 0; q < 4; q++) cu[q * PL + o] = CuT<S>(0);
        return;
    }
    FieldFetch<R> fetch{c1, c2, g.nx, g.pitch, g.ny, y_b, rows};
    Macro<R> m;
    window_macros(g, cls, P, x, kind == ST_LID ? y - 1 : y, fetch, m);
    const R u = R(ux[n]), v = R(uy[n]);
    const R pp = p ? R(p[n]) : R(0);
    for (int k = 0; k < 9; k++) {
        R e1, e2, eg;
        equilibria(k, P, m.c1, m.c2, m.mu1, m.mu2, m.rho, pp, u, v, e1, e2, eg);
        st_pop(fA, k, PL, o, e1);
        st_pop(fA, 9 + k, PL, o, e2);
        st_pop(fA, 18 + k, PL, o, eg);
    }
    cu[0 * PL + o] = CuT<S>(m.c1 * u);
    cu[1 * PL + o] = CuT<S>(m.c1 * v);
    cu[2 * PL + o] = CuT<S>(m.c2 * u);
    cu[3 * PL + o] = CuT<S>(m.c2 * v);
}

// ---------------------------------------------------------------------------
// Read-out of macroscopic fields as FP64 planes (order c1 c2 c3 rho ux uy p
// mu1 mu2 mu3, only the planes selected by `mask`).
// ---------------------------------------------------------------------------
template <typename S, typename R>
__global__ void k_read_fields(const S* __restrict__ fA, const uint8_t* __restrict__ cls, double* __restrict__ out,
                              uint32_t mask, Geo g, Prm<R> P)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= g.nx) return;
    const long long PL = g.plane;
    const long long o = (long long)y * g.pitch + x;
    const long long n = (long long)y * g.nx + x;
    const long long N = (long long)g.nx * g.ny;
    const int kind = cls[o] & CLS_KIND_MASK;
    double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (fluidlike(kind)) {
        DistFetch<S, R> fetch{fA, PL};
        const long long of = kind == ST_LID ? o - g.pitch : o;
        Macro<R> m;
        window_macros(g, cls, P, x, kind == ST_LID ? y - 1 : y, fetch, m);
        R gv[9];
        for (int k = 0; k < 9; k++) gv[k] = ld_pop<R>(fA, 18 + k, PL, of);
        Hydro<R> h;
        hydro_from_g(P, m, gv, h);
        if (kind == ST_LID) {
            h.ux = P.lid_u;
            h.uy = R(0);
        }
        const R mu3 = -fma(P.l3_l1, m.mu1, P.l3_l2 * m.mu2);
        v[0] = m.c1;
        v[1] = m.c2;
        v[2] = R(1) - m.c1 - m.c2;
        v[3] = m.rho;
        v[4] = h.ux;
        v[5] = h.uy;
        v[6] = h.p;
        v[7] = m.mu1;
        v[8] = m.mu2;
        v[9] = mu3;
    }
    int plane = 0;
    for (int q = 0; q < 10; q++) {
        if (mask & (1u << q)) {
            out[plane * N + n] = v[q];
            plane++;
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 mass totals: per-block partial sums in a fixed order, then one block
// sums the partials in a fixed order (deterministic).  part[b*4 + 0..3] =
// sum c1, sum c2, sum c3, non-finite count.
// ---------------------------------------------------------------------------
template <typename S, typename R>
__global__ void __launch_bounds__(256)
k_mass_partials(const S* __restrict__ fA, const uint8_t* __restrict__ cls, double* __restrict__ part, Geo g)
{
    __shared__ double red[4][256];
    const long long PL = g.plane;
    const long long N = (long long)g.nx * g.ny;
    double s1 = 0, s2 = 0, s3 = 0, bad = 0;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(n / g.nx), x = (int)(n - (long long)y * g.nx);
        long long o = (long long)y * g.pitch + x;
        const int kind = cls[o] & CLS_KIND_MASK;
        if (!fluidlike(kind)) continue;
        if (kind == ST_LID) o -= g.pitch;
        double v[18], gs = 0;
        for (int k = 0; k < 18; k++) v[k] = ld_pop<double>(fA, k, PL, o);
        v[0] += ld_lo<double>(fA, 0, PL, o);
        v[9] += ld_lo<double>(fA, 1, PL, o);
        for (int k = 0; k < 9; k++) gs += ld_pop<double>(fA, 18 + k, PL, o);
        const double c1 = sum9(v), c2 = sum9(v + 9);
        s1 += c1;
        s2 += c2;
        s3 += 1.0 - c1 - c2;
        if (!isfinite(c1) || !isfinite(c2) || !isfinite((double)gs)) bad += 1.0;
    }
    red[0][threadIdx.x] = s1;
    red[1][threadIdx.x] = s2;
    red[2][threadIdx.x] = s3;
    red[3][threadIdx.x] = bad;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; q++) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x][0];
}

static __global__ void __launch_bounds__(256) k_mass_final(const double* __restrict__ part, int nparts, double* __restrict__ out)
{
    __shared__ double red[4][256];
    double s[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x)
        for (int q = 0; q < 4; q++) s[q] += part[b * 4 + q];
    for (int q = 0; q < 4; q++) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; q++) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace tlb

namespace tlb {

// ---------------------------------------------------------------------------
// Contact-line diagnostic (Sec. III.A: theta_n = 2 atan(2 H_d / L_s)), in
// FP64 on the wall row y = 0.  Per column: the order parameter c_comp on the
// wall row, and the height of the c = 1/2 crossing reached by walking up from
// the wall through nodes with c >= 1/2 (linear interpolation), plus 1/2 for the
// half-way wall; -1 where the wall node is outside a drop.
// ---------------------------------------------------------------------------
template <typename S>
__global__ void k_contact_columns(const S* __restrict__ fA, const uint8_t* __restrict__ cls, int comp,
                                  double* __restrict__ wallc, double* __restrict__ colh, Geo g)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.nx) return;
    const long long PL = g.plane;
    const int base = comp == 1 ? 0 : 9;
    auto cval = [&](int y) {
        const long long o = (long long)y * g.pitch + x;
        const int kind = cls[o] & CLS_KIND_MASK;
        if (!fluidlike(kind)) return 0.0;
        const long long src = kind == ST_LID ? o - g.pitch : o;  // the lid row carries the row below
        double v[9];
        for (int k = 0; k < 9; k++) v[k] = ld_pop<double>(fA, base + k, PL, src);
        v[0] += ld_lo<double>(fA, comp == 1 ? 0 : 1, PL, src);
        return sum9(v);
    };
    const double c0 = cval(0);
    wallc[x] = c0;
    if (!(c0 >= 0.5)) {
        colh[x] = -1.0;
        return;
    }
    int y = 0;
    double cy = c0, cn = 0.0;
    while (y + 1 < g.ny) {
        cn = cval(y + 1);
        if (!(cn >= 0.5)) break;
        y++;
        cy = cn;
    }
    const double h = (y + 1 < g.ny) ? y + (cy - 0.5) / (cy - cn) : (double)y;
    colh[x] = h + 0.5;
}

// Film thickness above a solid (Sec. III.D, the film on top of the cylinder):
// in column x, starting at the fluid node above the solid node y_top (the
// half-way wall at y_top + 1/2), walk up through nodes whose selected order
// parameter sum (comps bit 0: c1, bit 1: c2) is >= 1/2; the film thickness is
// the c = 1/2 crossing (linear interpolation) minus y_top + 1/2, in FP64;
// 0 where the first node is below 1/2; up to row ny - 1 where it never drops.
template <typename S>
__global__ void k_film(const S* __restrict__ fA, const uint8_t* __restrict__ cls, int x, int y_top, int comps,
                       double* __restrict__ out, Geo g)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const long long PL = g.plane;
    auto cval = [&](int y) {
        const long long o = (long long)y * g.pitch + x;
        const int kind = cls[o] & CLS_KIND_MASK;
        if (!fluidlike(kind)) return 0.0;
        const long long src = kind == ST_LID ? o - g.pitch : o;
        double s = 0.0;
        for (int i = 0; i < 2; i++) {
            if (!(comps & (1 << i))) continue;
            double v[9];
            for (int k = 0; k < 9; k++) v[k] = ld_pop<double>(fA, 9 * i + k, PL, src);
            v[0] += ld_lo<double>(fA, i, PL, src);
            s += sum9(v);
        }
        return s;
    };
    int y = y_top + 1;
    double cy = cval(y);
    if (!(cy >= 0.5)) {
        out[0] = 0.0;
        return;
    }
    double cn = 0.0;
    while (y + 1 < g.ny) {
        cn = cval(y + 1);
        if (!(cn >= 0.5)) break;
        y++;
        cy = cn;
    }
    const double top = (y + 1 < g.ny) ? y + (cy - 0.5) / (cy - cn) : (double)y;
    out[0] = top - (y_top + 0.5);
}

// One thread: the c >= 1/2 segments of the (periodic) wall row, with their
// crossings, base length L_s, height H_d (largest column height over the
// segment) and theta_n.  out[4*i + 0..3] = L_s, H_d, theta_n (degrees), x_mid.
static __global__ void k_contact_scan(const double* __restrict__ wallc, const double* __restrict__ colh, int nx,
                                      double* __restrict__ out, int max_drops, int* __restrict__ count)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int start = -1;
    for (int i = 0; i < nx; i++)
        if (!(wallc[i] >= 0.5)) {
            start = i;
            break;
        }
    int n = 0;
    if (start >= 0) {
        auto r = [&](int i) { return wallc[(i + start) % nx]; };
        int i = 0;
        while (i < nx) {
            if (!(r(i) >= 0.5)) {
                i++;
                continue;
            }
            const int a = i;
            while (i < nx && r(i) >= 0.5) i++;
            const int b = i - 1;
            const double xl = (a - 1) + (0.5 - r(a - 1)) / (r(a) - r(a - 1));
            const double rb1 = wallc[(b + 1 + start) % nx];
            const double xr = b + (r(b) - 0.5) / (r(b) - rb1);
            double H = 0.0;
            for (int xx = a; xx <= b; xx++) H = fmax(H, colh[(xx + start) % nx]);
            const double Ls = xr - xl;
            if (n < max_drops) {
                out[4 * n + 0] = Ls;
                out[4 * n + 1] = H;
                out[4 * n + 2] = 2.0 * atan(2.0 * H / Ls) * (180.0 / 3.14159265358979323846);
                out[4 * n + 3] = fmod((xl + xr) / 2 + start, (double)nx);
            }
            n++;
        }
    }
    *count = n;
}

}  // namespace tlb

// Device-side building blocks of the ternary phase-field lattice Boltzmann
// update (Liang et al., arXiv:1710.09534, Sec. II): D2Q9 constants, node
// classification, the isotropic stencils of Eqs. 20a/20b, the chemical
// potential of Eq. 8, the wetting ghost offset of Eq. 42, and the BGK
// collide-and-push of Eqs. 1a, 1b, 2a, 2b, 4, 11a, 11b with half-way
// bounce-back (Eq. 44).
//
// Layout in HBM (structure of arrays, x fastest, rows padded to `pitch`):
//   dist[p][y][x], p = 0..8 f^1_k, 9..17 f^2_k, 18..26 g_k   (two buffers)
//   cu[q][y][x],   q = 0..3: c1 ux, c1 uy, c2 ux, c2 uy of the previous step
//   cls[y][x]:     node kind (bits 0-2) | interior flag (bit 3)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tlb {

// ---- D2Q9 (Eq. 10): e_1..4 axis, e_5..8 diagonal -------------------------
__host__ __device__ constexpr int ex(int k) { return (k == 1 || k == 5 || k == 8) ? 1 : ((k == 3 || k == 6 || k == 7) ? -1 : 0); }
__host__ __device__ constexpr int ey(int k) { return (k == 2 || k == 5 || k == 6) ? 1 : ((k == 4 || k == 7 || k == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : (k <= 4 ? ((k + 1) % 4) + 1 : ((k - 3) % 4) + 5); }
__host__ __device__ constexpr double wk(int k) { return k == 0 ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

// Site kinds (same semantics as the FP64 oracle's classification).
enum : int { ST_FLUID = 0, ST_LID = 1, ST_WET = 2, ST_NEUTRAL = 3, ST_VOID = 4 };
enum : int { EDGE_PERIODIC = 0, EDGE_WETTING = 1, EDGE_NEUTRAL = 2, EDGE_LID = 3 };
enum : uint8_t { CLS_KIND_MASK = 7, CLS_INTERIOR = 8 };

struct Geo {
    int nx, ny, pitch;
    int edge[4];  // left, right, bottom, top
    long long plane;  // elements per plane = ny * pitch
};

// Derived constants, computed on the host from tlb_params.
template <typename R>
struct Prm {
    R lam[3], lamT;
    R k12D;           // 12 / D
    R k34D;           // 3/4 D
    R k4D;            // 4 / D (Eq. 42 with dx = 1)
    R eta[2];         // eta_i = M_i / (cs^2 (tau_i - 1/2))
    R inv_tau[2];     // 1 / tau_i
    R src_f[2];       // (1 - 1/(2 tau_i)) * 3 (Eq. 11a with 1/cs^2)
    R rho[3], nu[3];
    R aM[2];          // (rho_i - rho_3) M_i (Eq. 12)
    R l3_l1, l3_l2;   // lambda_3 / lambda_i (mu_3 from sum mu_i / lambda_i = 0)
    R cos12, cos13, cos23;
    R gx, gy;
    R lid_u;
};

// Site of (x, y), possibly outside the lattice; on an inside site sets the
// wrapped element offset.  `cls` is the node-class map (kind in bits 0-2).
__device__ __forceinline__ int site_of(const Geo& g, const uint8_t* __restrict__ cls, int x, int y,
                                       long long& off)
{
    if (x < 0 || x >= g.nx) {
        const int e = g.edge[x < 0 ? 0 : 1];
        if (e != EDGE_PERIODIC) return e == EDGE_WETTING ? ST_WET : ST_NEUTRAL;
        x = x < 0 ? x + g.nx : x - g.nx;
    }
    if (y < 0 || y >= g.ny) {
        const int e = g.edge[y < 0 ? 2 : 3];
        if (e == EDGE_LID) return ST_VOID;
        if (e != EDGE_PERIODIC) return e == EDGE_WETTING ? ST_WET : ST_NEUTRAL;
        y = y < 0 ? y + g.ny : y - g.ny;
    }
    off = (long long)y * g.pitch + x;
    return cls[off] & CLS_KIND_MASK;
}

__device__ __forceinline__ bool fluidlike(int s) { return s == ST_FLUID || s == ST_LID; }

// ---- stencils (Eqs. 20a, 20b): v[k] = chi(x + e_k) -----------------------
template <typename R>
__device__ __forceinline__ void grad9(const R v[9], R& gx, R& gy)
{
    // w_k e_k / cs^2: 1/3 on axis links, 1/12 on diagonals
    gx = R(1.0 / 3.0) * (v[1] - v[3]) + R(1.0 / 12.0) * ((v[5] - v[7]) + (v[8] - v[6]));
    gy = R(1.0 / 3.0) * (v[2] - v[4]) + R(1.0 / 12.0) * ((v[5] - v[7]) + (v[6] - v[8]));
}

template <typename R>
__device__ __forceinline__ R lap9(const R v[9])
{
    // 2 w_k / cs^2: 2/3 on axis links, 1/6 on diagonals; centre weight -10/3
    return R(2.0 / 3.0) * ((v[1] + v[3]) + (v[2] + v[4])) +
           R(1.0 / 6.0) * ((v[5] + v[7]) + (v[6] + v[8])) - R(10.0 / 3.0) * v[0];
}

// ---- Eq. 8 for i = 1, 2 ---------------------------------------------------
template <typename R>
__device__ __forceinline__ void chem_pot(const Prm<R>& P, R c1, R c2, R lap1, R lap2, R& mu1, R& mu2)
{
    const R c3 = R(1) - c1 - c2;
    const R t = R(2) * P.lamT * (c1 * c2 * c3);
    const R b1 = P.lam[0] * (c1 * (R(1) - c1) * (R(1) - R(2) * c1)) - t;
    const R b2 = P.lam[1] * (c2 * (R(1) - c2) * (R(1) - R(2) * c2)) - t;
    mu1 = P.k12D * b1 - P.k34D * P.lam[0] * lap1;
    mu2 = P.k12D * b2 - P.k34D * P.lam[1] * lap2;
}

// ---- Eq. 42: c_ghost - c_f on a link into a wetting solid ----------------
template <typename R>
__device__ __forceinline__ void wet_offset(const Prm<R>& P, R c1, R c2, R& o1, R& o2)
{
    const R c3 = R(1) - c1 - c2;
    o1 = P.k4D * (P.cos13 * c1 * c3 + P.cos12 * c1 * c2);
    o2 = P.k4D * (-P.cos12 * c1 * c2 + P.cos23 * c2 * c3);
}

// Macroscopic state of one node, everything the collision needs.
template <typename R>
struct Macro {
    R c1, c2, mu1, mu2, rho;
    R g1x, g1y, g2x, g2y;   // grad c1, grad c2 (Eq. 20a)
    R lm1, lm2;             // lap mu1, lap mu2 (Eq. 20b)
};

// Velocity and pressure (Eqs. 13b, 13c) plus the forces of Eq. 12, given the
// node's g and macros.  Also returns the tau_g-dependent constants.
template <typename R>
struct Hydro {
    R ux, uy, p, usq;
    R Ftx, Fty;      // F_s + G
    R Fax, Fay;      // F_a
    R grx, gry;      // grad rho
    R inv_taug;
};

template <typename R>
__device__ __forceinline__ void surface_force(const Prm<R>& P, const Macro<R>& m, R& Fsx, R& Fsy)
{
    const R mu3 = -(P.l3_l1 * m.mu1 + P.l3_l2 * m.mu2);
    Fsx = (m.mu1 - mu3) * m.g1x + (m.mu2 - mu3) * m.g2x;
    Fsy = (m.mu1 - mu3) * m.g1y + (m.mu2 - mu3) * m.g2y;
}

template <typename R>
__device__ __forceinline__ void hydro_from_g(const Prm<R>& P, const Macro<R>& m, const R g[9], Hydro<R>& h)
{
    R Fsx, Fsy;
    surface_force(P, m, Fsx, Fsy);
    const R Gx = m.rho * P.gx, Gy = m.rho * P.gy;
    h.Ftx = Fsx + Gx;
    h.Fty = Fsy + Gy;
    h.grx = (P.rho[0] - P.rho[2]) * m.g1x + (P.rho[1] - P.rho[2]) * m.g2x;
    h.gry = (P.rho[0] - P.rho[2]) * m.g1y + (P.rho[1] - P.rho[2]) * m.g2y;
    const R mx = (g[1] - g[3]) + (g[5] - g[7]) + (g[8] - g[6]);
    const R my = (g[2] - g[4]) + (g[5] - g[7]) + (g[6] - g[8]);
    const R inv_rho = R(1) / m.rho;
    h.ux = (mx + R(0.5) * h.Ftx) * inv_rho;
    h.uy = (my + R(0.5) * h.Fty) * inv_rho;
    h.usq = h.ux * h.ux + h.uy * h.uy;
    const R sumg = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
    // p = cs^2/(1 - w0) [sum_{k!=0} g_k + u.grad rho / 2 + rho s_0(u)], s_0 = -w0 u.u / (2 cs^2)
    h.p = R(0.6) * (sumg + R(0.5) * (h.ux * h.grx + h.uy * h.gry) - R(2.0 / 3.0) * m.rho * h.usq);
    const R a = P.aM[0] * m.lm1 + P.aM[1] * m.lm2;
    h.Fax = h.ux * a;
    h.Fay = h.uy * a;
    const R c3 = R(1) - m.c1 - m.c2;
    const R nu = m.c1 * P.nu[0] + m.c2 * P.nu[1] + c3 * P.nu[2];
    h.inv_taug = R(1) / (R(3) * nu + R(0.5));
}

// Post-collision populations of direction k (Eqs. 1a, 1b, 2a, 2b, 4, 11a,
// 11b, 45) from the pre-collision values f1k, f2k, gk.
template <int K, typename R>
__device__ __forceinline__ void collide_k(const Prm<R>& P, const Macro<R>& m, const Hydro<R>& h,
                                          R d1x, R d1y, R d2x, R d2y, R f1k, R f2k, R gk,
                                          R& o1, R& o2, R& og)
{
    constexpr R w = R(wk(K));
    constexpr R exk = R(ex(K)), eyk = R(ey(K));
    const R eu = exk * h.ux + eyk * h.uy;
    const R sk = w * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * h.usq);
    R f1eq, f2eq, geq;
    if (K == 0) {
        f1eq = m.c1 + (w - R(1)) * P.eta[0] * m.mu1;
        f2eq = m.c2 + (w - R(1)) * P.eta[1] * m.mu2;
        geq = R(3) * h.p * (w - R(1)) + m.rho * sk;
    } else {
        f1eq = w * (P.eta[0] * m.mu1 + R(3) * m.c1 * eu);
        f2eq = w * (P.eta[1] * m.mu2 + R(3) * m.c2 * eu);
        geq = R(3) * h.p * w + m.rho * sk;
    }
    const R F1 = P.src_f[0] * w * (exk * d1x + eyk * d1y);
    const R F2 = P.src_f[1] * w * (exk * d2x + eyk * d2y);
    const R bx = sk * h.grx + R(3) * (sk + w) * h.Ftx;
    const R by = sk * h.gry + R(3) * (sk + w) * h.Fty;
    const R Gk = (R(1) - R(0.5) * h.inv_taug) * ((exk - h.ux) * bx + (eyk - h.uy) * by) +
                 R(3) * w * (exk * h.Fax + eyk * h.Fay);
    o1 = f1k - (f1k - f1eq) * P.inv_tau[0] + F1;
    o2 = f2k - (f2k - f2eq) * P.inv_tau[1] + F2;
    og = gk - (gk - geq) * h.inv_taug + Gk;
}

// Equilibria alone (Eqs. 2a, 2b), used by the lid (Eq. 51) and set-up.
template <typename R>
__device__ __forceinline__ void equilibria(int k, const Prm<R>& P, R c1, R c2, R mu1, R mu2, R rho, R p,
                                           R ux, R uy, R& f1eq, R& f2eq, R& geq)
{
    const R w = R(wk(k));
    const R eu = R(ex(k)) * ux + R(ey(k)) * uy;
    const R usq = ux * ux + uy * uy;
    const R sk = w * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * usq);
    if (k == 0) {
        f1eq = c1 + (w - R(1)) * P.eta[0] * mu1;
        f2eq = c2 + (w - R(1)) * P.eta[1] * mu2;
        geq = R(3) * p * (w - R(1)) + rho * sk;
    } else {
        f1eq = w * (P.eta[0] * mu1 + R(3) * c1 * eu);
        f2eq = w * (P.eta[1] * mu2 + R(3) * c2 * eu);
        geq = R(3) * p * w + rho * sk;
    }
}

template <typename S>
__device__ __forceinline__ S ldg(const S* p) { return __ldg(p); }

}  // namespace tlb

// Device-side building blocks of the ternary phase-field lattice Boltzmann
// update (Liang et al., arXiv:1710.09534, Sec. II): D2Q9 constants, node
// classification, the isotropic stencils of Eqs. 20a/20b, the chemical
// potential of Eq. 8, the wetting ghost offset of Eq. 42, the moments of
// Eqs. 13b/13c with the forces of Eq. 12, and the BGK collision of Eqs. 1a,
// 1b, 2a, 2b, 4, 11a, 11b rearranged for few FP64 instructions.
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
// Direction k as sign * (one of +x, +y, (1,1), (1,-1)): component index 0..3
__host__ __device__ constexpr int comp(int k) { return (k == 1 || k == 3) ? 0 : ((k == 2 || k == 4) ? 1 : ((k == 5 || k == 7) ? 2 : 3)); }
__host__ __device__ constexpr int sgn(int k) { return (k == 1 || k == 2 || k == 5 || k == 8) ? 1 : -1; }
__host__ __device__ constexpr int wclass(int k) { return k <= 4 ? 0 : 1; }  // 0 axis, 1 diagonal

// FP16 storage holds 2^kF16ScaleExp times each 16-bit population.
constexpr int kF16ScaleExp = 12;

// Site kinds (same semantics as the FP64 oracle's classification).
enum : int { ST_FLUID = 0, ST_LID = 1, ST_WET = 2, ST_NEUTRAL = 3, ST_VOID = 4 };
enum : int { EDGE_PERIODIC = 0, EDGE_WETTING = 1, EDGE_NEUTRAL = 2, EDGE_LID = 3 };
enum : uint8_t { CLS_KIND_MASK = 7, CLS_INTERIOR = 8 };

struct Geo {
    int nx, ny, pitch;
    int edge[4];  // left, right, bottom, top
    long long plane;  // elements per plane = ny * pitch
};

// Derived constants, computed on the host from tlb_params (index i: fluid
// 1, 2; index c: direction class 0 = axis (w = 1/9), 1 = diagonal (w = 1/36)).
template <typename R>
struct Prm {
    R lam[3], lamT;
    R two_lamT;       // 2 lambda_T
    R k12D;           // 12 / D
    R k34D;           // 3/4 D
    R k34Dlam[2];     // 3/4 D lambda_i
    R k4D;            // 4 / D (Eq. 42 with dx = 1)
    R eta[2];         // eta_i = M_i / (cs^2 (tau_i - 1/2))
    R inv_tau[2];     // 1 / tau_i
    R omt[2];         // 1 - 1 / tau_i
    R src_f[2];       // (1 - 1/(2 tau_i)) * 3 (Eq. 11a with 1/cs^2)
    R e0[2];          // (w_0 - 1) eta_i / tau_i  (k = 0 equilibrium, relaxed)
    R aw[2][2];       // eta_i w_c / tau_i
    R bw[2][2];       // 3 w_c / tau_i
    R sw[2][2];       // src_f_i w_c
    R rho[3], nu[3];
    R drho[2], dnu[2];  // rho_i - rho_3, nu_i - nu_3
    R aM[2];          // (rho_i - rho_3) M_i (Eq. 12)
    R l3_l1, l3_l2;   // lambda_3 / lambda_i (mu_3 from sum mu_i / lambda_i = 0)
    R cos12, cos13, cos23;
    R gx, gy;
    R lid_u;
    R mrt;            // 1: MRT collision (moment basis below), 0: BGK
    R mrt_s_f;        // MRT rate of the non-flux moments of f^i
    R mrt_s_g;        // MRT rate of the energy moments of g
    // equal densities and equal viscosities (rho_i = rho_3, nu_i = nu_3): the
    // constants the uniform-property update uses instead of per-node values
    R uni;            // 1 when both hold
    R inv_rho3, inv_taug3, omtg3, kG3;  // 1/rho, 1/tau_g, 1 - 1/tau_g, 1 - 1/(2 tau_g)
    R Rw3[2], Kw3[2];                   // rho w / tau_g, w (1 - 1/(2 tau_g)) per class
    R p3tg3;                            // 3 / tau_g
    R rg3x, rg3y;                       // rho g (the body force G of a uniform density)
    // constants of the scaled stencils (grad9s = 12 grad, lap9s = 6 lap)
    R Kl[2];          // 12 lambda_i / D
    R Kt;             // 12 / D * 2 lambda_T
    R K34l6[2];       // 3/4 D lambda_i / 6
    R qa[2][2];       // F_s weights: (mu_i - mu_3) / 12 = qa[i][0] mu_1 + qa[i][1] mu_2
    R drho12[2];      // (rho_i - rho_3) / 12
    R aM6[2];         // (rho_i - rho_3) M_i / 6
    R k3tau[2];       // 3 / tau_i
    R kq[2], ks[2];   // 3 w36 / tau_i, w36 src_f_i (the order-parameter sources per w36)
    R K3w3[2];        // 3 Kw3 (uniform properties: K_w T = K3w3 (F_s + G))
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

// ---- reciprocal -------------------------------------------------------------
// FP64: single-precision seed refined by two Newton-Raphson steps
// r <- r + r (1 - a r), each doubling the correct bits (24 -> 48 -> 96), i.e.
// within one ulp of 1/a for the positive, normal a used here (rho, tau_g).
__device__ __forceinline__ double rcp(double a)
{
    double r = (double)(1.0f / (float)a);
    double e = fma(-a, r, 1.0);
    r = fma(r, e, r);
    e = fma(-a, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ float rcp(float a) { return 1.0f / a; }

// ---- stencils (Eqs. 20a, 20b): v[k] = chi(x + e_k) -----------------------
// Both are returned scaled so that their weights are small integers (the
// constant factor is folded into the constants that multiply them):
// grad9s = 12 grad (w_k e_k / cs^2 is 1/3 on axis links, 1/12 on diagonals),
// lap9s = 6 lap (2 w_k / cs^2 is 2/3 on axis links, 1/6 on diagonals, the
// centre weight -10/3).
template <typename R>
__device__ __forceinline__ void grad9s(const R v[9], R& gx12, R& gy12)
{
    const R d57 = v[5] - v[7], d86 = v[8] - v[6];
    gx12 = fma(R(4), v[1] - v[3], d57 + d86);
    gy12 = fma(R(4), v[2] - v[4], d57 - d86);
}

template <typename R>
__device__ __forceinline__ R lap9s(const R v[9])
{
    const R ax = (v[1] + v[3]) + (v[2] + v[4]);
    const R dg = (v[5] + v[7]) + (v[6] + v[8]);
    return fma(R(4), ax, fma(R(-20), v[0], dg));
}

// ---- Eq. 8 for i = 1, 2, from the scaled Laplacians lap6_i = 6 lap c_i -------
//   mu_i = 12/D [lambda_i c_i (1 - c_i)(1 - 2 c_i) - 2 lambda_T c1 c2 c3] - 3/4 D lambda_i lap c_i
template <typename R>
__device__ __forceinline__ void chem_pot(const Prm<R>& P, R c1, R c2, R lap6_1, R lap6_2, R& mu1, R& mu2)
{
    const R c3 = R(1) - c1 - c2;
    const R tt = P.Kt * (c1 * c2) * c3;
    // c (1 - c)(1 - 2c) = c (1 + c (2c - 3))
    const R p1 = c1 * fma(c1, fma(R(2), c1, R(-3)), R(1));
    const R p2 = c2 * fma(c2, fma(R(2), c2, R(-3)), R(1));
    mu1 = fma(P.Kl[0], p1, -fma(P.K34l6[0], lap6_1, tt));
    mu2 = fma(P.Kl[1], p2, -fma(P.K34l6[1], lap6_2, tt));
}

// ---- Eq. 42: c_ghost - c_f on a link into a wetting solid ----------------
template <typename R>
__device__ __forceinline__ void wet_offset(const Prm<R>& P, R c1, R c2, R& o1, R& o2)
{
    const R c3 = R(1) - c1 - c2;
    o1 = P.k4D * (P.cos13 * c1 * c3 + P.cos12 * c1 * c2);
    o2 = P.k4D * (-P.cos12 * c1 * c2 + P.cos23 * c2 * c3);
}

// Macroscopic state of one node from the stencil phase.
template <typename R>
struct Macro {
    R c1, c2, mu1, mu2, rho;
    R g1x, g1y, g2x, g2y;   // 12 grad c1, 12 grad c2 (Eq. 20a, grad9s)
    R lm1, lm2;             // 6 lap mu1, 6 lap mu2 (Eq. 20b, lap9s)
};

// Velocity, pressure and forces (Eqs. 12, 13b, 13c).
template <typename R>
struct Hydro {
    R ux, uy, p, usq;
    R Ftx, Fty;      // F_s + G
    R a;             // sum_i (rho_i - rho_3) M_i lap mu_i, so that F_a = u a
    R grx, gry;      // grad rho
    R inv_taug;
};

template <typename R>
__device__ __forceinline__ R density(const Prm<R>& P, R c1, R c2)
{
    return fma(c2, P.drho[1], fma(c1, P.drho[0], P.rho[2]));
}

// UNI (equal densities and viscosities): grad rho, u.grad rho and F_a vanish
// identically and rho, tau_g are constants, so those terms are skipped (the
// general form would add exact zeros).
// SE: the g populations are given in units of 2^SE (see collide_all).
template <bool UNI = false, int SE = 0, typename R>
__device__ __forceinline__ void hydro_from_g(const Prm<R>& P, const Macro<R>& m, const R g[9], Hydro<R>& h)
{
    // F_s = sum_i mu_i grad c_i with grad c3 = -grad c1 - grad c2, i.e.
    // sum_{i=1,2} (mu_i - mu_3) grad c_i, mu_3 from sum_i mu_i / lambda_i = 0;
    // q_i = (mu_i - mu_3) / 12 against the scaled gradients; G = rho g
    const R q1 = fma(P.qa[0][0], m.mu1, P.qa[0][1] * m.mu2);
    const R q2 = fma(P.qa[1][0], m.mu1, P.qa[1][1] * m.mu2);
    const R Gx = UNI ? P.rg3x : m.rho * P.gx, Gy = UNI ? P.rg3y : m.rho * P.gy;
    h.Ftx = fma(q1, m.g1x, fma(q2, m.g2x, Gx));
    h.Fty = fma(q1, m.g1y, fma(q2, m.g2y, Gy));
    const R g57 = g[5] - g[7], g86 = g[8] - g[6];
    R mx = (g[1] - g[3]) + (g57 + g86);
    R my = (g[2] - g[4]) + (g57 - g86);
    R sumg = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
    if constexpr (SE != 0) {
        constexpr R inv = R(1.0 / double(1 << SE));
        mx *= inv;
        my *= inv;
        sumg *= inv;
    }
    if constexpr (UNI) {
        h.grx = h.gry = R(0);
        h.ux = fma(R(0.5), h.Ftx, mx) * P.inv_rho3;
        h.uy = fma(R(0.5), h.Fty, my) * P.inv_rho3;
        h.usq = fma(h.ux, h.ux, h.uy * h.uy);
        h.p = R(0.6) * fma(R(-2.0 / 3.0) * m.rho, h.usq, sumg);
        h.a = R(0);
        h.inv_taug = P.inv_taug3;
    } else {
        h.grx = fma(P.drho12[0], m.g1x, P.drho12[1] * m.g2x);
        h.gry = fma(P.drho12[0], m.g1y, P.drho12[1] * m.g2y);
        const R inv_rho = rcp(m.rho);
        h.ux = fma(R(0.5), h.Ftx, mx) * inv_rho;
        h.uy = fma(R(0.5), h.Fty, my) * inv_rho;
        h.usq = fma(h.ux, h.ux, h.uy * h.uy);
        // p = cs^2/(1 - w0) [sum_{k!=0} g_k + u.grad rho / 2 + rho s_0(u)], s_0 = -w0 u.u / (2 cs^2)
        const R ug = fma(h.ux, h.grx, h.uy * h.gry);
        h.p = R(0.6) * fma(R(-2.0 / 3.0) * m.rho, h.usq, fma(R(0.5), ug, sumg));
        h.a = fma(P.aM6[0], m.lm1, P.aM6[1] * m.lm2);
        const R nu = fma(m.c2, P.dnu[1], fma(m.c1, P.dnu[0], P.nu[2]));
        h.inv_taug = rcp(fma(R(3), nu, R(0.5)));
    }
}

// Per-node precomputation of the BGK update (Eqs. 1a, 1b, 2a, 2b, 4, 11a,
// 11b, 45), arranged so that a direction k and its opposite k-bar share most
// of their arithmetic.  With s = +1 for k and -1 for k-bar, E = e_k . u and
// beta = 3E:
//   f'^i = (1 - 1/tau_i) f^i + A_i + s V_i,
//     A_i = eta_i w mu_i / tau_i,  V_i = w e_k . Q_i,
//     Q_i = (3 c_i / tau_i) u + 3 (1 - 1/(2 tau_i)) d/dt(c_i u)   (Eqs. 2a, 11a, 19)
//   g'   = (1 - 1/tau_g) g + Sym + s Anti,
// where, with q = 3 e.u + 4.5 (e.u)^2 - 1.5 u.u = a + s beta
// (a = 4.5 E^2 - 1.5 u.u), the equilibrium and source of g (Eqs. 2b, 4, 11b),
//   g^eq / tau_g + G_k = Rw q + Pw + Kw [q (e - u).H + (e - u).T] + 3 w e.F_a,
//   Rw = w rho / tau_g, Pw = 3 w p / tau_g, Kw = w (1 - 1/(2 tau_g)),
//   H = grad rho + 3 (F_s + G), T = 3 (F_s + G), F_a = a_F u,
// expand to
//   Sym  = beta KX + a RX + PX,   Anti = a KX + beta RX + AX,
//   KX = Kw e.H, RX = Rw - Kw u.H, PX = Pw - Kw u.T,
//   AX = Kw e.T + 3 w a_F e.u   (= KX with equal densities, where H = T).
// Every term is small (of the size of the populations themselves): the O(1)
// parts of Rw and of (q + 1) never meet in a difference.
// V_i is formed per pair from Q'_i = w36 Q_i: 4 Q'_x or 4 Q'_y on the axis
// links (w_axis = 4 w36, folded into one fma with A_i), Q'_x +- Q'_y on the
// diagonal ones.
template <typename R, bool UNI = false>
struct Collider {
    R A1[2], A2[2];     // per class (0 axis, 1 diagonal)
    R Q1[2], Q2[2];     // w36 Q_i (x, y)
    R E1, E2;           // f^{i,eq}_0 / tau_i
    R b[4];             // beta = 3 e.u per component
    R t0;               // -1.5 u.u
    R KX[4], RX[2], PX[2], AX[4];
    R omt1, omt2, omtg;
    R P0;               // g^eq_0 / tau_g + G_0

    // SE: the moving populations and g_0 are handled in units of 2^SE (see
    // collide_all); the constants that add to them are scaled to match.
    template <int SE = 0>
    __device__ __forceinline__ void build(const Prm<R>& P, const Macro<R>& m, const Hydro<R>& h,
                                          R d1x, R d1y, R d2x, R d2y)
    {
        constexpr R w9 = R(1.0 / 9.0), w36 = R(1.0 / 36.0), w0 = R(4.0 / 9.0);
        // order parameters
        omt1 = P.omt[0];
        omt2 = P.omt[1];
        E1 = fma(P.e0[0], m.mu1, P.inv_tau[0] * m.c1);
        E2 = fma(P.e0[1], m.mu2, P.inv_tau[1] * m.c2);
#pragma unroll
        for (int c = 0; c < 2; c++) {
            A1[c] = P.aw[0][c] * m.mu1;
            A2[c] = P.aw[1][c] * m.mu2;
        }
        // w36 Q_i = (3 w36 / tau_i) c_i u + w36 src_f_i d(c_i u); the products
        // c_i u are the ones the caller stores for Eq. 19
        Q1[0] = fma(P.kq[0], m.c1 * h.ux, P.ks[0] * d1x);
        Q1[1] = fma(P.kq[0], m.c1 * h.uy, P.ks[0] * d1y);
        Q2[0] = fma(P.kq[1], m.c2 * h.ux, P.ks[1] * d2x);
        Q2[1] = fma(P.kq[1], m.c2 * h.uy, P.ks[1] * d2y);
        // hydrodynamics
        b[0] = R(3) * h.ux;
        b[1] = R(3) * h.uy;
        b[2] = b[0] + b[1];
        b[3] = b[0] - b[1];
        t0 = R(-1.5) * h.usq;
        const R itg = h.inv_taug;
        R uT, uH, kG, Kw[2];
        if constexpr (UNI) {
            // H = T = 3 (F_s + G) (grad rho = 0), F_a = 0; tau_g and rho are
            // constants; the factor 3 of T sits in the constants K3w
            omtg = P.omtg3;
            kG = P.kG3;
            const R uF = fma(h.ux, h.Ftx, h.uy * h.Fty);
            // K_w e.T: products of sums only, so that no instantiation of the
            // kernels can contract a product into an add differently
            KX[0] = P.K3w3[0] * h.Ftx;
            KX[1] = P.K3w3[0] * h.Fty;
            KX[2] = P.K3w3[1] * (h.Ftx + h.Fty);
            KX[3] = P.K3w3[1] * (h.Ftx - h.Fty);
            const R p3 = h.p * P.p3tg3;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                RX[c] = fma(-P.K3w3[c], uF, P.Rw3[c]);
                PX[c] = fma(-P.K3w3[c], uF, (c == 0 ? w9 : w36) * p3);
            }
#pragma unroll
            for (int c = 0; c < 4; c++) AX[c] = KX[c];
            uT = R(3) * uF;
            uH = uT;
        } else {
            const R Tx = R(3) * h.Ftx, Ty = R(3) * h.Fty;
            uT = fma(h.ux, Tx, h.uy * Ty);
            omtg = R(1) - itg;
            kG = fma(R(-0.5), itg, R(1));
            Kw[0] = w9 * kG;
            Kw[1] = w36 * kG;
            const R ri = m.rho * itg;
            const R Hx = h.grx + Tx, Hy = h.gry + Ty;
            uH = fma(h.ux, Hx, h.uy * Hy);
            KX[0] = Kw[0] * Hx;
            KX[1] = Kw[0] * Hy;
            KX[2] = Kw[1] * (Hx + Hy);
            KX[3] = Kw[1] * (Hx - Hy);
            const R p3 = R(3) * h.p * itg;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const R wc = c == 0 ? w9 : w36;
                RX[c] = fma(-Kw[c], uH, wc * ri);
                PX[c] = fma(-Kw[c], uT, wc * p3);
            }
            // AX = Kw e.T + 3 w a_F e.u = Kw e.T + (w a_F) beta
            const R wa0 = w9 * h.a, wa1 = w36 * h.a;
            AX[0] = fma(wa0, b[0], Kw[0] * Tx);
            AX[1] = fma(wa0, b[1], Kw[0] * Ty);
            AX[2] = fma(wa1, b[2], Kw[1] * (Tx + Ty));
            AX[3] = fma(wa1, b[3], Kw[1] * (Tx - Ty));
        }
        // k = 0: g^eq_0 = 3p (w0 - 1) + rho w0 t0; G_0 = -w0 kG (t0 u.H + u.T)
        const R geq0 = fma(m.rho * w0, t0, R(3) * (w0 - R(1)) * h.p);
        P0 = fma(geq0, itg, -(w0 * kG) * fma(t0, uH, uT));
        if constexpr (SE != 0) {
            constexpr R sc = R(1 << SE);
#pragma unroll
            for (int c = 0; c < 2; c++) {
                A1[c] *= sc;
                A2[c] *= sc;
                RX[c] *= sc;
                PX[c] *= sc;
                Q1[c] *= sc;
                Q2[c] *= sc;
            }
#pragma unroll
            for (int c = 0; c < 4; c++) {
                KX[c] *= sc;
                AX[c] *= sc;
            }
            P0 *= sc;
        }
    }

    // rest direction
    __device__ __forceinline__ void post0(R f10, R f20, R g0, R& o1, R& o2, R& og) const
    {
        o1 = fma(omt1, f10, E1);
        o2 = fma(omt2, f20, E2);
        og = fma(omtg, g0, P0);
    }

    // direction K (one of 1, 2, 5, 8: s = +1) and its opposite opp(K)
    template <int K>
    __device__ __forceinline__ void pair(R f1p, R f2p, R gp, R f1m, R f2m, R gm, R& o1p, R& o2p, R& ogp, R& o1m,
                                         R& o2m, R& ogm) const
    {
        static_assert(K == 1 || K == 2 || K == 5 || K == 8, "pair<K> takes the direction with s = +1");
        constexpr int C = comp(K), W = wclass(K);
        R s1p, s1m, s2p, s2m;  // A_i +- V_i
        if constexpr (C < 2) {
            s1p = fma(R(4), Q1[C], A1[W]);
            s1m = fma(R(-4), Q1[C], A1[W]);
            s2p = fma(R(4), Q2[C], A2[W]);
            s2m = fma(R(-4), Q2[C], A2[W]);
        } else {
            const R V1 = C == 2 ? Q1[0] + Q1[1] : Q1[0] - Q1[1];
            const R V2 = C == 2 ? Q2[0] + Q2[1] : Q2[0] - Q2[1];
            s1p = A1[W] + V1;
            s1m = A1[W] - V1;
            s2p = A2[W] + V2;
            s2m = A2[W] - V2;
        }
        o1p = fma(omt1, f1p, s1p);
        o1m = fma(omt1, f1m, s1m);
        o2p = fma(omt2, f2p, s2p);
        o2m = fma(omt2, f2m, s2m);
        const R beta = b[C];
        const R a = fma(beta, R(0.5) * beta, t0);
        const R sym = fma(beta, KX[C], fma(a, RX[W], PX[W]));
        const R anti = fma(a, KX[C], fma(beta, RX[W], AX[C]));
        ogp = fma(omtg, gp, sym + anti);
        ogm = fma(omtg, gm, sym - anti);
    }
};

// The four directions with s = +1 of the opposite pairs (k, opp(k)).
__host__ __device__ constexpr int pair_dir(int p) { return p == 0 ? 1 : (p == 1 ? 2 : (p == 2 ? 5 : 8)); }

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

// ---- MRT option: orthogonal D2Q9 moment basis (Lallemand and Luo) --------
// rows: 1, -4 + 3|e|^2, 4 - 21/2 |e|^2 + 9/2 |e|^4, e_x, (-5 + 3|e|^2) e_x, e_y,
// (-5 + 3|e|^2) e_y, e_x^2 - e_y^2, e_x e_y; squared norms 9 36 36 6 12 6 12 4 4.
__host__ __device__ constexpr int mrt_m(int r, int k)
{
    return r == 0 ? 1
         : r == 1 ? -4 + 3 * (ex(k) * ex(k) + ey(k) * ey(k))
         : r == 2 ? (8 - 21 * (ex(k) * ex(k) + ey(k) * ey(k)) + 9 * (ex(k) * ex(k) + ey(k) * ey(k)) * (ex(k) * ex(k) + ey(k) * ey(k))) / 2
         : r == 3 ? ex(k)
         : r == 4 ? (-5 + 3 * (ex(k) * ex(k) + ey(k) * ey(k))) * ex(k)
         : r == 5 ? ey(k)
         : r == 6 ? (-5 + 3 * (ex(k) * ex(k) + ey(k) * ey(k))) * ey(k)
         : r == 7 ? ex(k) * ex(k) - ey(k) * ey(k)
                  : ex(k) * ey(k);
}
__host__ __device__ constexpr double mrt_inv_norm(int r)
{
    return r == 0 ? 1.0 / 9 : (r == 1 || r == 2) ? 1.0 / 36 : (r == 3 || r == 5) ? 1.0 / 6 : (r == 4 || r == 6) ? 1.0 / 12 : 1.0 / 4;
}

// v' = v + M^-1 [ -S M (v - veq) + (I - S/2) M src ]  (equal rates: the BGK update)
template <typename R>
__device__ __forceinline__ void mrt_relax(const R v[9], const R veq[9], const R src[9], const R s[9], R out[9])
{
    R mp[9];
#pragma unroll
    for (int r = 0; r < 9; r++) {
        R mn = R(0), ms = R(0);
#pragma unroll
        for (int k = 0; k < 9; k++) {
            if (mrt_m(r, k) != 0) {
                mn = fma(R(mrt_m(r, k)), v[k] - veq[k], mn);
                ms = fma(R(mrt_m(r, k)), src[k], ms);
            }
        }
        mp[r] = fma(fma(R(-0.5), s[r], R(1)), ms, -s[r] * mn) * R(mrt_inv_norm(r));
    }
#pragma unroll
    for (int k = 0; k < 9; k++) {
        R acc = v[k];
#pragma unroll
        for (int r = 0; r < 9; r++)
            if (mrt_m(r, k) != 0) acc = fma(R(mrt_m(r, k)), mp[r], acc);
        out[k] = acc;
    }
}

// Per-node inputs of the MRT update: equilibria (Eqs. 2a, 2b) and the source
// terms of Eqs. 11a, 11b without their (1 - 1/(2 tau)) factors; the F_a part of
// Eq. 11b is added after the relaxation.
template <typename R>
struct MrtNode {
    R c[2], emu[2], d[2][2];  // c_i, eta_i mu_i, d/dt (c_i u)
    R ux, uy, t0, p, rho;
    R H[4], T[4], uH, uT, Z[4];
    R s_f[2][9], s_g[9];

    template <int SE = 0>
    __device__ __forceinline__ void build(const Prm<R>& P, const Macro<R>& m, const Hydro<R>& h,
                                          R d1x, R d1y, R d2x, R d2y)
    {
        static_assert(SE == 0, "the MRT update works in plain units");
        c[0] = m.c1;
        c[1] = m.c2;
        emu[0] = P.eta[0] * m.mu1;
        emu[1] = P.eta[1] * m.mu2;
        d[0][0] = d1x;
        d[0][1] = d1y;
        d[1][0] = d2x;
        d[1][1] = d2y;
        ux = h.ux;
        uy = h.uy;
        t0 = R(-1.5) * h.usq;
        p = h.p;
        rho = m.rho;
        const R Tx = R(3) * h.Ftx, Ty = R(3) * h.Fty;
        const R Hx = h.grx + Tx, Hy = h.gry + Ty;
        H[0] = Hx;
        H[1] = Hy;
        H[2] = Hx + Hy;
        H[3] = Hx - Hy;
        T[0] = Tx;
        T[1] = Ty;
        T[2] = Tx + Ty;
        T[3] = Tx - Ty;
        uH = fma(ux, Hx, uy * Hy);
        uT = fma(ux, Tx, uy * Ty);
        const R za = R(3.0 / 9.0) * h.a, zd = R(3.0 / 36.0) * h.a;
        Z[0] = za * ux;
        Z[1] = za * uy;
        Z[2] = zd * (ux + uy);
        Z[3] = zd * (ux - uy);
#pragma unroll
        for (int r = 0; r < 9; r++) {
            const bool flux = r == 0 || r == 3 || r == 5;
            s_f[0][r] = flux ? P.inv_tau[0] : P.mrt_s_f;
            s_f[1][r] = flux ? P.inv_tau[1] : P.mrt_s_f;
            s_g[r] = (r == 1 || r == 2 || r == 4 || r == 6) ? P.mrt_s_g : h.inv_taug;
        }
    }

    // post-collision populations of f^1, f^2, g from the pre-collision ones
    __device__ __forceinline__ void apply(const R f1[9], const R f2[9], const R g[9], R o1[9], R o2[9], R og[9]) const
    {
        R eq[9], src[9];
#pragma unroll
        for (int i = 0; i < 2; i++) {
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const R w = R(wk(k));
                const R eu = R(ex(k)) * ux + R(ey(k)) * uy;
                eq[k] = k == 0 ? c[i] + (w - R(1)) * emu[i] : w * fma(R(3) * c[i], eu, emu[i]);
                src[k] = R(3) * w * (R(ex(k)) * d[i][0] + R(ey(k)) * d[i][1]);
            }
            mrt_relax(i == 0 ? f1 : f2, eq, src, s_f[i], i == 0 ? o1 : o2);
        }
        R fa[9];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const R w = R(wk(k));
            if (k == 0) {
                eq[0] = fma(rho * w, t0, R(3) * (w - R(1)) * p);
                src[0] = w * -fma(t0, uH, uT);
                fa[0] = R(0);
            } else {
                const R sg = R(sgn(k));
                const R e = sg * (comp(k) == 0 ? ux : comp(k) == 1 ? uy : comp(k) == 2 ? ux + uy : ux - uy);
                const R q = fma(e, fma(R(4.5), e, R(3)), t0);
                eq[k] = w * fma(rho, q, R(3) * p);
                src[k] = w * fma(q, fma(sg, H[comp(k)], -uH), fma(sg, T[comp(k)], -uT));
                fa[k] = sg * Z[comp(k)];
            }
        }
        mrt_relax(g, eq, src, s_g, og);
#pragma unroll
        for (int k = 0; k < 9; k++) og[k] += fa[k];
    }
};

template <typename S>
__device__ __forceinline__ S ldg(const S* p) { return __ldg(p); }

}  // namespace tlb

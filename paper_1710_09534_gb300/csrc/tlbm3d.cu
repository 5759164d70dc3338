// D3Q19 form of the lattice update (Sec. II.A of Liang et al.,
// arXiv:1710.09534, states the model for D dimensions): FP64 storage and
// arithmetic, BGK collision, push streaming with half-way bounce-back, the
// Eq. 42 wetting ghosts on every link into a solid.
//
// One time step is three launches over all nodes of the lattice:
//   k3_csum    c_1, c_2 of every node (Eq. 13a) into two planes
//   k3_mu      mu_1, mu_2 (Eq. 8 with the Eq. 20b Laplacian and the Eq. 42
//              ghosts) into two planes
//   k3_update  gradients (Eq. 20a/20b, Eq. 43 ghosts), u and p (Eqs. 13b,
//              13c), forces (Eq. 12), Eq. 19, the equilibria and sources of
//              Eqs. 2a, 2b, 4, 11a, 11b, BGK relaxation and the push to
//              x + e_k (Eq. 44 on links into solids)
// The radius-2 stencil of the update (c for mu, mu for lap mu) goes through
// the two pairs of planes, which stay in L2 for the lattices this path
// serves; the update itself is bound by the FP64 unit.
//
// Layout (x fastest, rows padded to a multiple of 32): dist[q][z][y][x] with
// q = 0..18 f^1_k, 19..37 f^2_k, 38..56 g_k (two buffers); cu[6]: c1 ux, c1 uy,
// c1 uz, c2 ux, c2 uy, c2 uz of the previous step; cpl[2], mpl[2]; node kinds.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "tlbm.h"
#include "tlbm_internal.h"
#include "tlbm_device.cuh"

namespace tlb3 {

// ---- D3Q19: e_0 = 0, e_1..6 axis (+x -x +y -y +z -z), e_7..18 face
// diagonals; opposite directions adjacent (odd k <-> k + 1)
__host__ __device__ constexpr int ex(int k)
{
    return (k == 1 || k == 7 || k == 9 || k == 11 || k == 13) ? 1 : ((k == 2 || k == 8 || k == 10 || k == 12 || k == 14) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int k)
{
    return (k == 3 || k == 7 || k == 10 || k == 15 || k == 17) ? 1 : ((k == 4 || k == 8 || k == 9 || k == 16 || k == 18) ? -1 : 0);
}
__host__ __device__ constexpr int ez(int k)
{
    return (k == 5 || k == 11 || k == 14 || k == 15 || k == 18) ? 1 : ((k == 6 || k == 12 || k == 13 || k == 16 || k == 17) ? -1 : 0);
}
__host__ __device__ constexpr double wk(int k) { return k == 0 ? 1.0 / 3.0 : (k <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : (k % 2 == 1 ? k + 1 : k - 1); }
constexpr int Q = 19;
constexpr int NPLANES = 57;

enum : int { EDGE_PERIODIC = 0, EDGE_WETTING = 1, EDGE_NEUTRAL = 2 };
enum : uint8_t { K_FLUID = 0, K_WET = 2, K_NEUTRAL = 3 };

struct Geo3 {
    int nx, ny, nz, pitch;
    int edge[6];      // x-, x+, y-, y+, z-, z+
    long long plane;  // elements per plane = nz * ny * pitch
};

// Derived constants (host-computed from tlb_params).  Stencils are formed
// scaled so that their weights are small integers: G = 12 grad (weights 2 on
// the axis links, 1 on the diagonal ones), L6 = 6 lap (the same weights, minus
// 24 times the centre); the factors 1/12 and 1/6 sit in these constants.
template <typename R>
struct Prm3 {
    R eta[2], rho[3], nu[3];
    R l3_l1, l3_l2;
    R k4D;                    // 4 / D (Eq. 42)
    R cos12, cos13, cos23;
    R kl[2], kT, kd6[2];      // Eq. 8: 12 lambda_i / D, 24 lambda_T / D, (3/4) D lambda_i / 6
    R qa[2][2];               // (mu_i - mu_3) / 12 = qa[i][0] mu_1 + qa[i][1] mu_2
    R drho12[2];              // (rho_i - rho_3) / 12
    R aM6[2];                 // (rho_i - rho_3) M_i / 6 (Eq. 12 from L6 mu_i)
    R nu3, dnu[2];            // nu_3, nu_i - nu_3 (Eq. 15)
    R gx, gy;                 // G = rho (gx, gy, 0)
    // order parameters (Eqs. 1a, 2a, 11a)
    R omt[2];                 // 1 - 1/tau_i
    R e0[2], itau[2];         // (w_0 - 1) eta_i / tau_i, 1 / tau_i
    R aw[2][2];               // w eta_i / tau_i (axis, diagonal)
    R kq[2], sq[2];           // 3 w36 / tau_i, 3 w36 (1 - 1/(2 tau_i))
    // uniform properties (rho, nu equal in the three fluids)
    R rho0, irho, hirho, prho;  // rho, 1/rho, 1/(2 rho), -rho/4
    R itg0, omtg0, kG0, Kw0[2], Rw0[2], p3tg0, Gc[2];
};

// Per-node link word: bit k-1 (k = 1..18) set when x + e_k is a fluid node
// (inside the lattice or across a periodic edge); bits 18..22 the wetting
// weight n_w = sum of 36 w_k over the links into wetting solids; bit 31 set
// on solid nodes.
constexpr uint32_t LNK_SOLID = 1u << 31;
constexpr int LNK_NW = 18;

// FP32 storage keeps the rest populations f^1_0, f^2_0 as float pairs hi + lo
// (the lo parts in planes 57, 58 of a distribution buffer) and sets them after
// the collision to the old pair plus sum_k (f_k - f'_k) over the moving
// directions, so that each component's mass changes only by the rounding of
// those small differences (Eq. 1a conserves c_i).
template <typename R>
constexpr bool kLo3 = std::is_same<R, float>::value;
template <typename R>
constexpr int kPlanes3 = kLo3<R> ? NPLANES + 2 : NPLANES;
constexpr int kLoPlane = NPLANES;  // f^1_0 lo; f^2_0 lo follows

// hi + lo plus a small increment d, renormalised (Knuth's TwoSum keeps the
// rounding of hi + d, which joins lo)
__device__ __forceinline__ void rest_add3(float hi, float lo, float d, float& nhi, float& nlo)
{
    const float s = hi + d;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (d - bb);
    const float t = e + lo;
    nhi = s + t;
    nlo = t - (nhi - s);
}

__device__ __forceinline__ long long node_off(const Geo3& g, int x, int y, int z)
{
    return ((long long)z * g.ny + y) * g.pitch + x;
}

// Kind of site (x, y, z), at most one step outside the lattice per axis; on
// an inside site *off is its wrapped element offset.  The first outside axis
// in x, y, z order whose edge is not periodic decides.
__device__ __forceinline__ int site(const Geo3& g, const uint8_t* __restrict__ kind, int x, int y, int z,
                                    long long& off)
{
    int c[3] = {x, y, z};
    const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (c[a] < 0 || c[a] >= n[a]) {
            const int e = g.edge[2 * a + (c[a] < 0 ? 0 : 1)];
            if (e != EDGE_PERIODIC) return e == EDGE_WETTING ? K_WET : K_NEUTRAL;
            c[a] = c[a] < 0 ? c[a] + n[a] : c[a] - n[a];
        }
    }
    off = node_off(g, c[0], c[1], c[2]);
    return kind[off];
}

// Eq. 8 for i = 1, 2 from c_1, c_2 and L6 = 6 lap c_i; c (1 - c)(1 - 2c) in
// Horner form c (1 + c (2c - 3)).
template <typename R>
__device__ __forceinline__ void chem_pot(const Prm3<R>& P, R c1, R c2, R l6c1, R l6c2, R& mu1,
                                         R& mu2)
{
    const R c3 = R(1.0) - c1 - c2;
    const R t = P.kT * (c1 * c2) * c3;
    const R h1 = c1 * fma(c1, fma(R(2.0), c1, -R(3.0)), R(1.0));
    const R h2 = c2 * fma(c2, fma(R(2.0), c2, -R(3.0)), R(1.0));
    mu1 = fma(-P.kd6[0], l6c1, fma(P.kl[0], h1, -t));
    mu2 = fma(-P.kd6[1], l6c2, fma(P.kl[1], h2, -t));
}

// Element offsets of the 18 neighbours of node (x, y, z), periodic wrap
// included (the wrapped offset is in range on every edge; a link into a
// solid or a wall is never followed).
struct Nb3 {
    long long dx[3], dy[3], dz[3];
    __device__ __forceinline__ Nb3(const Geo3& g, int x, int y, int z)
    {
        const long long P = g.pitch, RZ = (long long)g.ny * g.pitch;
        dx[0] = x == 0 ? g.nx - 1 : -1;
        dx[1] = 0;
        dx[2] = x == g.nx - 1 ? -(long long)(g.nx - 1) : 1;
        dy[0] = y == 0 ? (g.ny - 1) * P : -P;
        dy[1] = 0;
        dy[2] = y == g.ny - 1 ? -(g.ny - 1) * P : P;
        dz[0] = z == 0 ? (g.nz - 1) * RZ : -RZ;
        dz[1] = 0;
        dz[2] = z == g.nz - 1 ? -(g.nz - 1) * RZ : RZ;
    }
    __device__ __forceinline__ long long off(int k) const { return dx[ex(k) + 1] + dy[ey(k) + 1] + dz[ez(k) + 1]; }
    // the neighbour's element offset when link k is fluid, else the node's own
    // (Eq. 43: a solid neighbour takes the centre's value)
    __device__ __forceinline__ long long at(uint32_t L, long long o, int k) const
    {
        return (L >> (k - 1)) & 1u ? o + off(k) : o;
    }
};

// ---- kernels --------------------------------------------------------------

// Node (x, y, z) of a launch over the whole lattice, one thread per node in
// x-fastest order (no idle threads at the row ends): grid ceil(nodes / 128).
#define NODE_OF_THREAD                                                         \
    const unsigned i_ = blockIdx.x * blockDim.x + threadIdx.x;                 \
    if (i_ >= (unsigned)g.nx * (unsigned)g.ny * (unsigned)g.nz) return;        \
    const unsigned r_ = i_ / (unsigned)g.nx;                                   \
    const int x = (int)(i_ - r_ * (unsigned)g.nx);                             \
    const int y = (int)(r_ % (unsigned)g.ny), z = (int)(r_ / (unsigned)g.ny);  \
    const long long o = node_off(g, x, y, z);

// Link words of every node (from the node kinds and the edges).
__global__ void k3_links(const uint8_t* __restrict__ kind, uint32_t* __restrict__ lnk, Geo3 g)
{
    NODE_OF_THREAD
    uint32_t w = LNK_SOLID;
    if (kind[o] == K_FLUID) {
        w = 0;
        uint32_t nw = 0;
#pragma unroll
        for (int k = 1; k < Q; k++) {
            long long nb = 0;
            const int s = site(g, kind, x + ex(k), y + ey(k), z + ez(k), nb);
            if (s == K_FLUID) w |= 1u << (k - 1);
            else if (s == K_WET) nw += k <= 6 ? 2u : 1u;
        }
        w |= nw << LNK_NW;
    }
    lnk[o] = w;
}

// c_1, c_2 of every node (Eq. 13a); zero on solids.
template <typename R>
__global__ void k3_csum(const R* __restrict__ f, R* __restrict__ cpl, const uint8_t* __restrict__ kind,
                        Geo3 g)
{
    NODE_OF_THREAD
    const long long PL = g.plane;
    R a = R(0.0), b = R(0.0);
    if (kind[o] == K_FLUID) {
        if constexpr (kLo3<R>) {
            // the rest population as hi + lo
            a = f[kLoPlane * PL + o];
            b = f[(kLoPlane + 1) * PL + o];
        }
#pragma unroll
        for (int k = 0; k < Q; k++) {
            a += f[k * PL + o];
            b += f[(Q + k) * PL + o];
        }
    }
    cpl[o] = a;
    cpl[PL + o] = b;
}

// Sum over the 9 opposite pairs of a pair-wise quantity: axis pairs weighted
// 2, diagonal pairs 1 (the integer weights 36 w_k).
#define W36_SUM(S) fma(R(2.0), ((S)[0] + (S)[1]) + (S)[2], (((S)[3] + (S)[4]) + ((S)[5] + (S)[6])) + ((S)[7] + (S)[8]))

// mu_1, mu_2 of a fluid node from the pair sums s_p = c(x + e_k) + c(x - e_k)
// of its link-selected neighbours: Eq. 8 with the Eq. 20b Laplacian, whose
// links into wetting solids take the Eq. 42 ghost c + o_i (with the wall
// value of c taken as the node's own, dx = 1) and into neutral solids c.
template <typename R>
__device__ __forceinline__ void mu_from_sums(const Prm3<R>& P, uint32_t L, R c1, R c2, const R s1[9],
                                             const R s2[9], R& mu1, R& mu2)
{
    R l1 = fma(-R(24.0), c1, W36_SUM(s1));
    R l2 = fma(-R(24.0), c2, W36_SUM(s2));
    const unsigned nwi = (L >> LNK_NW) & 31u;
    if (nwi) {
        const R c3 = R(1.0) - c1 - c2, nw = (R)(int)nwi;
        const R o1 = P.k4D * fma(P.cos13, c1 * c3, P.cos12 * (c1 * c2));
        const R o2 = P.k4D * fma(-P.cos12, c1 * c2, P.cos23 * (c2 * c3));
        l1 = fma(nw, o1, l1);
        l2 = fma(nw, o2, l2);
    }
    chem_pot(P, c1, c2, l1, l2, mu1, mu2);
}

// mu_1, mu_2 of every fluid node (zero on solids).
template <typename R>
__global__ void k3_mu(const R* __restrict__ cpl, R* __restrict__ mpl, const uint32_t* __restrict__ lnk,
                      Geo3 g, Prm3<R> P)
{
    NODE_OF_THREAD
    const long long PL = g.plane;
    const uint32_t L = lnk[o];
    R mu1 = R(0.0), mu2 = R(0.0);
    if (!(L & LNK_SOLID)) {
        const Nb3 nb(g, x, y, z);
        const R c1 = cpl[o], c2 = cpl[PL + o];
        R s1[9], s2[9];
#pragma unroll
        for (int p = 0; p < 9; p++) {
            const long long ap = nb.at(L, o, 2 * p + 1), am = nb.at(L, o, 2 * p + 2);
            s1[p] = cpl[ap] + cpl[am];
            s2[p] = cpl[PL + ap] + cpl[PL + am];
        }
        mu_from_sums(P, L, c1, c2, s1, s2, mu1, mu2);
    }
    mpl[o] = mu1;
    mpl[PL + o] = mu2;
}

// X . e_k of the direction k = 2p + 1 of opposite pair p (the odd member),
// and the same weighted by 36 w_k (x 2 on the axis pairs).
template <int p, typename R>
__device__ __forceinline__ R edot(const R X[3])
{
    if constexpr (p < 3) return X[p];
    else if constexpr (p == 3) return X[0] + X[1];
    else if constexpr (p == 4) return X[0] - X[1];
    else if constexpr (p == 5) return X[0] + X[2];
    else if constexpr (p == 6) return X[0] - X[2];
    else if constexpr (p == 7) return X[1] + X[2];
    else return X[1] - X[2];
}
template <int p, typename R>
__device__ __forceinline__ R wdot(const R X[3])
{
    if constexpr (p < 3) return R(2.0) * X[p];
    else return edot<p>(X);
}

// Macroscopic state of a fluid node: c, mu (from the planes), rho (Eq. 14),
// 12 grad c_i (Eq. 20a with the Eq. 43 ghosts), u and p (Eqs. 13b, 13c),
// F_s + G, and in the general case grad rho, the F_a factor of Eq. 12 (Eq.
// 20b on mu_i, Eq. 43 ghosts) and 1/tau_g (Eqs. 15, 18b); the g populations.
// The g populations of the update node: FP64 keeps them in registers from
// the moments to the collision; FP32 storage reads them again there (from
// its shared-memory stage), which frees registers for more resident warps
// (GB300, 192x96x192, before the stage, reading again through L1: update
// 0.922 -> 0.642 ms; FP64 2.331 -> 2.372 ms the same way).
template <typename R>
constexpr bool kGReg3 = !kLo3<R>;

// Where a node's own planes (populations, rest lo parts, c_i u) are read
// from: global memory (plane stride PL, element o), or, with STG, the
// block's shared-memory stage (stride = block size, element = thread) that
// the update fills by asynchronous copies at its start; ready() waits for
// this thread's copies.
template <typename R, bool STG>
struct PopSrc {
    const R* b;  // plane 0 of the node
    long long pl;
    __device__ __forceinline__ R operator()(int q) const { return b[q * pl]; }
    __device__ __forceinline__ void ready() const
    {
        if constexpr (STG) asm volatile("cp.async.wait_all;" ::: "memory");
    }
};

template <typename R>
struct Node3 {
    R c1, c2, mu1, mu2, rho;
    R u[3], usq, p;
    R T[3];  // 3 (F_s + G)
    R H[3];  // grad rho + T
    R aF, itg;
    R g[Q];
};

template <bool UNI, typename R, bool STG, bool FUSE_MU = false>
__device__ __forceinline__ void node3(const Geo3& g, const Prm3<R>& P, const PopSrc<R, STG>& fs,
                                      const R* __restrict__ cpl, const R* __restrict__ mpl, uint32_t L,
                                      const Nb3& nb, long long o, Node3<R>& n)
{
    const long long PL = g.plane;
    constexpr bool FUSE = FUSE_MU && UNI;
    n.c1 = cpl[o];
    n.c2 = cpl[PL + o];
    if constexpr (!FUSE) {
        n.mu1 = mpl[o];
        n.mu2 = mpl[PL + o];
    }
    R d1[9], d2[9], s1[9], s2[9];
#pragma unroll
    for (int p = 0; p < 9; p++) {
        const long long ap = nb.at(L, o, 2 * p + 1), am = nb.at(L, o, 2 * p + 2);
        const R a1 = cpl[ap], b1 = cpl[am], a2 = cpl[PL + ap], b2 = cpl[PL + am];
        d1[p] = a1 - b1;
        d2[p] = a2 - b2;
        if constexpr (FUSE) {  // the c sums of the node's own mu
            s1[p] = a1 + b1;
            s2[p] = a2 + b2;
        } else if constexpr (!UNI) {
            s1[p] = mpl[ap] + mpl[am];
            s2[p] = mpl[PL + ap] + mpl[PL + am];
        }
    }
    if constexpr (FUSE) mu_from_sums(P, L, n.c1, n.c2, s1, s2, n.mu1, n.mu2);
    R G1[3], G2[3];
    G1[0] = fma(R(2.0), d1[0], (d1[3] + d1[4]) + (d1[5] + d1[6]));
    G1[1] = fma(R(2.0), d1[1], (d1[3] - d1[4]) + (d1[7] + d1[8]));
    G1[2] = fma(R(2.0), d1[2], (d1[5] - d1[6]) + (d1[7] - d1[8]));
    G2[0] = fma(R(2.0), d2[0], (d2[3] + d2[4]) + (d2[5] + d2[6]));
    G2[1] = fma(R(2.0), d2[1], (d2[3] - d2[4]) + (d2[7] + d2[8]));
    G2[2] = fma(R(2.0), d2[2], (d2[5] - d2[6]) + (d2[7] - d2[8]));
    // g moments from the sums and differences of opposite pairs
    fs.ready();
    if constexpr (kGReg3<R>) n.g[0] = fs(2 * Q);
    R gs[9], gd[9];
#pragma unroll
    for (int p = 0; p < 9; p++) {
        const R gp = fs(2 * Q + 2 * p + 1), gm = fs(2 * Q + 2 * p + 2);
        if constexpr (kGReg3<R>) {
            n.g[2 * p + 1] = gp;
            n.g[2 * p + 2] = gm;
        }
        gs[p] = gp + gm;
        gd[p] = gp - gm;
    }
    const R sum = (((gs[0] + gs[1]) + (gs[2] + gs[3])) + ((gs[4] + gs[5]) + (gs[6] + gs[7]))) + gs[8];
    R mom[3];
    mom[0] = gd[0] + ((gd[3] + gd[4]) + (gd[5] + gd[6]));
    mom[1] = gd[1] + ((gd[3] - gd[4]) + (gd[7] + gd[8]));
    mom[2] = gd[2] + ((gd[5] - gd[6]) + (gd[7] - gd[8]));
    // F_s = sum_i mu_i grad c_i with grad c_3 = -grad c_1 - grad c_2 and
    // mu_3 from sum_i mu_i / lambda_i = 0
    const R m1 = fma(P.qa[0][0], n.mu1, P.qa[0][1] * n.mu2);
    const R m2 = fma(P.qa[1][0], n.mu1, P.qa[1][1] * n.mu2);
    R F[3];
    if constexpr (UNI) {
        n.rho = P.rho0;
        F[0] = fma(m1, G1[0], fma(m2, G2[0], P.Gc[0]));
        F[1] = fma(m1, G1[1], fma(m2, G2[1], P.Gc[1]));
        F[2] = fma(m1, G1[2], m2 * G2[2]);
#pragma unroll
        for (int a = 0; a < 3; a++) n.u[a] = fma(P.hirho, F[a], P.irho * mom[a]);
        n.usq = fma(n.u[0], n.u[0], fma(n.u[1], n.u[1], n.u[2] * n.u[2]));
        // Eq. 13c: p = (1/2) [sum_{k != 0} g_k + rho w_0 (-3/2) u.u] (grad rho = 0)
        n.p = fma(R(0.5), sum, P.prho * n.usq);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            n.T[a] = R(3.0) * F[a];
            n.H[a] = n.T[a];
        }
        n.aF = R(0.0);
        n.itg = P.itg0;
    } else {
        n.rho = fma(n.c1, P.rho[0] - P.rho[2], fma(n.c2, P.rho[1] - P.rho[2], P.rho[2]));
        R gr[3];
#pragma unroll
        for (int a = 0; a < 3; a++) gr[a] = fma(P.drho12[0], G1[a], P.drho12[1] * G2[a]);
        F[0] = fma(m1, G1[0], fma(m2, G2[0], n.rho * P.gx));
        F[1] = fma(m1, G1[1], fma(m2, G2[1], n.rho * P.gy));
        F[2] = fma(m1, G1[2], m2 * G2[2]);
        const R ir = tlb::rcp(n.rho);
#pragma unroll
        for (int a = 0; a < 3; a++) n.u[a] = fma(R(0.5), F[a], mom[a]) * ir;
        n.usq = fma(n.u[0], n.u[0], fma(n.u[1], n.u[1], n.u[2] * n.u[2]));
        const R ug = fma(n.u[0], gr[0], fma(n.u[1], gr[1], n.u[2] * gr[2]));
        // Eq. 13c: p = (1/2) [sum_{k != 0} g_k + u.grad rho / 2 + rho w_0 (-3/2) u.u]
        n.p = fma(R(0.5), sum, fma(R(0.25), ug, (-R(0.25) * n.rho) * n.usq));
#pragma unroll
        for (int a = 0; a < 3; a++) {
            n.T[a] = R(3.0) * F[a];
            n.H[a] = gr[a] + n.T[a];
        }
        const R l1 = fma(-R(24.0), n.mu1, W36_SUM(s1));
        const R l2 = fma(-R(24.0), n.mu2, W36_SUM(s2));
        n.aF = fma(P.aM6[0], l1, P.aM6[1] * l2);
        const R nu = fma(n.c1, P.dnu[0], fma(n.c2, P.dnu[1], P.nu3));
        n.itg = tlb::rcp(fma(R(3.0), nu, R(0.5)));
    }
}

// Collision and push of opposite pair p (directions k = 2p + 1 and k + 1).
// With beta = 3 e_k.u and a = beta^2/2 - (3/2) u.u the BGK updates of Eqs. 1a,
// 1b with Eqs. 2a, 2b, 4, 11a, 11b take the form
//   f'_{k, k+1} = (1 - 1/tau) f + A_w +- V,
//   g'_{k, k+1} = (1 - 1/tau_g) g + Sym +- Anti,
//   Sym = beta K_X + a R_X + P_X,  Anti = a K_X + beta R_X + A_X,
// K_X = K_w e.H, R_X = w rho/tau_g - K_w u.H, P_X = 3 w p/tau_g - K_w u.T,
// A_X = K_w e.T + w a_F beta, K_w = w (1 - 1/(2 tau_g)).
template <typename R>
struct Coll3 {
    R omt1, omt2, omtg, t0;
    R A1[2], A2[2], RX[2], PX[2];
    R b3[3], Q1[3], Q2[3], Hs[3], Ts[3];
    R wa36;
};

template <bool UNI, int p, typename R, bool STG>
__device__ __forceinline__ void pair3(const Coll3<R>& C, const PopSrc<R, STG>& fs, R* __restrict__ fB,
                                      const Node3<R>& n, const Nb3& nb, uint32_t L, long long o, long long PL,
                                      R& d1, R& d2)
{
    constexpr int kp = 2 * p + 1, km = 2 * p + 2, c = p < 3 ? 0 : 1;
    const R beta = edot<p>(C.b3);
    const R KX = wdot<p>(C.Hs);
    // A_i +- V_i with V_i = 36 w_k e_k.Q'_i (on the axis pairs one fma each)
    R s1p, s1m, s2p, s2m;
    if constexpr (p < 3) {
        s1p = fma(R(2.0), C.Q1[p], C.A1[c]);
        s1m = fma(-R(2.0), C.Q1[p], C.A1[c]);
        s2p = fma(R(2.0), C.Q2[p], C.A2[c]);
        s2m = fma(-R(2.0), C.Q2[p], C.A2[c]);
    } else {
        const R V1 = edot<p>(C.Q1), V2 = edot<p>(C.Q2);
        s1p = C.A1[c] + V1;
        s1m = C.A1[c] - V1;
        s2p = C.A2[c] + V2;
        s2m = C.A2[c] - V2;
    }
    R AX;
    if constexpr (UNI) AX = KX;
    else AX = fma(p < 3 ? R(2.0) * C.wa36 : C.wa36, beta, wdot<p>(C.Ts));
    const R a = fma(beta, R(0.5) * beta, C.t0);
    const R sym = fma(beta, KX, fma(a, C.RX[c], C.PX[c]));
    const R anti = fma(a, KX, fma(beta, C.RX[c], AX));
    const R f1p = fs(kp), f1m = fs(km);
    const R f2p = fs(Q + kp), f2m = fs(Q + km);
    const R o1p = fma(C.omt1, f1p, s1p);
    const R o1m = fma(C.omt1, f1m, s1m);
    const R o2p = fma(C.omt2, f2p, s2p);
    const R o2m = fma(C.omt2, f2m, s2m);
    if constexpr (kLo3<R>) {
        // the moving populations' share of the rest pair update
        d1 += (f1p - o1p) + (f1m - o1m);
        d2 += (f2p - o2p) + (f2m - o2m);
    }
    R gkp, gkm;
    if constexpr (kGReg3<R>) {
        gkp = n.g[kp];
        gkm = n.g[km];
    } else {  // read again instead of holding 19 values in registers
        gkp = fs(2 * Q + kp);
        gkm = fs(2 * Q + km);
    }
    const R ogp = fma(C.omtg, gkp, sym + anti);
    const R ogm = fma(C.omtg, gkm, sym - anti);
    // push to x + e_k, or back into slot k-bar of this node (Eq. 44)
    const long long dp = (L >> (kp - 1)) & 1u ? kp * PL + o + nb.off(kp) : km * PL + o;
    const long long dm = (L >> (km - 1)) & 1u ? km * PL + o + nb.off(km) : kp * PL + o;
    fB[dp] = o1p;
    fB[Q * PL + dp] = o2p;
    fB[2 * Q * PL + dp] = ogp;
    fB[dm] = o1m;
    fB[Q * PL + dm] = o2m;
    fB[2 * Q * PL + dm] = ogm;
}

// One BGK time step of every fluid node: collision (Eqs. 1a, 1b, 2a, 2b, 4,
// 11a, 11b, 19) and the push to x + e_k.  UNI: equal densities and
// viscosities (grad rho = 0, F_a = 0, tau_g constant).
// resident blocks per SM the update is compiled for: the uniform-property
// update at 3 (168 registers, 16 bytes spilled; GB300, 192x96x192: R(2.447) ->
// R(2.348) ms per launch; R(2.344) at 4); the general update gains nothing at 2 or 3
#ifndef TLB3_MINB
#define TLB3_MINB 3
#endif
#ifndef TLB3_MINB_GEN
#define TLB3_MINB_GEN 1
#endif
// FP32 storage (bound by memory): resident blocks per SM of the uniform and
// the general update; with the stage below, GB300, 192x96x192, uniform:
// 0.432 / 0.377 / 0.370 / 0.384 ms per launch at 2 / 3 / 4 / 5 blocks (4: 128
// registers, 8 bytes spilled; the general update would spill 76 bytes at 4)
#ifndef TLB3_MINB32
#define TLB3_MINB32 4
#endif
#ifndef TLB3_MINB32_GEN
#define TLB3_MINB32_GEN 3
#endif
// FP32 storage: the update node's 59 population planes and 6 c_i u values
// are copied asynchronously into a shared-memory stage at the start of the
// update (no registers held while they are in flight; 33 KB per block) and
// read from there: GB300, 192x96x192, update 0.643 -> 0.377 ms per launch at
// 3 blocks per SM (whole step 4.40 -> 6.59 G node updates/s).  Before, the
// populations were loaded where each direction pair is collided, a memory
// latency the 12 resident warps per SM could not cover.
#ifndef TLB3_STAGE32
#define TLB3_STAGE32 1
#endif
// FP64: the same stage (57 + 6 rows of 8 bytes: 64.5 KB of dynamic shared
// memory per block) gains nothing, the update being bound by the FP64 unit:
// GB300, 192x96x192, uniform update 2.331 -> 2.339 ms per launch, general
// step 973.6 -> 976.7 M node updates/s; off
#ifndef TLB3_STAGE64
#define TLB3_STAGE64 0
#endif
template <typename R>
constexpr bool kStage3 = kLo3<R> ? TLB3_STAGE32 != 0 : TLB3_STAGE64 != 0;
// FP32 storage, uniform update: the node's mu computed in the update from
// the c stencil it loads anyway, so a step has no k3_mu launch and reads no
// mu plane (the general update needs the neighbours' mu: k3_mu stays)
#ifndef TLB3_FUSE_MU32
#define TLB3_FUSE_MU32 1
#endif
template <typename R>
constexpr bool kFuseMu3 = kLo3<R> && TLB3_FUSE_MU32 != 0;
template <typename R>
constexpr int kStageRows3 = kPlanes3<R> + 6;
// dynamic shared memory of one update block (the FP32 stage is static)
template <typename R>
constexpr size_t kStageDyn3 = (kStage3<R> && !kLo3<R>) ? sizeof(R) * 128 * kStageRows3<R> : 0;

template <int N>
__device__ __forceinline__ void cp_async(unsigned dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(N) : "memory");
}

template <typename R, bool UNI, bool STG>
__device__ __forceinline__ void update3_node(const PopSrc<R, STG>& fs, const PopSrc<R, STG>& cs, R* __restrict__ fB,
                                             R* __restrict__ cu, const R* __restrict__ cpl,
                                             const R* __restrict__ mpl, uint32_t L, const Geo3& g, int x, int y,
                                             int z, long long o, const Prm3<R>& P)
{
    const long long PL = g.plane;
    const Nb3 nb(g, x, y, z);
    Node3<R> n;
    node3<UNI, R, STG, kFuseMu3<R>>(g, P, fs, cpl, mpl, L, nb, o, n);
    constexpr R w0 = R(1.0) / R(3.0), w36 = R(1.0) / R(36.0);
    Coll3<R> C;
    // order parameters: Q_i = 3 w36 [c_i u / tau_i + (1 - 1/(2 tau_i)) d(c_i u)],
    // d(c_i u) against the previous step's (Eq. 19), which is replaced
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const R cu1 = n.c1 * n.u[a], cu2 = n.c2 * n.u[a];
        const R d1 = cu1 - cs(a), d2 = cu2 - cs(3 + a);
        cu[a * PL + o] = cu1;
        cu[(3 + a) * PL + o] = cu2;
        C.Q1[a] = fma(P.kq[0], cu1, P.sq[0] * d1);
        C.Q2[a] = fma(P.kq[1], cu2, P.sq[1] * d2);
    }
    C.omt1 = P.omt[0];
    C.omt2 = P.omt[1];
    const R E1 = fma(P.e0[0], n.mu1, P.itau[0] * n.c1);
    const R E2 = fma(P.e0[1], n.mu2, P.itau[1] * n.c2);
#pragma unroll
    for (int c = 0; c < 2; c++) {
        C.A1[c] = P.aw[0][c] * n.mu1;
        C.A2[c] = P.aw[1][c] * n.mu2;
    }
    // hydrodynamics
#pragma unroll
    for (int a = 0; a < 3; a++) C.b3[a] = R(3.0) * n.u[a];
    C.t0 = -R(1.5) * n.usq;
    R kG, Kw[2], Rw[2], p3;
    if constexpr (UNI) {
        C.omtg = P.omtg0;
        kG = P.kG0;
        Kw[0] = P.Kw0[0];
        Kw[1] = P.Kw0[1];
        Rw[0] = P.Rw0[0];
        Rw[1] = P.Rw0[1];
        p3 = n.p * P.p3tg0;
    } else {
        C.omtg = R(1.0) - n.itg;
        kG = fma(-R(0.5), n.itg, R(1.0));
        Kw[0] = (R(2.0) * w36) * kG;
        Kw[1] = w36 * kG;
        const R ri = n.rho * n.itg;
        Rw[0] = (R(2.0) * w36) * ri;
        Rw[1] = w36 * ri;
        p3 = R(3.0) * n.p * n.itg;
    }
    const R uT = fma(n.u[0], n.T[0], fma(n.u[1], n.T[1], n.u[2] * n.T[2]));
    R uH = uT;
    if constexpr (!UNI) uH = fma(n.u[0], n.H[0], fma(n.u[1], n.H[1], n.u[2] * n.H[2]));
#pragma unroll
    for (int c = 0; c < 2; c++) {
        C.RX[c] = fma(-Kw[c], uH, Rw[c]);
        C.PX[c] = fma(-Kw[c], uT, (c == 0 ? R(2.0) * w36 : w36) * p3);
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C.Hs[a] = Kw[1] * n.H[a];
        C.Ts[a] = UNI ? C.Hs[a] : Kw[1] * n.T[a];
    }
    C.wa36 = w36 * n.aF;
    // rest direction: g^eq_0 = 3p (w_0 - 1) + rho w_0 t0, G_0 = -w_0 K_G (t0 u.H + u.T)
    const R geq0 = fma(n.rho * w0, C.t0, (R(3.0) * (w0 - R(1.0))) * n.p);
    const R P0 = fma(geq0, n.itg, -(w0 * kG) * fma(C.t0, uH, uT));
    R d1 = R(0), d2 = R(0);  // sum_k (f_k - f'_k) over the moving directions (FP32)
    if constexpr (!kLo3<R>) {
        fB[o] = fma(C.omt1, fs(0), E1);
        fB[Q * PL + o] = fma(C.omt2, fs(Q), E2);
    }
    fB[2 * Q * PL + o] = fma(C.omtg, kGReg3<R> ? n.g[0] : fs(2 * Q), P0);
    pair3<UNI, 0>(C, fs, fB, n, nb, L, o, PL, d1, d2);
    pair3<UNI, 1>(C, fs, fB, n, nb, L, o, PL, d1, d2);
    pair3<UNI, 2>(C, fs, fB, n, nb, L, o, PL, d1, d2);
    pair3<UNI, 3>(C, fs, fB, n, nb, L, o, PL, d1, d2);
    pair3<UNI, 4>(C, fs, fB, n, nb, L, o, PL, d1, d2);
    pair3<UNI, 5>(C, fs, fB, n, nb, L, o, PL, d1, d2);
    pair3<UNI, 6>(C, fs, fB, n, nb, L, o, PL, d1, d2);
    pair3<UNI, 7>(C, fs, fB, n, nb, L, o, PL, d1, d2);
    pair3<UNI, 8>(C, fs, fB, n, nb, L, o, PL, d1, d2);
    if constexpr (kLo3<R>) {
        // rest pairs: the old pair plus the moving populations' decrease
        R h1, l1, h2, l2;
        rest_add3(fs(0), fs(kLoPlane), d1, h1, l1);
        rest_add3(fs(Q), fs(kLoPlane + 1), d2, h2, l2);
        fB[o] = h1;
        fB[Q * PL + o] = h2;
        fB[kLoPlane * PL + o] = l1;
        fB[(kLoPlane + 1) * PL + o] = l2;
    }
}

template <typename R, bool UNI>
__global__ void __launch_bounds__(128, kLo3<R> ? (UNI ? TLB3_MINB32 : TLB3_MINB32_GEN) : (UNI ? TLB3_MINB : TLB3_MINB_GEN))
k3_update(const R* __restrict__ fA, R* __restrict__ fB, R* __restrict__ cu,
          const R* __restrict__ cpl, const R* __restrict__ mpl, const uint32_t* __restrict__ lnk, Geo3 g,
          Prm3<R> P)
{
    NODE_OF_THREAD
    const long long PL = g.plane;
    if constexpr (kStage3<R>) {
        // launched with 128 threads: row q of the stage holds plane q of the
        // block's nodes (the 6 c_i u planes after the populations)
        R(*stg)[128];
        if constexpr (kLo3<R>) {
            __shared__ float s32[kStageRows3<float>][128];
            stg = s32;
        } else {
            extern __shared__ __align__(16) unsigned char s64[];
            stg = reinterpret_cast<R(*)[128]>(s64);
        }
        const int t = threadIdx.x;
        constexpr unsigned E = sizeof(R);
        const unsigned sb = (unsigned)__cvta_generic_to_shared(&stg[0][t]);
#pragma unroll
        for (int q = 0; q < kPlanes3<R>; q++) cp_async<E>(sb + E * 128u * q, fA + q * PL + o);
#pragma unroll
        for (int a = 0; a < 6; a++) cp_async<E>(sb + E * 128u * (kPlanes3<R> + a), cu + a * PL + o);
        const PopSrc<R, true> fs{&stg[0][t], 128}, cs{&stg[kPlanes3<R>][t], 128};
        const uint32_t L = lnk[o];
        if (L & LNK_SOLID) {
            fs.ready();  // no copy into the stage may outlive the block
            return;
        }
        update3_node<R, UNI>(fs, cs, fB, cu, cpl, mpl, L, g, x, y, z, o, P);
    } else {
        const uint32_t L = lnk[o];
        if (L & LNK_SOLID) return;
        update3_node<R, UNI>(PopSrc<R, false>{fA + o, PL}, PopSrc<R, false>{cu + o, PL}, fB, cu, cpl, mpl, L, g, x,
                             y, z, o, P);
    }
}

// c of every node from dense host-order arrays (c1 then c2, nx*ny*nz each).
template <typename R>
__global__ void k3_load_c(const double* __restrict__ in, R* __restrict__ cpl, const uint8_t* __restrict__ kind,
                          Geo3 g)
{
    NODE_OF_THREAD
    const long long n = ((long long)z * g.ny + y) * g.nx + x, N = (long long)g.nx * g.ny * g.nz;
    const bool fl = kind[o] == K_FLUID;
    cpl[o] = fl ? R(in[n]) : R(0.0);
    cpl[g.plane + o] = fl ? R(in[N + n]) : R(0.0);
}

// Initial state from c, mu (planes) and u, p (dense FP64 arrays ux, uy,
// uz[, p]): f = f^eq(c, mu, u), g = g^eq(p, rho, u), c_i u stored (Eq. 19);
// with FP32 storage the rest pairs start with lo = 0.
template <typename R>
__global__ void k3_init(R* __restrict__ f, R* __restrict__ cu, const R* __restrict__ cpl,
                        const R* __restrict__ mpl, const uint8_t* __restrict__ kind,
                        const double* __restrict__ in, int has_p, Geo3 g, Prm3<R> P)
{
    NODE_OF_THREAD
    const long long PL = g.plane;
    const long long n = ((long long)z * g.ny + y) * g.nx + x, N = (long long)g.nx * g.ny * g.nz;
    if (kind[o] != K_FLUID) {
        for (int q = 0; q < kPlanes3<R>; q++) f[q * PL + o] = R(0.0);
        for (int q = 0; q < 6; q++) cu[q * PL + o] = R(0.0);
        return;
    }
    const R c[2] = {cpl[o], cpl[PL + o]}, mu[2] = {mpl[o], mpl[PL + o]};
    const R u[3] = {R(in[n]), R(in[N + n]), R(in[2 * N + n])};
    const R p = has_p ? R(in[3 * N + n]) : R(0.0);
    const R rho = c[0] * P.rho[0] + c[1] * P.rho[1] + (R(1.0) - c[0] - c[1]) * P.rho[2];
    const R usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int k = 0; k < Q; k++) {
        const R w = R(wk(k));
        const R eu = R(ex(k)) * u[0] + R(ey(k)) * u[1] + R(ez(k)) * u[2];
        const R s = w * (R(3.0) * eu + R(4.5) * eu * eu - R(1.5) * usq);
        for (int q = 0; q < 2; q++) {
            const R em = P.eta[q] * mu[q];
            f[(Q * q + k) * PL + o] = k == 0 ? c[q] + (w - R(1.0)) * em : w * (em + R(3.0) * c[q] * eu);
        }
        f[(2 * Q + k) * PL + o] = k == 0 ? R(3.0) * p * (w - R(1.0)) + rho * s : R(3.0) * p * w + rho * s;
    }
    if constexpr (kLo3<R>) {
        f[kLoPlane * PL + o] = R(0.0);
        f[(kLoPlane + 1) * PL + o] = R(0.0);
    }
    for (int q = 0; q < 2; q++)
        for (int a = 0; a < 3; a++) cu[(3 * q + a) * PL + o] = c[q] * u[a];
}

// The 11 macroscopic fields c1 c2 c3 rho ux uy uz p mu1 mu2 mu3 as dense FP64
// planes of nx*ny*nz (zero on solids), from the same node3 as the update.
template <typename R, bool UNI>
__global__ void k3_read(const R* __restrict__ f, const R* __restrict__ cpl, const R* __restrict__ mpl,
                        const uint32_t* __restrict__ lnk, double* __restrict__ out, Geo3 g, Prm3<R> P)
{
    NODE_OF_THREAD
    const long long n = ((long long)z * g.ny + y) * g.nx + x, N = (long long)g.nx * g.ny * g.nz;
    double v[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const uint32_t L = lnk[o];
    if (!(L & LNK_SOLID)) {
        const Nb3 nb(g, x, y, z);
        Node3<R> m;
        node3<UNI>(g, P, PopSrc<R, false>{f + o, g.plane}, cpl, mpl, L, nb, o, m);
        v[0] = m.c1;
        v[1] = m.c2;
        v[2] = R(1.0) - m.c1 - m.c2;
        v[3] = m.rho;
        v[4] = m.u[0];
        v[5] = m.u[1];
        v[6] = m.u[2];
        v[7] = m.p;
        v[8] = m.mu1;
        v[9] = m.mu2;
        v[10] = -(P.l3_l1 * m.mu1 + P.l3_l2 * m.mu2);
    }
    for (int q = 0; q < 11; q++) out[q * N + n] = v[q];
}

// FP64 mass totals in a fixed order: per-block partials of c1, c2, c3 and
// the non-finite count over fluid nodes, each c_i summed in FP64 from the
// stored populations (FP32 storage: the rest pairs' lo parts included), then
// one block.
template <typename R>
__global__ void __launch_bounds__(256) k3_mass_partials(const R* __restrict__ f,
                                                        const uint8_t* __restrict__ kind, double* __restrict__ part,
                                                        Geo3 g)
{
    __shared__ double red[4][256];
    const long long N = (long long)g.nx * g.ny * g.nz;
    double s[4] = {0, 0, 0, 0};
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % g.nx);
        const long long r = n / g.nx;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        const long long o = node_off(g, x, y, z);
        if (kind[o] != K_FLUID) continue;
        const long long PL = g.plane;
        double c1 = 0.0, c2 = 0.0;
        if constexpr (kLo3<R>) {
            c1 = (double)f[kLoPlane * PL + o];
            c2 = (double)f[(kLoPlane + 1) * PL + o];
        }
        for (int k = 0; k < Q; k++) {
            c1 += (double)f[k * PL + o];
            c2 += (double)f[(Q + k) * PL + o];
        }
        s[0] += c1;
        s[1] += c2;
        s[2] += 1.0 - c1 - c2;
        if (!isfinite(c1) || !isfinite(c2)) s[3] += 1.0;
    }
    for (int q = 0; q < 4; q++) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; q++) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) k3_mass_final(const double* __restrict__ part, int nparts,
                                                     double* __restrict__ out)
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

}  // namespace tlb3

// ---------------------------------------------------------------------------
// C ABI (include/tlbm.h, "D3Q19")
// ---------------------------------------------------------------------------

namespace {

constexpr int64_t kAlign3 = 256;
constexpr int kMassParts3 = 608;
int64_t align3(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

int err3(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return tlb::set_error(code, buf);
}

#define T3_CUDA(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return err3(TLB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

struct Layout3 {
    int pitch = 0;
    int64_t plane = 0;
    int64_t fA = 0, fB = 0, cu = 0, cpl = 0, mpl = 0, lnk = 0, kind = 0, part = 0, diag = 0, total = 0;
};

// at least 3 nodes per axis; fewer than 2^31 nodes (one 32-bit thread index per node)
bool size_ok(int nx, int ny, int nz)
{
    return nx >= 3 && ny >= 3 && nz >= 3 && (int64_t)nx * ny * nz < ((int64_t)1 << 31);
}

// FP64: 57 distribution planes per buffer; FP32: 59 (the rest pairs' lo
// parts); c_i u, c and mu planes in the storage type.  Either buffer holds at
// least 6 FP64 planes (the staging of tlb3_set_fields) and 11 (tlb3_read_fields).
Layout3 layout3(int nx, int ny, int nz, int precision)
{
    Layout3 L;
    L.pitch = (int)align3(nx, 32);
    L.plane = (int64_t)L.pitch * ny * nz;
    const int64_t e = precision == TLB_FP32 ? 4 : 8;
    const int np = precision == TLB_FP32 ? tlb3::kPlanes3<float> : tlb3::kPlanes3<double>;
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        const int64_t at = off;
        off = align3(off + bytes, kAlign3);
        return at;
    };
    L.fA = take(np * L.plane * e);
    L.fB = take(np * L.plane * e);
    L.cu = take(6 * L.plane * e);
    L.cpl = take(2 * L.plane * e);
    L.mpl = take(2 * L.plane * e);
    L.lnk = take(L.plane * 4);
    L.kind = take(L.plane);
    L.part = take((int64_t)kMassParts3 * 4 * 8);
    L.diag = take(4 * 8);
    L.total = off;
    return L;
}

}  // namespace

struct tlb3_lattice {
    int nx = 0, ny = 0, nz = 0, device = 0;
    int32_t edge[6] = {0, 0, 0, 0, 0, 0};
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    Layout3 lay;
    tlb3::Geo3 geo{};
    int prec = TLB_FP64;
    tlb3::Prm3<double> prm{};
    tlb3::Prm3<float> prmf{};
    int cur = 0;
    bool have_params = false, have_fields = false, uni = false;
    std::vector<uint8_t> mask;
    // per-kernel timing (tlb3_profile): 4 events per step around the three launches
    bool prof = false;
    bool stage_attr = false;  // the update's dynamic shared memory limit raised
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    double prof_ms[3] = {0, 0, 0};
    int64_t prof_n[3] = {0, 0, 0};

    // the regions in the storage type R
    template <typename R>
    R* buf(int which) { return (R*)(ws + (which == 0 ? lay.fA : lay.fB)); }
    template <typename R>
    R* fcur() { return buf<R>(cur); }
    template <typename R>
    R* fspare() { return buf<R>(cur ^ 1); }
    template <typename R>
    R* cu() { return (R*)(ws + lay.cu); }
    template <typename R>
    R* cpl() { return (R*)(ws + lay.cpl); }
    template <typename R>
    R* mpl() { return (R*)(ws + lay.mpl); }
    double* stage() { return (double*)(ws + (cur ? lay.fA : lay.fB)); }  // the spare buffer as FP64 staging
    template <typename R>
    const tlb3::Prm3<R>& P() const
    {
        if constexpr (std::is_same<R, float>::value) return prmf;
        else return prm;
    }
    uint8_t* kind() { return (uint8_t*)(ws + lay.kind); }
    uint32_t* lnk() { return (uint32_t*)(ws + lay.lnk); }
    int64_t n() const { return (int64_t)nx * ny * nz; }
};

namespace {

int check3(tlb3_lattice* L)
{
    if (!L) return err3(TLB_EINVAL, "null lattice handle");
    T3_CUDA(cudaSetDevice(L->device));
    return TLB_OK;
}

dim3 grid3(const tlb3_lattice* L) { return dim3((unsigned)((L->n() + 127) / 128)); }

constexpr int kProfSteps3 = 256;

// Adds the recorded intervals to the totals (synchronizes on the last event).
int prof_fold3(tlb3_lattice* L)
{
    if (L->ev_used == 0) return TLB_OK;
    T3_CUDA(cudaEventSynchronize(L->ev[4 * (L->ev_used - 1) + 3]));
    for (int u = 0; u < L->ev_used; u++)
        for (int j = 0; j < 3; j++) {
            float ms = 0.0f;
            T3_CUDA(cudaEventElapsedTime(&ms, L->ev[4 * u + j], L->ev[4 * u + j + 1]));
            L->prof_ms[j] += ms;
            L->prof_n[j]++;
        }
    L->ev_used = 0;
    return TLB_OK;
}

// event j (0..3) of the current profiled step
int prof_mark3(tlb3_lattice* L, int j)
{
    if (!L->prof) return TLB_OK;
    T3_CUDA(cudaEventRecord(L->ev[4 * L->ev_used + j], L->stream));
    if (j == 3) L->ev_used++;
    return TLB_OK;
}

// c and mu planes of the current state (the first two launches of a step;
// in_step: mu only where the update does not form it itself)
template <typename R>
int order_params3_t(tlb3_lattice* L, bool in_step)
{
    tlb3::k3_csum<R><<<grid3(L), 128, 0, L->stream>>>(L->fcur<R>(), L->cpl<R>(), L->kind(), L->geo);
    int rc = prof_mark3(L, 1);
    if (rc) return rc;
    if (!(in_step && L->uni && tlb3::kFuseMu3<R>))
        tlb3::k3_mu<R><<<grid3(L), 128, 0, L->stream>>>(L->cpl<R>(), L->mpl<R>(), L->lnk(), L->geo, L->P<R>());
    T3_CUDA(cudaGetLastError());
    return TLB_OK;
}
int order_params3(tlb3_lattice* L, bool in_step = false)
{
    return L->prec == TLB_FP32 ? order_params3_t<float>(L, in_step) : order_params3_t<double>(L, in_step);
}

// the fused update and push of one step, current buffer -> spare buffer
template <typename R>
int update3_t(tlb3_lattice* L)
{
    constexpr size_t dyn = tlb3::kStageDyn3<R>;
    if (dyn > 0 && !L->stage_attr) {
        // above the default 48 KB of dynamic shared memory (per device: the
        // lattice lives on one)
        T3_CUDA(cudaFuncSetAttribute(tlb3::k3_update<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        T3_CUDA(cudaFuncSetAttribute(tlb3::k3_update<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        L->stage_attr = true;
    }
    if (L->uni)
        tlb3::k3_update<R, true><<<grid3(L), 128, dyn, L->stream>>>(L->fcur<R>(), L->fspare<R>(), L->cu<R>(),
                                                                    L->cpl<R>(), L->mpl<R>(), L->lnk(), L->geo,
                                                                    L->P<R>());
    else
        tlb3::k3_update<R, false><<<grid3(L), 128, dyn, L->stream>>>(L->fcur<R>(), L->fspare<R>(), L->cu<R>(),
                                                                     L->cpl<R>(), L->mpl<R>(), L->lnk(), L->geo,
                                                                     L->P<R>());
    T3_CUDA(cudaGetLastError());
    return TLB_OK;
}

// initial state from the FP64 staging (c1, c2 at stage, then ux, uy, uz[, p])
template <typename R>
int init3_t(tlb3_lattice* L, const double* stage, bool has_p)
{
    const size_t N = (size_t)L->n();
    tlb3::k3_load_c<R><<<grid3(L), 128, 0, L->stream>>>(stage, L->cpl<R>(), L->kind(), L->geo);
    tlb3::k3_mu<R><<<grid3(L), 128, 0, L->stream>>>(L->cpl<R>(), L->mpl<R>(), L->lnk(), L->geo, L->P<R>());
    tlb3::k3_init<R><<<grid3(L), 128, 0, L->stream>>>(L->fcur<R>(), L->cu<R>(), L->cpl<R>(), L->mpl<R>(), L->kind(),
                                                      stage + 2 * N, has_p ? 1 : 0, L->geo, L->P<R>());
    T3_CUDA(cudaGetLastError());
    return TLB_OK;
}

// the 11 fields as FP64 planes into `out` (device)
template <typename R>
int read3_t(tlb3_lattice* L, double* out)
{
    if (L->uni)
        tlb3::k3_read<R, true><<<grid3(L), 128, 0, L->stream>>>(L->fcur<R>(), L->cpl<R>(), L->mpl<R>(), L->lnk(), out,
                                                                L->geo, L->P<R>());
    else
        tlb3::k3_read<R, false><<<grid3(L), 128, 0, L->stream>>>(L->fcur<R>(), L->cpl<R>(), L->mpl<R>(), L->lnk(), out,
                                                                 L->geo, L->P<R>());
    T3_CUDA(cudaGetLastError());
    return TLB_OK;
}

// FP64 mass totals of the current state into the diag slots
template <typename R>
int mass3_t(tlb3_lattice* L, double* part, double* diag)
{
    tlb3::k3_mass_partials<R><<<kMassParts3, 256, 0, L->stream>>>(L->fcur<R>(), L->kind(), part, L->geo);
    tlb3::k3_mass_final<<<1, 256, 0, L->stream>>>(part, kMassParts3, diag);
    T3_CUDA(cudaGetLastError());
    return TLB_OK;
}

// link words from the node kinds (after every change of the geometry)
int links3(tlb3_lattice* L)
{
    tlb3::k3_links<<<grid3(L), 128, 0, L->stream>>>(L->kind(), L->lnk(), L->geo);
    T3_CUDA(cudaGetLastError());
    return TLB_OK;
}

}  // namespace

extern "C" {

int64_t tlb3_workspace_bytes(int nx, int ny, int nz, int precision)
{
    if (!size_ok(nx, ny, nz)) return err3(TLB_EINVAL, "lattice size %dx%dx%d out of range", nx, ny, nz);
    if (precision != TLB_FP64 && precision != TLB_FP32) return err3(TLB_EINVAL, "precision must be TLB_FP64 or TLB_FP32");
    tlb::clear_error();
    return layout3(nx, ny, nz, precision).total;
}

int tlb3_create(int nx, int ny, int nz, int precision, const int32_t edges[6], void* dev_workspace,
                int64_t ws_bytes, void* cuda_stream, tlb3_lattice** out)
{
    if (!out) return err3(TLB_EINVAL, "out is null");
    *out = nullptr;
    if (!size_ok(nx, ny, nz)) return err3(TLB_EINVAL, "lattice size %dx%dx%d out of range", nx, ny, nz);
    if (precision != TLB_FP64 && precision != TLB_FP32) return err3(TLB_EINVAL, "precision must be TLB_FP64 or TLB_FP32");
    if (!edges) return err3(TLB_EINVAL, "edges is null");
    for (int a = 0; a < 3; a++) {
        const int lo = edges[2 * a], hi = edges[2 * a + 1];
        if (lo < 0 || lo > 2 || hi < 0 || hi > 2)
            return err3(TLB_EINVAL, "edge kinds must be periodic, wetting or neutral (no lid in 3D)");
        if ((lo == 0) != (hi == 0)) return err3(TLB_EINVAL, "a periodic edge needs a periodic opposite edge");
    }
    const Layout3 lay = layout3(nx, ny, nz, precision);
    if (!dev_workspace || ((uintptr_t)dev_workspace) % kAlign3) return err3(TLB_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < lay.total)
        return err3(TLB_ENOMEM, "workspace has %lld bytes, needs %lld", (long long)ws_bytes, (long long)lay.total);
    auto* L = new tlb3_lattice;
    L->prec = precision;
    L->nx = nx;
    L->ny = ny;
    L->nz = nz;
    for (int e = 0; e < 6; e++) L->edge[e] = edges[e];
    L->stream = (cudaStream_t)cuda_stream;
    L->ws = (char*)dev_workspace;
    L->lay = lay;
    if (cudaGetDevice(&L->device) != cudaSuccess) {
        delete L;
        return err3(TLB_ECUDA, "no current device");
    }
    L->geo.nx = nx;
    L->geo.ny = ny;
    L->geo.nz = nz;
    L->geo.pitch = lay.pitch;
    L->geo.plane = lay.plane;
    for (int e = 0; e < 6; e++) L->geo.edge[e] = edges[e];
    L->mask.assign((size_t)L->n(), 0);
    if (cudaMemsetAsync(L->ws + lay.kind, 0, (size_t)lay.plane, L->stream) != cudaSuccess || links3(L) != TLB_OK ||
        cudaStreamSynchronize(L->stream) != cudaSuccess) {
        delete L;
        return err3(TLB_ECUDA, "clearing the node kinds failed");
    }
    *out = L;
    return tlb::clear_error();
}

int tlb3_set_geometry(tlb3_lattice* L, const uint8_t* host_mask)
{
    int rc = check3(L);
    if (rc) return rc;
    const int64_t N = L->n();
    std::vector<uint8_t> kind((size_t)L->lay.plane, 0);
    for (int64_t i = 0; i < N; i++) {
        const uint8_t m = host_mask ? host_mask[i] : 0;
        if (m > 2) return err3(TLB_EINVAL, "mask value %d at node %lld (0 fluid, 1 wetting, 2 neutral)", m, (long long)i);
        const int64_t x = i % L->nx, r = i / L->nx;
        kind[(size_t)(r * L->lay.pitch + x)] = m == 0 ? tlb3::K_FLUID : (m == 1 ? tlb3::K_WET : tlb3::K_NEUTRAL);
        L->mask[(size_t)i] = m;
    }
    T3_CUDA(cudaMemcpyAsync(L->kind(), kind.data(), kind.size(), cudaMemcpyHostToDevice, L->stream));
    if ((rc = links3(L))) return rc;
    T3_CUDA(cudaStreamSynchronize(L->stream));
    L->have_fields = false;
    return tlb::clear_error();
}

int tlb3_set_params(tlb3_lattice* L, const tlb_params* p)
{
    int rc = check3(L);
    if (rc) return rc;
    if (!p) return err3(TLB_EINVAL, "params is null");
    const double v[] = {p->sigma12, p->sigma13, p->sigma23, p->theta12_deg, p->theta13_deg, p->theta23_deg,
                        p->rho1, p->rho2, p->rho3, p->nu1, p->nu2, p->nu3, p->M0, p->D, p->tau1, p->tau2, p->gx, p->gy};
    for (double x : v)
        if (!std::isfinite(x)) return err3(TLB_EINVAL, "non-finite parameter");
    if (p->collision != 0.0) return err3(TLB_EINVAL, "the D3Q19 lattice has the BGK collision only (collision = 0)");
    if (p->lid_u != 0.0) return err3(TLB_EINVAL, "the D3Q19 lattice has no velocity lid (lid_u = 0)");
    if (p->sigma12 <= 0 || p->sigma13 <= 0 || p->sigma23 <= 0) return err3(TLB_EINVAL, "surface tensions must be > 0");
    const double l1 = p->sigma12 + p->sigma13 - p->sigma23;
    const double l2 = p->sigma12 + p->sigma23 - p->sigma13;
    const double l3 = p->sigma13 + p->sigma23 - p->sigma12;
    if (l1 <= 0 || l2 <= 0 || l3 < 0) return err3(TLB_EINVAL, "Eq. 7 gives lambda = (%g, %g, %g): need l1, l2 > 0, l3 >= 0", l1, l2, l3);
    if (p->D <= 0 || p->rho1 <= 0 || p->rho2 <= 0 || p->rho3 <= 0 || p->nu1 <= 0 || p->nu2 <= 0 || p->nu3 <= 0 || p->M0 <= 0)
        return err3(TLB_EINVAL, "D, densities, viscosities and M0 must be > 0");
    if (p->tau1 <= 0.5 || p->tau2 <= 0.5) return err3(TLB_EINVAL, "tau_i must be > 1/2");
    const double deg = 3.14159265358979323846 / 180.0;
    const double c12 = std::cos(p->theta12_deg * deg), c13 = std::cos(p->theta13_deg * deg),
                 c23 = std::cos(p->theta23_deg * deg);
    const double smax = std::fmax(p->sigma12, std::fmax(p->sigma13, p->sigma23));
    const double resid = p->sigma12 * c12 - p->sigma13 * c13 + p->sigma23 * c23;
    if (std::fabs(resid) > 1e-6 * smax) return err3(TLB_EINVAL, "contact angles violate Eq. 39 (residual %g)", resid);
    const double den = l1 * l2 + l1 * l3 + l2 * l3;
    const double lamT = den != 0 ? 3.0 * l1 * l2 * l3 / den : 0.0;  // Eq. 9, continuous form
    const double lam[2] = {l1, l2}, tau[2] = {p->tau1, p->tau2};
    const double rho[3] = {p->rho1, p->rho2, p->rho3}, nu[3] = {p->nu1, p->nu2, p->nu3};
    constexpr double w0 = 1.0 / 3.0, w18 = 1.0 / 18.0, w36 = 1.0 / 36.0;
    tlb3::Prm3<double> P{};
    for (int i = 0; i < 3; i++) {
        P.rho[i] = rho[i];
        P.nu[i] = nu[i];
    }
    P.l3_l1 = l3 / l1;
    P.l3_l2 = l3 / l2;
    P.k4D = 4.0 / p->D;
    P.cos12 = c12;
    P.cos13 = c13;
    P.cos23 = c23;
    P.kT = 24.0 * lamT / p->D;
    P.qa[0][0] = (1.0 + P.l3_l1) / 12.0;
    P.qa[0][1] = P.l3_l2 / 12.0;
    P.qa[1][0] = P.l3_l1 / 12.0;
    P.qa[1][1] = (1.0 + P.l3_l2) / 12.0;
    P.nu3 = nu[2];
    P.gx = p->gx;
    P.gy = p->gy;
    for (int i = 0; i < 2; i++) {
        const double M = p->M0 / lam[i];                       // Eq. 12
        P.eta[i] = M / ((1.0 / 3.0) * (tau[i] - 0.5));         // Eq. 18a, per component
        P.kl[i] = 12.0 * lam[i] / p->D;
        P.kd6[i] = 0.75 * p->D * lam[i] / 6.0;
        P.drho12[i] = (rho[i] - rho[2]) / 12.0;
        P.aM6[i] = (rho[i] - rho[2]) * M / 6.0;
        P.dnu[i] = nu[i] - nu[2];
        P.omt[i] = 1.0 - 1.0 / tau[i];
        P.itau[i] = 1.0 / tau[i];
        P.e0[i] = (w0 - 1.0) * P.eta[i] / tau[i];
        P.aw[i][0] = w18 * P.eta[i] / tau[i];
        P.aw[i][1] = w36 * P.eta[i] / tau[i];
        P.kq[i] = 3.0 * w36 / tau[i];
        P.sq[i] = 3.0 * w36 * (1.0 - 0.5 / tau[i]);
    }
    // uniform properties: the constants of the UNI update
    P.rho0 = rho[0];
    P.irho = 1.0 / rho[0];
    P.hirho = 0.5 / rho[0];
    P.prho = -0.25 * rho[0];
    P.itg0 = 1.0 / (3.0 * nu[0] + 0.5);
    P.omtg0 = 1.0 - P.itg0;
    P.kG0 = 1.0 - 0.5 * P.itg0;
    P.Kw0[0] = w18 * P.kG0;
    P.Kw0[1] = w36 * P.kG0;
    P.Rw0[0] = w18 * rho[0] * P.itg0;
    P.Rw0[1] = w36 * rho[0] * P.itg0;
    P.p3tg0 = 3.0 * P.itg0;
    P.Gc[0] = rho[0] * p->gx;
    P.Gc[1] = rho[0] * p->gy;
    L->prm = P;
    // the FP32 copy: every member of Prm3 is one scalar of its type
    static_assert(sizeof(tlb3::Prm3<double>) == 2 * sizeof(tlb3::Prm3<float>), "Prm3 holds scalars only");
    {
        const double* src = reinterpret_cast<const double*>(&L->prm);
        float* dst = reinterpret_cast<float*>(&L->prmf);
        for (size_t i = 0; i < sizeof(tlb3::Prm3<double>) / sizeof(double); i++) dst[i] = (float)src[i];
    }
    L->uni = rho[0] == rho[1] && rho[1] == rho[2] && nu[0] == nu[1] && nu[1] == nu[2];
    L->have_params = true;
    return tlb::clear_error();
}

int tlb3_set_fields(tlb3_lattice* L, const double* c1, const double* c2, const double* ux, const double* uy,
                    const double* uz, const double* p)
{
    int rc = check3(L);
    if (rc) return rc;
    if (!L->have_params) return err3(TLB_ESTATE, "set_params first");
    if (!c1 || !c2 || !ux || !uy || !uz) return err3(TLB_EINVAL, "c1, c2, ux, uy, uz must not be null");
    const size_t N = (size_t)L->n(), bytes = N * sizeof(double);
    double* stage = L->stage();  // the spare buffer: room for >= 11 FP64 planes of N
    T3_CUDA(cudaMemcpyAsync(stage, c1, bytes, cudaMemcpyHostToDevice, L->stream));
    T3_CUDA(cudaMemcpyAsync(stage + N, c2, bytes, cudaMemcpyHostToDevice, L->stream));
    double* in = stage + 2 * N;
    T3_CUDA(cudaMemcpyAsync(in, ux, bytes, cudaMemcpyHostToDevice, L->stream));
    T3_CUDA(cudaMemcpyAsync(in + N, uy, bytes, cudaMemcpyHostToDevice, L->stream));
    T3_CUDA(cudaMemcpyAsync(in + 2 * N, uz, bytes, cudaMemcpyHostToDevice, L->stream));
    if (p) T3_CUDA(cudaMemcpyAsync(in + 3 * N, p, bytes, cudaMemcpyHostToDevice, L->stream));
    rc = L->prec == TLB_FP32 ? init3_t<float>(L, stage, p != nullptr) : init3_t<double>(L, stage, p != nullptr);
    if (rc) return rc;
    T3_CUDA(cudaStreamSynchronize(L->stream));
    L->have_fields = true;
    return tlb::clear_error();
}

int tlb3_step(tlb3_lattice* L, int64_t n)
{
    int rc = check3(L);
    if (rc) return rc;
    if (n < 0) return err3(TLB_EINVAL, "negative step count");
    if (!L->have_params || !L->have_fields) return err3(TLB_ESTATE, "set_params and set_fields first");
    for (int64_t s = 0; s < n; s++) {
        if (L->prof && L->ev_used == kProfSteps3 && (rc = prof_fold3(L))) return rc;
        if ((rc = prof_mark3(L, 0))) return rc;
        if ((rc = order_params3(L, true))) return rc;
        if ((rc = prof_mark3(L, 2))) return rc;
        if ((rc = L->prec == TLB_FP32 ? update3_t<float>(L) : update3_t<double>(L))) return rc;
        if ((rc = prof_mark3(L, 3))) return rc;
        L->cur ^= 1;
    }
    return tlb::clear_error();
}

int tlb3_profile(tlb3_lattice* L, int enable)
{
    int rc = check3(L);
    if (rc) return rc;
    if (enable && L->ev.empty()) {
        L->ev.resize(4 * kProfSteps3);
        for (auto& e : L->ev) T3_CUDA(cudaEventCreate(&e));
    }
    if (!enable && (rc = prof_fold3(L))) return rc;
    L->prof = enable != 0;
    for (int j = 0; j < 3; j++) {
        L->prof_ms[j] = 0.0;
        L->prof_n[j] = 0;
    }
    L->ev_used = 0;
    return tlb::clear_error();
}

int tlb3_profile_read(tlb3_lattice* L, double ms[3], int64_t launches[3])
{
    int rc = check3(L);
    if (rc) return rc;
    if (!ms || !launches) return err3(TLB_EINVAL, "null output");
    if ((rc = prof_fold3(L))) return rc;
    for (int j = 0; j < 3; j++) {
        ms[j] = L->prof_ms[j];
        launches[j] = L->prof_n[j];
    }
    return tlb::clear_error();
}

int tlb3_sync(tlb3_lattice* L)
{
    int rc = check3(L);
    if (rc) return rc;
    T3_CUDA(cudaStreamSynchronize(L->stream));
    return tlb::clear_error();
}

int tlb3_read_fields(tlb3_lattice* L, uint32_t mask, double* host_out)
{
    int rc = check3(L);
    if (rc) return rc;
    if (!L->have_params || !L->have_fields) return err3(TLB_ESTATE, "no state yet");
    if (!host_out || !mask || (mask >> 11)) return err3(TLB_EINVAL, "bad output or field mask (11 fields)");
    if ((rc = order_params3(L))) return rc;
    const size_t N = (size_t)L->n();
    double* stage = L->stage();
    if ((rc = L->prec == TLB_FP32 ? read3_t<float>(L, stage) : read3_t<double>(L, stage))) return rc;
    size_t done = 0;
    for (int q = 0; q < 11; q++) {
        if (!(mask & (1u << q))) continue;
        T3_CUDA(cudaMemcpyAsync(host_out + done * N, stage + q * N, N * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
        done++;
    }
    T3_CUDA(cudaStreamSynchronize(L->stream));
    return tlb::clear_error();
}

int tlb3_read_state(tlb3_lattice* L, double* host_out)
{
    int rc = check3(L);
    if (rc) return rc;
    if (!L->have_fields) return err3(TLB_ESTATE, "no state yet");
    if (!host_out) return err3(TLB_EINVAL, "host_out is null");
    const size_t N = (size_t)L->n(), rows = (size_t)L->ny * L->nz;
    const size_t PL = (size_t)L->lay.plane;
    if (L->prec == TLB_FP32) {
        // 57 + 2 lo + 6 FP32 planes to the host, then widened; the rest
        // populations reported as hi + lo
        std::vector<float> h((size_t)65 * N);
        for (int q = 0; q < 65; q++) {
            const float* src = q < 59 ? L->fcur<float>() + q * PL : L->cu<float>() + (q - 59) * PL;
            T3_CUDA(cudaMemcpy2DAsync(h.data() + q * N, (size_t)L->nx * sizeof(float), src,
                                      (size_t)L->lay.pitch * sizeof(float), (size_t)L->nx * sizeof(float), rows,
                                      cudaMemcpyDeviceToHost, L->stream));
        }
        T3_CUDA(cudaStreamSynchronize(L->stream));
        for (int q = 0; q < 63; q++) {
            const float* src = h.data() + (size_t)(q < 57 ? q : q + 2) * N;
            for (size_t i = 0; i < N; i++) host_out[q * N + i] = (double)src[i];
        }
        for (int c = 0; c < 2; c++) {
            const float* lo = h.data() + (size_t)(tlb3::kLoPlane + c) * N;
            double* rest = host_out + (size_t)(c * tlb3::Q) * N;
            for (size_t i = 0; i < N; i++) rest[i] += (double)lo[i];
        }
    } else {
        for (int q = 0; q < 63; q++) {
            const double* src = q < 57 ? L->fcur<double>() + q * PL : L->cu<double>() + (q - 57) * PL;
            T3_CUDA(cudaMemcpy2DAsync(host_out + q * N, (size_t)L->nx * sizeof(double), src,
                                      (size_t)L->lay.pitch * sizeof(double), (size_t)L->nx * sizeof(double), rows,
                                      cudaMemcpyDeviceToHost, L->stream));
        }
        T3_CUDA(cudaStreamSynchronize(L->stream));
    }
    // solid nodes hold no populations (their slots in the two buffers also
    // serve as staging for set_fields and read_fields): report zeros
    for (size_t i = 0; i < N; i++)
        if (L->mask[i])
            for (int q = 0; q < 63; q++) host_out[q * N + i] = 0.0;
    return tlb::clear_error();
}

int tlb3_diagnostics(tlb3_lattice* L, tlb_diag* out)
{
    int rc = check3(L);
    if (rc) return rc;
    if (!L->have_params || !L->have_fields) return err3(TLB_ESTATE, "no state yet");
    if (!out) return err3(TLB_EINVAL, "out is null");
    double* part = (double*)(L->ws + L->lay.part);
    double* diag = (double*)(L->ws + L->lay.diag);
    if ((rc = L->prec == TLB_FP32 ? mass3_t<float>(L, part, diag) : mass3_t<double>(L, part, diag))) return rc;
    double h[4];
    T3_CUDA(cudaMemcpyAsync(h, diag, sizeof h, cudaMemcpyDeviceToHost, L->stream));
    T3_CUDA(cudaStreamSynchronize(L->stream));
    for (int i = 0; i < 3; i++) out->mass[i] = h[i];
    out->nonfinite = (int64_t)h[3];
    if (out->nonfinite > 0) return err3(TLB_EUNSTABLE, "%lld fluid nodes with non-finite order parameters", (long long)out->nonfinite);
    return tlb::clear_error();
}

void tlb3_destroy(tlb3_lattice* L)
{
    if (!L) return;
    cudaSetDevice(L->device);
    cudaStreamSynchronize(L->stream);
    for (auto e : L->ev) cudaEventDestroy(e);
    delete L;
}

}  // extern "C"

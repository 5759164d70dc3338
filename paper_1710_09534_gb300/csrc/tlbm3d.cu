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
#include <vector>

#include "tlbm.h"
#include "tlbm_internal.h"

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

// Derived constants (host-computed from tlb_params).
struct Prm3 {
    double lam[3], lamT, two_lamT, k12D, k34Dlam[2], k4D;
    double eta[2], tau[2];
    double rho[3], nu[3], M[2];
    double l3_l1, l3_l2;
    double cos12, cos13, cos23;
    double gx, gy;
};

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

// Eq. 8 for i = 1, 2 from c_1, c_2 and their Laplacians.
__device__ __forceinline__ void chem_pot(const Prm3& P, double c1, double c2, double lap1, double lap2, double& mu1,
                                         double& mu2)
{
    const double c3 = 1.0 - c1 - c2;
    const double t = P.two_lamT * c1 * c2 * c3;
    mu1 = P.k12D * (P.lam[0] * c1 * (1.0 - c1) * (1.0 - 2.0 * c1) - t) - P.k34Dlam[0] * lap1;
    mu2 = P.k12D * (P.lam[1] * c2 * (1.0 - c2) * (1.0 - 2.0 * c2) - t) - P.k34Dlam[1] * lap2;
}

// ---- kernels --------------------------------------------------------------

// Node (x, y, z) of a launch over the whole lattice: grid (ceil(nx/128), ny, nz).
#define NODE_OF_THREAD                                           \
    const int x = blockIdx.x * blockDim.x + threadIdx.x;         \
    const int y = blockIdx.y, z = blockIdx.z;                    \
    if (x >= g.nx) return;                                       \
    const long long o = node_off(g, x, y, z);

// c_1, c_2 of every node (Eq. 13a); zero on solids.
__global__ void k3_csum(const double* __restrict__ f, double* __restrict__ cpl, const uint8_t* __restrict__ kind,
                        Geo3 g)
{
    NODE_OF_THREAD
    const long long PL = g.plane;
    double a = 0.0, b = 0.0;
    if (kind[o] == K_FLUID) {
#pragma unroll
        for (int k = 0; k < Q; k++) {
            a += f[k * PL + o];
            b += f[(Q + k) * PL + o];
        }
    }
    cpl[o] = a;
    cpl[PL + o] = b;
}

// mu_1, mu_2 of every fluid node (Eq. 8, Eq. 20b with the Eq. 42 ghosts).
__global__ void k3_mu(const double* __restrict__ cpl, double* __restrict__ mpl, const uint8_t* __restrict__ kind,
                      Geo3 g, Prm3 P)
{
    NODE_OF_THREAD
    const long long PL = g.plane;
    double mu1 = 0.0, mu2 = 0.0;
    if (kind[o] == K_FLUID) {
        const double c1 = cpl[o], c2 = cpl[PL + o];
        const double c3 = 1.0 - c1 - c2;
        // Eq. 42 with the wall value of c taken as the node's own (dx = 1)
        const double o1 = P.k4D * (P.cos13 * c1 * c3 + P.cos12 * c1 * c2);
        const double o2 = P.k4D * (-P.cos12 * c1 * c2 + P.cos23 * c2 * c3);
        double l1 = 0.0, l2 = 0.0;
#pragma unroll
        for (int k = 1; k < Q; k++) {
            long long nb = 0;
            const int s = site(g, kind, x + ex(k), y + ey(k), z + ez(k), nb);
            double v1, v2;
            if (s == K_FLUID) {
                v1 = cpl[nb];
                v2 = cpl[PL + nb];
            } else if (s == K_WET) {
                v1 = c1 + o1;
                v2 = c2 + o2;
            } else {
                v1 = c1;
                v2 = c2;
            }
            // 2 w_k / cs^2 = 6 w_k
            l1 += 6.0 * wk(k) * (v1 - c1);
            l2 += 6.0 * wk(k) * (v2 - c2);
        }
        chem_pot(P, c1, c2, l1, l2, mu1, mu2);
    }
    mpl[o] = mu1;
    mpl[PL + o] = mu2;
}

// Macroscopic state of a fluid node: c, mu (from the planes), rho (Eq. 14),
// the Eq. 20 gradients with the Eq. 43 symmetric ghosts, F_s + G, u and p
// (Eqs. 13b, 13c), the F_a factor of Eq. 12 and 1/tau_g (Eqs. 15, 18b).
struct Mac3 {
    double c1, c2, rho, mu1, mu2;
    double u[3], usq, p;
    double gr[3], Ft[3];
    double a, itg;
};

__device__ __forceinline__ void macros(const Geo3& g, const uint8_t* __restrict__ kind, const double* __restrict__ f,
                                       const double* __restrict__ cpl, const double* __restrict__ mpl,
                                       const Prm3& P, int x, int y, int z, long long o, Mac3& m)
{
    const long long PL = g.plane;
    m.c1 = cpl[o];
    m.c2 = cpl[PL + o];
    m.mu1 = mpl[o];
    m.mu2 = mpl[PL + o];
    m.rho = m.c1 * P.rho[0] + m.c2 * P.rho[1] + (1.0 - m.c1 - m.c2) * P.rho[2];
    double g1[3] = {0, 0, 0}, g2[3] = {0, 0, 0}, lm1 = 0.0, lm2 = 0.0;
#pragma unroll
    for (int k = 1; k < Q; k++) {
        long long nb = 0;
        const int s = site(g, kind, x + ex(k), y + ey(k), z + ez(k), nb);
        double v1 = m.c1, v2 = m.c2, w1 = m.mu1, w2 = m.mu2;  // Eq. 43: a solid neighbour takes the centre's value
        if (s == K_FLUID) {
            v1 = cpl[nb];
            v2 = cpl[PL + nb];
            w1 = mpl[nb];
            w2 = mpl[PL + nb];
        }
        const double w3 = 3.0 * wk(k);  // w_k / cs^2
        const int e[3] = {ex(k), ey(k), ez(k)};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (e[a] != 0) {
                g1[a] += e[a] * w3 * v1;
                g2[a] += e[a] * w3 * v2;
            }
        }
        lm1 += 2.0 * w3 * (w1 - m.mu1);
        lm2 += 2.0 * w3 * (w2 - m.mu2);
    }
    // mu_3 from sum_i mu_i / lambda_i = 0; F_s = sum_i mu_i grad c_i with grad c3 = -grad c1 - grad c2
    const double mu3 = -(P.l3_l1 * m.mu1 + P.l3_l2 * m.mu2);
    const double G[3] = {m.rho * P.gx, m.rho * P.gy, 0.0};
    double mom[3] = {0, 0, 0}, sum = 0.0;
    const double* gq = f + 2 * Q * PL;
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const double gk = gq[k * PL + o];
        if (ex(k)) mom[0] += ex(k) * gk;
        if (ey(k)) mom[1] += ey(k) * gk;
        if (ez(k)) mom[2] += ez(k) * gk;
        if (k) sum += gk;
    }
    double ug = 0.0;
    m.usq = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        m.gr[a] = (P.rho[0] - P.rho[2]) * g1[a] + (P.rho[1] - P.rho[2]) * g2[a];
        m.Ft[a] = m.mu1 * g1[a] + m.mu2 * g2[a] - mu3 * (g1[a] + g2[a]) + G[a];
        m.u[a] = (mom[a] + 0.5 * m.Ft[a]) / m.rho;
        ug += m.u[a] * m.gr[a];
        m.usq += m.u[a] * m.u[a];
    }
    // Eq. 13c: p = cs^2 / (1 - w_0) [sum_{k != 0} g_k + u.grad rho / 2 + rho s_0(u)], cs^2 / (1 - w_0) = 1/2
    m.p = 0.5 * (sum + 0.5 * ug + m.rho * (wk(0) * (-1.5 * m.usq)));
    m.a = (P.rho[0] - P.rho[2]) * P.M[0] * lm1 + (P.rho[1] - P.rho[2]) * P.M[1] * lm2;
    const double nu = m.c1 * P.nu[0] + m.c2 * P.nu[1] + (1.0 - m.c1 - m.c2) * P.nu[2];
    m.itg = 1.0 / (3.0 * nu + 0.5);
}

// One BGK time step of every fluid node: collision (Eqs. 1a, 1b, 2a, 2b, 4,
// 11a, 11b, 19) and the push to x + e_k, or back into slot k-bar of the node
// itself on a link into a solid (Eq. 44).
__global__ void __launch_bounds__(128)
k3_update(const double* __restrict__ fA, double* __restrict__ fB, double* __restrict__ cu,
          const double* __restrict__ cpl, const double* __restrict__ mpl, const uint8_t* __restrict__ kind, Geo3 g,
          Prm3 P)
{
    NODE_OF_THREAD
    if (kind[o] != K_FLUID) return;
    const long long PL = g.plane;
    Mac3 m;
    macros(g, kind, fA, cpl, mpl, P, x, y, z, o, m);
    const double c[2] = {m.c1, m.c2};
    const double mu[2] = {m.mu1, m.mu2};
    double dcu[2][3];
#pragma unroll
    for (int q = 0; q < 2; q++) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double cua = c[q] * m.u[a];
            dcu[q][a] = cua - cu[(3 * q + a) * PL + o];
            cu[(3 * q + a) * PL + o] = cua;
        }
    }
    const double Fa[3] = {m.u[0] * m.a, m.u[1] * m.a, m.u[2] * m.a};
    const double kg = 1.0 - 0.5 * m.itg;
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const double w = wk(k);
        const int e[3] = {ex(k), ey(k), ez(k)};
        const double eu = e[0] * m.u[0] + e[1] * m.u[1] + e[2] * m.u[2];
        const double s = w * (3.0 * eu + 4.5 * eu * eu - 1.5 * m.usq);  // Eq. 4
        double o1, o2, og;
        {
            double post[2];
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const double em = P.eta[q] * mu[q];
                const double feq = k == 0 ? c[q] + (w - 1.0) * em : w * (em + 3.0 * c[q] * eu);  // Eq. 2a
                const double ed = e[0] * dcu[q][0] + e[1] * dcu[q][1] + e[2] * dcu[q][2];
                const double src = (1.0 - 0.5 / P.tau[q]) * 3.0 * w * ed;                            // Eq. 11a
                const double fk = fA[(Q * q + k) * PL + o];
                post[q] = fk - (fk - feq) / P.tau[q] + src;                                          // Eq. 1a
            }
            o1 = post[0];
            o2 = post[1];
        }
        {
            const double geq = k == 0 ? 3.0 * m.p * (w - 1.0) + m.rho * s : 3.0 * m.p * w + m.rho * s;  // Eq. 2b
            double br = 0.0, efa = 0.0;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                br += (e[a] - m.u[a]) * (s * m.gr[a] + 3.0 * (s + w) * m.Ft[a]);
                efa += e[a] * Fa[a];
            }
            const double src = kg * br + 3.0 * w * efa;  // Eq. 11b
            const double gk = fA[(2 * Q + k) * PL + o];
            og = gk - (gk - geq) * m.itg + src;          // Eq. 1b
        }
        long long d = o;
        int slot = k;
        if (k != 0) {
            long long nb = 0;
            if (site(g, kind, x + e[0], y + e[1], z + e[2], nb) == K_FLUID) d = nb;
            else slot = opp(k);
        }
        fB[slot * PL + d] = o1;
        fB[(Q + slot) * PL + d] = o2;
        fB[(2 * Q + slot) * PL + d] = og;
    }
}

// c of every node from dense host-order arrays (c1 then c2, nx*ny*nz each).
__global__ void k3_load_c(const double* __restrict__ in, double* __restrict__ cpl, const uint8_t* __restrict__ kind,
                          Geo3 g)
{
    NODE_OF_THREAD
    const long long n = ((long long)z * g.ny + y) * g.nx + x, N = (long long)g.nx * g.ny * g.nz;
    const bool fl = kind[o] == K_FLUID;
    cpl[o] = fl ? in[n] : 0.0;
    cpl[g.plane + o] = fl ? in[N + n] : 0.0;
}

// Initial state from c, mu (planes) and u, p (dense arrays ux, uy, uz[, p]):
// f = f^eq(c, mu, u), g = g^eq(p, rho, u), c_i u stored (Eq. 19).
__global__ void k3_init(double* __restrict__ f, double* __restrict__ cu, const double* __restrict__ cpl,
                        const double* __restrict__ mpl, const uint8_t* __restrict__ kind,
                        const double* __restrict__ in, int has_p, Geo3 g, Prm3 P)
{
    NODE_OF_THREAD
    const long long PL = g.plane;
    const long long n = ((long long)z * g.ny + y) * g.nx + x, N = (long long)g.nx * g.ny * g.nz;
    if (kind[o] != K_FLUID) {
        for (int q = 0; q < NPLANES; q++) f[q * PL + o] = 0.0;
        for (int q = 0; q < 6; q++) cu[q * PL + o] = 0.0;
        return;
    }
    const double c[2] = {cpl[o], cpl[PL + o]}, mu[2] = {mpl[o], mpl[PL + o]};
    const double u[3] = {in[n], in[N + n], in[2 * N + n]};
    const double p = has_p ? in[3 * N + n] : 0.0;
    const double rho = c[0] * P.rho[0] + c[1] * P.rho[1] + (1.0 - c[0] - c[1]) * P.rho[2];
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int k = 0; k < Q; k++) {
        const double w = wk(k);
        const double eu = ex(k) * u[0] + ey(k) * u[1] + ez(k) * u[2];
        const double s = w * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
        for (int q = 0; q < 2; q++) {
            const double em = P.eta[q] * mu[q];
            f[(Q * q + k) * PL + o] = k == 0 ? c[q] + (w - 1.0) * em : w * (em + 3.0 * c[q] * eu);
        }
        f[(2 * Q + k) * PL + o] = k == 0 ? 3.0 * p * (w - 1.0) + rho * s : 3.0 * p * w + rho * s;
    }
    for (int q = 0; q < 2; q++)
        for (int a = 0; a < 3; a++) cu[(3 * q + a) * PL + o] = c[q] * u[a];
}

// The 11 macroscopic fields c1 c2 c3 rho ux uy uz p mu1 mu2 mu3 as dense
// planes of nx*ny*nz (zero on solids).
__global__ void k3_read(const double* __restrict__ f, const double* __restrict__ cpl, const double* __restrict__ mpl,
                        const uint8_t* __restrict__ kind, double* __restrict__ out, Geo3 g, Prm3 P)
{
    NODE_OF_THREAD
    const long long n = ((long long)z * g.ny + y) * g.nx + x, N = (long long)g.nx * g.ny * g.nz;
    double v[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (kind[o] == K_FLUID) {
        Mac3 m;
        macros(g, kind, f, cpl, mpl, P, x, y, z, o, m);
        v[0] = m.c1;
        v[1] = m.c2;
        v[2] = 1.0 - m.c1 - m.c2;
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
// the non-finite count over fluid nodes (from the c planes), then one block.
__global__ void __launch_bounds__(256) k3_mass_partials(const double* __restrict__ cpl,
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
        const double c1 = cpl[o], c2 = cpl[g.plane + o];
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
    int64_t fA = 0, fB = 0, cu = 0, cpl = 0, mpl = 0, kind = 0, part = 0, diag = 0, total = 0;
};

bool size_ok(int nx, int ny, int nz) { return nx >= 3 && ny >= 3 && nz >= 3 && nx <= 65536 && ny <= 65535 && nz <= 65535; }

Layout3 layout3(int nx, int ny, int nz)
{
    Layout3 L;
    L.pitch = (int)align3(nx, 32);
    L.plane = (int64_t)L.pitch * ny * nz;
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        const int64_t at = off;
        off = align3(off + bytes, kAlign3);
        return at;
    };
    L.fA = take(tlb3::NPLANES * L.plane * 8);
    L.fB = take(tlb3::NPLANES * L.plane * 8);
    L.cu = take(6 * L.plane * 8);
    L.cpl = take(2 * L.plane * 8);
    L.mpl = take(2 * L.plane * 8);
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
    tlb3::Prm3 prm{};
    int cur = 0;
    bool have_params = false, have_fields = false;
    std::vector<uint8_t> mask;

    double* buf(int which) { return (double*)(ws + (which == 0 ? lay.fA : lay.fB)); }
    double* fcur() { return buf(cur); }
    double* fspare() { return buf(cur ^ 1); }
    double* cu() { return (double*)(ws + lay.cu); }
    double* cpl() { return (double*)(ws + lay.cpl); }
    double* mpl() { return (double*)(ws + lay.mpl); }
    uint8_t* kind() { return (uint8_t*)(ws + lay.kind); }
    int64_t n() const { return (int64_t)nx * ny * nz; }
};

namespace {

int check3(tlb3_lattice* L)
{
    if (!L) return err3(TLB_EINVAL, "null lattice handle");
    T3_CUDA(cudaSetDevice(L->device));
    return TLB_OK;
}

dim3 grid3(const tlb3_lattice* L) { return dim3((unsigned)((L->nx + 127) / 128), (unsigned)L->ny, (unsigned)L->nz); }

// c and mu planes of the current state (the first two launches of a step)
int order_params3(tlb3_lattice* L)
{
    tlb3::k3_csum<<<grid3(L), 128, 0, L->stream>>>(L->fcur(), L->cpl(), L->kind(), L->geo);
    tlb3::k3_mu<<<grid3(L), 128, 0, L->stream>>>(L->cpl(), L->mpl(), L->kind(), L->geo, L->prm);
    T3_CUDA(cudaGetLastError());
    return TLB_OK;
}

}  // namespace

extern "C" {

int64_t tlb3_workspace_bytes(int nx, int ny, int nz)
{
    if (!size_ok(nx, ny, nz)) return err3(TLB_EINVAL, "lattice size %dx%dx%d out of range", nx, ny, nz);
    tlb::clear_error();
    return layout3(nx, ny, nz).total;
}

int tlb3_create(int nx, int ny, int nz, const int32_t edges[6], void* dev_workspace, int64_t ws_bytes,
                void* cuda_stream, tlb3_lattice** out)
{
    if (!out) return err3(TLB_EINVAL, "out is null");
    *out = nullptr;
    if (!size_ok(nx, ny, nz)) return err3(TLB_EINVAL, "lattice size %dx%dx%d out of range", nx, ny, nz);
    if (!edges) return err3(TLB_EINVAL, "edges is null");
    for (int a = 0; a < 3; a++) {
        const int lo = edges[2 * a], hi = edges[2 * a + 1];
        if (lo < 0 || lo > 2 || hi < 0 || hi > 2)
            return err3(TLB_EINVAL, "edge kinds must be periodic, wetting or neutral (no lid in 3D)");
        if ((lo == 0) != (hi == 0)) return err3(TLB_EINVAL, "a periodic edge needs a periodic opposite edge");
    }
    const Layout3 lay = layout3(nx, ny, nz);
    if (!dev_workspace || ((uintptr_t)dev_workspace) % kAlign3) return err3(TLB_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < lay.total)
        return err3(TLB_ENOMEM, "workspace has %lld bytes, needs %lld", (long long)ws_bytes, (long long)lay.total);
    auto* L = new tlb3_lattice;
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
    if (cudaMemsetAsync(L->ws + lay.kind, 0, (size_t)lay.plane, L->stream) != cudaSuccess ||
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
    tlb3::Prm3& P = L->prm;
    P.lam[0] = l1;
    P.lam[1] = l2;
    P.lam[2] = l3;
    P.lamT = den != 0 ? 3.0 * l1 * l2 * l3 / den : 0.0;  // Eq. 9, continuous form
    P.two_lamT = 2.0 * P.lamT;
    P.k12D = 12.0 / p->D;
    P.k4D = 4.0 / p->D;
    const double tau[2] = {p->tau1, p->tau2};
    for (int i = 0; i < 2; i++) {
        P.k34Dlam[i] = 0.75 * p->D * P.lam[i];
        P.M[i] = p->M0 / P.lam[i];                       // Eq. 12
        P.eta[i] = P.M[i] / ((1.0 / 3.0) * (tau[i] - 0.5));  // Eq. 18a, per component
        P.tau[i] = tau[i];
    }
    P.rho[0] = p->rho1;
    P.rho[1] = p->rho2;
    P.rho[2] = p->rho3;
    P.nu[0] = p->nu1;
    P.nu[1] = p->nu2;
    P.nu[2] = p->nu3;
    P.l3_l1 = l3 / l1;
    P.l3_l2 = l3 / l2;
    P.cos12 = c12;
    P.cos13 = c13;
    P.cos23 = c23;
    P.gx = p->gx;
    P.gy = p->gy;
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
    double* stage = L->fspare();  // 57 planes of >= N doubles
    T3_CUDA(cudaMemcpyAsync(stage, c1, bytes, cudaMemcpyHostToDevice, L->stream));
    T3_CUDA(cudaMemcpyAsync(stage + N, c2, bytes, cudaMemcpyHostToDevice, L->stream));
    tlb3::k3_load_c<<<grid3(L), 128, 0, L->stream>>>(stage, L->cpl(), L->kind(), L->geo);
    tlb3::k3_mu<<<grid3(L), 128, 0, L->stream>>>(L->cpl(), L->mpl(), L->kind(), L->geo, L->prm);
    T3_CUDA(cudaGetLastError());
    // u, p after the c staging has been consumed (same stream)
    double* in = stage + 2 * N;
    T3_CUDA(cudaMemcpyAsync(in, ux, bytes, cudaMemcpyHostToDevice, L->stream));
    T3_CUDA(cudaMemcpyAsync(in + N, uy, bytes, cudaMemcpyHostToDevice, L->stream));
    T3_CUDA(cudaMemcpyAsync(in + 2 * N, uz, bytes, cudaMemcpyHostToDevice, L->stream));
    if (p) T3_CUDA(cudaMemcpyAsync(in + 3 * N, p, bytes, cudaMemcpyHostToDevice, L->stream));
    tlb3::k3_init<<<grid3(L), 128, 0, L->stream>>>(L->fcur(), L->cu(), L->cpl(), L->mpl(), L->kind(), in, p ? 1 : 0,
                                                   L->geo, L->prm);
    T3_CUDA(cudaGetLastError());
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
        if ((rc = order_params3(L))) return rc;
        tlb3::k3_update<<<grid3(L), 128, 0, L->stream>>>(L->fcur(), L->fspare(), L->cu(), L->cpl(), L->mpl(), L->kind(),
                                                         L->geo, L->prm);
        T3_CUDA(cudaGetLastError());
        L->cur ^= 1;
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
    double* stage = L->fspare();
    tlb3::k3_read<<<grid3(L), 128, 0, L->stream>>>(L->fcur(), L->cpl(), L->mpl(), L->kind(), stage, L->geo, L->prm);
    T3_CUDA(cudaGetLastError());
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
    for (int q = 0; q < 63; q++) {
        const double* src = q < 57 ? L->fcur() + q * PL : L->cu() + (q - 57) * PL;
        T3_CUDA(cudaMemcpy2DAsync(host_out + q * N, (size_t)L->nx * sizeof(double), src,
                                  (size_t)L->lay.pitch * sizeof(double), (size_t)L->nx * sizeof(double), rows,
                                  cudaMemcpyDeviceToHost, L->stream));
    }
    T3_CUDA(cudaStreamSynchronize(L->stream));
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
    tlb3::k3_csum<<<grid3(L), 128, 0, L->stream>>>(L->fcur(), L->cpl(), L->kind(), L->geo);
    double* part = (double*)(L->ws + L->lay.part);
    double* diag = (double*)(L->ws + L->lay.diag);
    tlb3::k3_mass_partials<<<kMassParts3, 256, 0, L->stream>>>(L->cpl(), L->kind(), part, L->geo);
    tlb3::k3_mass_final<<<1, 256, 0, L->stream>>>(part, kMassParts3, diag);
    T3_CUDA(cudaGetLastError());
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
    delete L;
}

}  // extern "C"

/*
 * Plain FP64 CPU oracle of the same per-time-step update on the D3Q19
 * lattice.  Sec. II.A of Liang, Li, Shi and Chai (arXiv:1710.09534) states the
 * model for D dimensions: Eqs. 1-20 hold with the D3Q19 velocity set and
 * weights, the isotropic stencils of Eq. 20 summed over its 18 links, and the
 * wetting condition of Eq. 42 applied on every link into a solid.
 *
 * TEST INFRASTRUCTURE ONLY, like tlb_oracle.c: only the test suite and the
 * benchmark's CPU-baseline leg load it; the CUDA library shares no source
 * with it.  Whole-field arrays, one pass per stage, each equation written out,
 * compiled with -ffp-contract=off.
 *
 * Readings (in addition to R1-R4 of tlb_oracle.c, which carry over):
 *   R3D1 D3Q19: e_0 = 0; e_1..6 = +-x, +-y, +-z; e_7..18 the 12 face
 *        diagonals; weights 1/3, 1/18, 1/36; cs^2 = 1/3.  Opposite links are
 *        adjacent (k odd <-> k + 1).
 *   R3D2 Edges x-, x+, y-, y+, z-, z+, each periodic, wetting or neutral (no
 *        velocity lid in 3D).  At a site outside in several axes, the first
 *        outside axis in the order x, y, z that is not periodic decides.
 *   R3D3 Body force G = rho (gx, gy, 0).
 *   R3D4 BGK collision only.
 * Node arrays are [nz][ny][nx], x fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "tlb_oracle.h"

static const int E3[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
#define Q3 19
#define NPL3 57
#define CS2 (1.0 / 3.0)

static double w3(int k) { return k == 0 ? 1.0 / 3.0 : (k <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
static int opp3(int k) { return k == 0 ? 0 : (k % 2 == 1 ? k + 1 : k - 1); }

enum { P3 = 0, WET3 = 1, NEU3 = 2 };                /* edge kinds */
enum { S_FLUID = 0, S_WET = 2, S_NEUTRAL = 3 };     /* site kinds */

typedef struct {
    int nx, ny, nz;
    int edge[6];
    unsigned char *mask; /* 0 fluid, 1 wetting solid, 2 neutral solid */
    orc_params P;
    double lam[3], lamT, M[2], eta[2], cos12, cos13, cos23;
    double *f, *fn, *cu; /* 57 distribution planes; 6 planes c_i u_a (Eq. 19) */
    double *c1, *c2, *rho, *mu1, *mu2, *mu3;
    double *gc1[3], *gc2[3], *gr[3], *lm1, *lm2, *u[3], *p;
    unsigned char *kind, *nbk;
    long *nbi;
    int have_params;
} orc3_lattice;

/* ---- lattice constants and stencils, exported for the tests ------------- */

int orc3_e(int k, int a) { return E3[k][a]; }
double orc3_w(int k) { return w3(k); }
int orc3_opp(int k) { return opp3(k); }

/* Eq. 20a on D3Q19: v[k] = chi(x + e_k). */
void orc3_grad(const double v[19], double g[3])
{
    for (int a = 0; a < 3; a++) {
        g[a] = 0.0;
        for (int k = 1; k < Q3; k++)
            g[a] += w3(k) * E3[k][a] * v[k] / CS2;
    }
}

/* Eq. 20b on D3Q19. */
double orc3_lap(const double v[19])
{
    double s = 0.0;
    for (int k = 1; k < Q3; k++)
        s += 2.0 * w3(k) * (v[k] - v[0]) / CS2;
    return s;
}

/* Eq. 4. */
static double sk3(int k, const double u[3])
{
    double eu = E3[k][0] * u[0] + E3[k][1] * u[1] + E3[k][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return w3(k) * (eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. 2a. */
static double feq3(int k, double c, double mu, double eta, const double u[3])
{
    if (k == 0)
        return c + (w3(0) - 1.0) * eta * mu;
    double eu = E3[k][0] * u[0] + E3[k][1] * u[1] + E3[k][2] * u[2];
    return w3(k) * eta * mu + w3(k) * c * eu / CS2;
}

/* Eq. 2b. */
static double geq3(int k, double p, double rho, const double u[3])
{
    double s = sk3(k, u);
    if (k == 0)
        return p / CS2 * (w3(0) - 1.0) + rho * s;
    return p / CS2 * w3(k) + rho * s;
}

/* Eq. 11a. */
static double srcf3(int k, double tau, const double dcu[3])
{
    double ed = E3[k][0] * dcu[0] + E3[k][1] * dcu[1] + E3[k][2] * dcu[2];
    return (1.0 - 1.0 / (2.0 * tau)) * w3(k) * ed / CS2;
}

/* Eq. 11b with Ft = F_s + G and the interfacial force Fa. */
static double srcg3(int k, double taug, const double u[3], const double gr[3], const double Ft[3],
                    const double Fa[3])
{
    double s = sk3(k, u);
    double sum = 0.0, efa = 0.0;
    for (int a = 0; a < 3; a++) {
        double b = s * gr[a] + (s + w3(k)) * Ft[a] / CS2;
        sum += (E3[k][a] - u[a]) * b;
        efa += E3[k][a] * Fa[a];
    }
    return (1.0 - 1.0 / (2.0 * taug)) * sum + w3(k) * efa / CS2;
}

double orc3_feq(int k, double c, double mu, double eta, double ux, double uy, double uz)
{
    double u[3] = {ux, uy, uz};
    return feq3(k, c, mu, eta, u);
}

double orc3_geq(int k, double p, double rho, double ux, double uy, double uz)
{
    double u[3] = {ux, uy, uz};
    return geq3(k, p, rho, u);
}

/* ---- lattice ------------------------------------------------------------- */

static double *dz(size_t n) { return (double *)calloc(n, sizeof(double)); }

orc3_lattice *orc3_create(int nx, int ny, int nz, const int edge[6])
{
    if (nx < 3 || ny < 3 || nz < 3)
        return NULL;
    orc3_lattice *L = (orc3_lattice *)calloc(1, sizeof(orc3_lattice));
    size_t n = (size_t)nx * ny * nz;
    L->nx = nx;
    L->ny = ny;
    L->nz = nz;
    for (int e = 0; e < 6; e++)
        L->edge[e] = edge[e];
    L->mask = (unsigned char *)calloc(n, 1);
    L->kind = (unsigned char *)calloc(n, 1);
    L->nbk = (unsigned char *)calloc((size_t)Q3 * n, 1);
    L->nbi = (long *)calloc((size_t)Q3 * n, sizeof(long));
    L->f = dz(NPL3 * n);
    L->fn = dz(NPL3 * n);
    L->cu = dz(6 * n);
    L->c1 = dz(n);
    L->c2 = dz(n);
    L->rho = dz(n);
    L->mu1 = dz(n);
    L->mu2 = dz(n);
    L->mu3 = dz(n);
    L->lm1 = dz(n);
    L->lm2 = dz(n);
    L->p = dz(n);
    for (int a = 0; a < 3; a++) {
        L->gc1[a] = dz(n);
        L->gc2[a] = dz(n);
        L->gr[a] = dz(n);
        L->u[a] = dz(n);
    }
    return L;
}

void orc3_destroy(orc3_lattice *L)
{
    if (!L)
        return;
    free(L->mask);
    free(L->kind);
    free(L->nbk);
    free(L->nbi);
    free(L->f);
    free(L->fn);
    free(L->cu);
    double *fl[] = {L->c1, L->c2, L->rho, L->mu1, L->mu2, L->mu3, L->lm1, L->lm2, L->p};
    for (size_t i = 0; i < sizeof fl / sizeof fl[0]; i++)
        free(fl[i]);
    for (int a = 0; a < 3; a++) {
        free(L->gc1[a]);
        free(L->gc2[a]);
        free(L->gr[a]);
        free(L->u[a]);
    }
    free(L);
}

/* Derived constants: Eqs. 7, 9 (R2), 12, 18a (R1), 38. */
void orc3_set_params(orc3_lattice *L, const orc_params *P)
{
    const double deg = 3.14159265358979323846 / 180.0;
    L->P = *P;
    double lam[4];
    orc_lambdas(P->sigma12, P->sigma13, P->sigma23, lam);
    for (int i = 0; i < 3; i++)
        L->lam[i] = lam[i];
    L->lamT = lam[3];
    double tau[2] = {P->tau1, P->tau2};
    for (int i = 0; i < 2; i++) {
        L->M[i] = P->M0 / lam[i];
        L->eta[i] = L->M[i] / (CS2 * (tau[i] - 0.5));
    }
    L->cos12 = cos(P->theta12_deg * deg);
    L->cos13 = cos(P->theta13_deg * deg);
    L->cos23 = cos(P->theta23_deg * deg);
    L->have_params = 1;
}

/* Kind of site (x, y, z), possibly outside the lattice (R3D2); *idx is the
 * wrapped index of an inside site. */
static int site3(const orc3_lattice *L, int x, int y, int z, long *idx)
{
    int c[3] = {x, y, z}, n[3] = {L->nx, L->ny, L->nz};
    for (int a = 0; a < 3; a++) {
        if (c[a] < 0 || c[a] >= n[a]) {
            int e = L->edge[2 * a + (c[a] < 0 ? 0 : 1)];
            if (e != P3)
                return e == WET3 ? S_WET : S_NEUTRAL;
            c[a] = (c[a] + n[a]) % n[a];
        }
    }
    *idx = ((long)c[2] * n[1] + c[1]) * n[0] + c[0];
    if (L->mask[*idx] == 1)
        return S_WET;
    if (L->mask[*idx] == 2)
        return S_NEUTRAL;
    return S_FLUID;
}

void orc3_set_geometry(orc3_lattice *L, const unsigned char *mask)
{
    long n = (long)L->nx * L->ny * L->nz;
    memcpy(L->mask, mask, (size_t)n);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        int x = (int)(i % L->nx), y = (int)((i / L->nx) % L->ny), z = (int)(i / ((long)L->nx * L->ny));
        long j = i;
        L->kind[i] = (unsigned char)site3(L, x, y, z, &j);
        for (int k = 0; k < Q3; k++) {
            j = -1;
            L->nbk[(long)k * n + i] = (unsigned char)site3(L, x + E3[k][0], y + E3[k][1], z + E3[k][2], &j);
            L->nbi[(long)k * n + i] = j;
        }
    }
}

static int nbr3(const orc3_lattice *L, int k, long i, long *j)
{
    long n = (long)L->nx * L->ny * L->nz;
    *j = L->nbi[(long)k * n + i];
    return L->nbk[(long)k * n + i];
}

/* Stage 1 (Eqs. 13a, 3, 14). */
static void stage3_order_parameters(orc3_lattice *L, const double *f)
{
    long n = (long)L->nx * L->ny * L->nz;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        L->c1[i] = L->c2[i] = L->rho[i] = 0.0;
        if (L->kind[i] != S_FLUID)
            continue;
        double a = 0.0, b = 0.0;
        for (int k = 0; k < Q3; k++) {
            a += f[(long)k * n + i];
            b += f[(long)(Q3 + k) * n + i];
        }
        L->c1[i] = a;
        L->c2[i] = b;
        L->rho[i] = a * L->P.rho1 + b * L->P.rho2 + (1.0 - a - b) * L->P.rho3;
    }
}

/* Stage 2 (Eqs. 8, 20b, 42): chemical potentials with wetting ghosts. */
static void stage3_chemical_potentials(orc3_lattice *L)
{
    long n = (long)L->nx * L->ny * L->nz;
    double lam4[4] = {L->lam[0], L->lam[1], L->lam[2], L->lamT};
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        L->mu1[i] = L->mu2[i] = L->mu3[i] = 0.0;
        if (L->kind[i] != S_FLUID)
            continue;
        double v1[Q3], v2[Q3];
        v1[0] = L->c1[i];
        v2[0] = L->c2[i];
        for (int k = 1; k < Q3; k++) {
            long nb;
            int s = nbr3(L, k, i, &nb);
            if (s == S_FLUID) {
                v1[k] = L->c1[nb];
                v2[k] = L->c2[nb];
            } else if (s == S_WET) {
                double off[3];
                orc_wet_offset(L->cos12, L->cos13, L->cos23, L->P.D, L->c1[i], L->c2[i], off);
                v1[k] = L->c1[i] + off[0];
                v2[k] = L->c2[i] + off[1];
            } else {
                v1[k] = L->c1[i];
                v2[k] = L->c2[i];
            }
        }
        double mu[3];
        orc_chem_pot(lam4, L->P.D, L->c1[i], L->c2[i], orc3_lap(v1), orc3_lap(v2), mu);
        L->mu1[i] = mu[0];
        L->mu2[i] = mu[1];
        L->mu3[i] = mu[2];
    }
}

/* Stage 3 (Eqs. 20a, 20b, 43): grad c_i, grad rho, lap mu_i, symmetric ghosts. */
static void stage3_gradients(orc3_lattice *L)
{
    long n = (long)L->nx * L->ny * L->nz;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        for (int a = 0; a < 3; a++)
            L->gc1[a][i] = L->gc2[a][i] = L->gr[a][i] = 0.0;
        L->lm1[i] = L->lm2[i] = 0.0;
        if (L->kind[i] != S_FLUID)
            continue;
        double vc1[Q3], vc2[Q3], vr[Q3], vm1[Q3], vm2[Q3];
        for (int k = 0; k < Q3; k++) {
            long nb = i;
            int s = k == 0 ? S_FLUID : nbr3(L, k, i, &nb);
            long src = s == S_FLUID ? nb : i; /* Eq. 43 */
            vc1[k] = L->c1[src];
            vc2[k] = L->c2[src];
            vr[k] = L->rho[src];
            vm1[k] = L->mu1[src];
            vm2[k] = L->mu2[src];
        }
        double g[3];
        orc3_grad(vc1, g);
        for (int a = 0; a < 3; a++)
            L->gc1[a][i] = g[a];
        orc3_grad(vc2, g);
        for (int a = 0; a < 3; a++)
            L->gc2[a][i] = g[a];
        orc3_grad(vr, g);
        for (int a = 0; a < 3; a++)
            L->gr[a][i] = g[a];
        L->lm1[i] = orc3_lap(vm1);
        L->lm2[i] = orc3_lap(vm2);
    }
}

/* F_s = sum_{i=1..3} mu_i grad c_i with grad c_3 = -grad c_1 - grad c_2. */
static void surface_force3(const orc3_lattice *L, long i, double F[3])
{
    for (int a = 0; a < 3; a++) {
        double g3 = -L->gc1[a][i] - L->gc2[a][i];
        F[a] = L->mu1[i] * L->gc1[a][i] + L->mu2[i] * L->gc2[a][i] + L->mu3[i] * g3;
    }
}

/* Stage 4 (Eqs. 13b, 13c): velocity and pressure. */
static void stage3_velocity_pressure(orc3_lattice *L, const double *f)
{
    long n = (long)L->nx * L->ny * L->nz;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        for (int a = 0; a < 3; a++)
            L->u[a][i] = 0.0;
        L->p[i] = 0.0;
        if (L->kind[i] != S_FLUID)
            continue;
        const double *g = f + 2 * Q3 * n;
        double Fs[3];
        surface_force3(L, i, Fs);
        double rho = L->rho[i];
        double G[3] = {rho * L->P.gx, rho * L->P.gy, 0.0}; /* R3D3 */
        double m[3] = {0.0, 0.0, 0.0}, sum = 0.0;
        for (int k = 0; k < Q3; k++) {
            double gk = g[(long)k * n + i];
            for (int a = 0; a < 3; a++)
                m[a] += E3[k][a] * gk;
            if (k != 0)
                sum += gk;
        }
        double u[3], ug = 0.0;
        for (int a = 0; a < 3; a++) {
            u[a] = (m[a] + 0.5 * (Fs[a] + G[a])) / rho;
            ug += u[a] * L->gr[a][i];
        }
        L->p[i] = CS2 / (1.0 - w3(0)) * (sum + 0.5 * ug + rho * sk3(0, u));
        for (int a = 0; a < 3; a++)
            L->u[a][i] = u[a];
    }
}

static void compute3_macros(orc3_lattice *L, const double *f)
{
    stage3_order_parameters(L, f);
    stage3_chemical_potentials(L);
    stage3_gradients(L);
    stage3_velocity_pressure(L, f);
}

/* One time step: stages 1-4, the forces (Eq. 12), BGK collision (Eqs. 1a,
 * 1b, 45) and streaming with half-way bounce-back (Eq. 44). */
int orc3_step(orc3_lattice *L, long nsteps)
{
    if (!L->have_params)
        return -1;
    long n = (long)L->nx * L->ny * L->nz;
    const double tau[2] = {L->P.tau1, L->P.tau2};
    for (long step = 0; step < nsteps; step++) {
        compute3_macros(L, L->f);
        memset(L->fn, 0, NPL3 * n * sizeof(double));
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; i++) {
            if (L->kind[i] != S_FLUID)
                continue;
            double c[2] = {L->c1[i], L->c2[i]};
            double mu[2] = {L->mu1[i], L->mu2[i]};
            double u[3] = {L->u[0][i], L->u[1][i], L->u[2][i]};
            double p = L->p[i], rho = L->rho[i];
            double c3 = 1.0 - c[0] - c[1];
            /* Eqs. 15, 18b */
            double nu = c[0] * L->P.nu1 + c[1] * L->P.nu2 + c3 * L->P.nu3;
            double taug = nu / CS2 + 0.5;
            double Fs[3], Ft[3], Fa[3], gr[3];
            surface_force3(L, i, Fs);
            /* Eq. 12: F_a = u sum_{i=1,2} (rho_i - rho_3) M_i lap mu_i */
            double af = (L->P.rho1 - L->P.rho3) * L->M[0] * L->lm1[i] +
                        (L->P.rho2 - L->P.rho3) * L->M[1] * L->lm2[i];
            double G[3] = {rho * L->P.gx, rho * L->P.gy, 0.0};
            for (int a = 0; a < 3; a++) {
                Ft[a] = Fs[a] + G[a];
                Fa[a] = u[a] * af;
                gr[a] = L->gr[a][i];
            }
            /* Eq. 19 */
            double dcu[2][3];
            for (int q = 0; q < 2; q++)
                for (int a = 0; a < 3; a++)
                    dcu[q][a] = c[q] * u[a] - L->cu[(long)(3 * q + a) * n + i];
            double fpost[NPL3];
            for (int k = 0; k < Q3; k++) {
                for (int q = 0; q < 2; q++) {
                    double eq = feq3(k, c[q], mu[q], L->eta[q], u);
                    double src = srcf3(k, tau[q], dcu[q]);
                    double fk = L->f[(long)(Q3 * q + k) * n + i];
                    fpost[Q3 * q + k] = fk - (fk - eq) / tau[q] + src;
                }
                double geq = geq3(k, p, rho, u);
                double src = srcg3(k, taug, u, gr, Ft, Fa);
                double gk = L->f[(long)(2 * Q3 + k) * n + i];
                fpost[2 * Q3 + k] = gk - (gk - geq) / taug + src;
            }
            /* Streaming and half-way bounce-back (Eq. 44). */
            for (int k = 0; k < Q3; k++) {
                long dst = i;
                int sd = k == 0 ? S_FLUID : nbr3(L, k, i, &dst);
                for (int q = 0; q < 3; q++) {
                    double v = fpost[Q3 * q + k];
                    if (sd == S_FLUID)
                        L->fn[(long)(Q3 * q + k) * n + dst] = v;
                    else
                        L->fn[(long)(Q3 * q + opp3(k)) * n + i] = v;
                }
            }
            for (int q = 0; q < 2; q++)
                for (int a = 0; a < 3; a++)
                    L->cu[(long)(3 * q + a) * n + i] = c[q] * u[a];
        }
        double *t = L->f;
        L->f = L->fn;
        L->fn = t;
    }
    return 0;
}

/* Initial state (reading 9 of tlb_oracle.c in 3D): f = f^eq(c, mu(c), u),
 * g = g^eq(p, rho(c), u), c_i u stored.  Node arrays of nx*ny*nz; p may be
 * NULL (zero). */
int orc3_set_fields(orc3_lattice *L, const double *c1, const double *c2, const double *ux, const double *uy,
                    const double *uz, const double *p)
{
    if (!L->have_params)
        return -1;
    long n = (long)L->nx * L->ny * L->nz;
    memset(L->fn, 0, NPL3 * n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        L->fn[i] = c1[i];
        L->fn[Q3 * n + i] = c2[i];
    }
    stage3_order_parameters(L, L->fn);
    stage3_chemical_potentials(L);
    memset(L->f, 0, NPL3 * n * sizeof(double));
    memset(L->fn, 0, NPL3 * n * sizeof(double));
    memset(L->cu, 0, 6 * n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        if (L->kind[i] != S_FLUID)
            continue;
        double c[2] = {L->c1[i], L->c2[i]};
        double mu[2] = {L->mu1[i], L->mu2[i]};
        double u[3] = {ux[i], uy[i], uz[i]};
        double pi = p ? p[i] : 0.0;
        for (int k = 0; k < Q3; k++) {
            for (int q = 0; q < 2; q++)
                L->f[(long)(Q3 * q + k) * n + i] = feq3(k, c[q], mu[q], L->eta[q], u);
            L->f[(long)(2 * Q3 + k) * n + i] = geq3(k, pi, L->rho[i], u);
        }
        for (int q = 0; q < 2; q++)
            for (int a = 0; a < 3; a++)
                L->cu[(long)(3 * q + a) * n + i] = c[q] * u[a];
    }
    return 0;
}

/* Macroscopic fields, 11 planes: c1, c2, c3, rho, ux, uy, uz, p, mu1, mu2,
 * mu3 (zero at solid nodes). */
int orc3_read_fields(orc3_lattice *L, double *out)
{
    if (!L->have_params)
        return -1;
    long n = (long)L->nx * L->ny * L->nz;
    compute3_macros(L, L->f);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        int fl = L->kind[i] == S_FLUID;
        double v[11] = {L->c1[i], L->c2[i], 1.0 - L->c1[i] - L->c2[i], L->rho[i], L->u[0][i], L->u[1][i],
                        L->u[2][i], L->p[i], L->mu1[i], L->mu2[i], L->mu3[i]};
        for (int q = 0; q < 11; q++)
            out[(long)q * n + i] = fl ? v[q] : 0.0;
    }
    return 0;
}

/* Raw state: 57 distribution planes (f^1_k, f^2_k, g_k, k = 0..18), then the
 * 6 planes c1 ux, c1 uy, c1 uz, c2 ux, c2 uy, c2 uz. */
void orc3_get_state(const orc3_lattice *L, double *out)
{
    long n = (long)L->nx * L->ny * L->nz;
    memcpy(out, L->f, NPL3 * n * sizeof(double));
    memcpy(out + NPL3 * n, L->cu, 6 * n * sizeof(double));
}

void orc3_set_state(orc3_lattice *L, const double *in)
{
    long n = (long)L->nx * L->ny * L->nz;
    memcpy(L->f, in, NPL3 * n * sizeof(double));
    memcpy(L->cu, in + NPL3 * n, 6 * n * sizeof(double));
}

/* Per-direction formulas of the step, exported for the moment tests. */
double orc3_sk(int k, double ux, double uy, double uz)
{
    double u[3] = {ux, uy, uz};
    return sk3(k, u);
}

double orc3_src_f(int k, double tau, double dx, double dy, double dz_)
{
    double d[3] = {dx, dy, dz_};
    return srcf3(k, tau, d);
}

double orc3_src_g(int k, double taug, const double u[3], const double gr[3], const double Ft[3], const double Fa[3])
{
    return srcg3(k, taug, u, gr, Ft, Fa);
}

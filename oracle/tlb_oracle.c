/*
 * Plain FP64 CPU oracle for the per-time-step lattice update of the
 * phase-field lattice Boltzmann ternary-fluid model with the ternary wetting
 * boundary scheme of Liang, Li, Shi and Chai, "Lattice Boltzmann modeling of
 * wall-bounded ternary fluid flows" (arXiv:1710.09534).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The CUDA library
 * never calls, links or includes it, and it shares no source with it.
 *
 * The code is written for reading against the paper, not for speed: whole
 * field arrays, one pass per stage of the update, direct transcription of
 * each equation, no fusion.  Every function names the passage it follows.
 * Compiled with -ffp-contract=off so that x86 and Arm give the same bits.
 *
 * Readings of the paper where it is silent or ambiguous (each one is also
 * implemented by the CUDA path):
 *   R1  eta is per component: eta_i = M_i / (cs^2 (tau_i - 1/2)) (Eqs. 2a, 18a)
 *       with M_i = M0 / lambda_i (Eq. 12).
 *   R2  lambda_T = 3 l1 l2 l3 / (l1 l2 + l1 l3 + l2 l3), the continuous form
 *       of Eq. 9 (equals 0 when one lambda_i is 0).
 *   R3  The Eq. 42 ghost offset is applied on every link into a solid, axis
 *       or diagonal, with c at the wall taken as c at the fluid node.  It is
 *       used only for the Laplacian of c_i inside mu_i (Eq. 8).  A neutral
 *       (non-wetting) wall uses cos = 0, i.e. the symmetric ghost.
 *   R4  Eq. 43 symmetric ghosts (value of the centre node) feed grad c_i,
 *       grad rho and lap mu_i.
 *   R5  Velocity lid (Eqs. 51-53): the top row y = ny-1 is the boundary row
 *       x_u, its neighbour x_f is the node directly below.  At x_u the
 *       macroscopic c_i, mu_i, rho, p and the gradients are those of x_f,
 *       u = (U0, 0).  The pre-collision distributions at x_u are rebuilt at
 *       the start of each step by Eq. 51 from the pre-collision
 *       distributions of x_f, then x_u collides and streams like any node.
 *       Populations that would leave the lattice through the lid are
 *       dropped; the slots of x_u that nothing streams into are zero.
 *   R6  At a lattice corner that is outside in both x and y, the x edge
 *       decides the kind of the outside site.
 *   R7  Body force G = rho * (gx, gy); the paper's gravity is (0, -g).
 *   R8  MRT option (the paper uses BGK only): each distribution relaxes in the
 *       orthogonal D2Q9 moment basis of Lallemand and Luo (density, energy,
 *       energy squared, x flux, x energy flux, y flux, y energy flux, two
 *       stresses) with f' = f - M^-1 S (M f - M f^eq) + M^-1 (I - S/2) M F,
 *       F the source without its (1 - 1/(2 tau)) factor, so S = I / tau is
 *       exactly the BGK update.  f^i: fluxes (and the conserved density) at
 *       1/tau_i, which fixes the mobility of Eq. 18a; the other moments at
 *       mrt_s_f.  g: density, fluxes and stresses at 1/tau_g, which fixes the
 *       viscosity of Eq. 18b; energy, energy squared and energy fluxes at
 *       mrt_s_g.  The F_a part of Eq. 11b carries no (1 - 1/(2 tau_g)) factor
 *       and is added after the relaxation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "tlb_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- D2Q9 lattice, Eq. 10 ------------------------------------------------ */
/* e_0 = 0; e_1..e_4 along (k-1) pi/2; e_5..e_8 along (k-5) pi/2 + pi/4. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WK[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* k-bar: the direction opposite to k (Eq. 44). */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#define CS2 (1.0 / 3.0) /* c_s^2 = c^2 / 3 with c = dx/dt = 1 */

/* ---- parameters: orc_params (tlb_oracle.h) ------------------------------- */

enum { EDGE_PERIODIC = 0, EDGE_WETTING = 1, EDGE_NEUTRAL = 2, EDGE_LID = 3 };
enum { SITE_FLUID = 0, SITE_LID = 1, SITE_WET = 2, SITE_NEUTRAL = 3, SITE_VOID = 4 };
enum { E_LEFT = 0, E_RIGHT = 1, E_BOTTOM = 2, E_TOP = 3 };

typedef struct {
    int nx, ny;
    int edge[4];
    unsigned char *mask; /* 0 fluid, 1 wetting solid, 2 neutral solid */
    orc_params P;
    /* derived constants */
    double lam[3], lamT, M[2], eta[2], cos12, cos13, cos23;
    /* state: 27 planes (f1 k=0..8, f2 k=0..8, g k=0..8) and 4 planes of
     * (c1 ux, c1 uy, c2 ux, c2 uy) from the previous step (Eq. 19) */
    double *f, *fn, *cu;
    /* macroscopic fields of the current step */
    double *c1, *c2, *rho, *mu1, *mu2, *mu3;
    double *gc1x, *gc1y, *gc2x, *gc2y, *grx, *gry, *lm1, *lm2;
    double *ux, *uy, *p;
    /* site kind of every node and of its 9 neighbours, with the wrapped
     * neighbour index (a lookup table of site(), built by orc_set_geometry) */
    unsigned char *kind, *nbk;
    long *nbi;
    int have_params;
} orc_lattice;

#define NPL 27

/* ---- small helpers exported for the unit tests --------------------------- */

/* Eq. 7 and Eq. 9 (reading R2). */
void orc_lambdas(double s12, double s13, double s23, double lam[4])
{
    lam[0] = s12 + s13 - s23;
    lam[1] = s12 + s23 - s13;
    lam[2] = s13 + s23 - s12;
    double den = lam[0] * lam[1] + lam[0] * lam[2] + lam[1] * lam[2];
    lam[3] = den != 0.0 ? 3.0 * lam[0] * lam[1] * lam[2] / den : 0.0;
}

/* Eq. 8: chemical potentials mu_1, mu_2, mu_3 from c_1, c_2 (c_3 = 1 - c_1 -
 * c_2, Eq. 3) and the Laplacians of c_1, c_2 (lap c_3 = -lap c_1 - lap c_2). */
void orc_chem_pot(const double lam[4], double D, double c1, double c2,
                  double lap1, double lap2, double mu[3])
{
    double c[3] = {c1, c2, 1.0 - c1 - c2};
    double lap[3] = {lap1, lap2, -lap1 - lap2};
    double lamT = lam[3];
    for (int i = 0; i < 3; i++) {
        double bulk = lam[i] * c[i] * (1.0 - c[i]) * (1.0 - 2.0 * c[i]) -
                      2.0 * lamT * c1 * c2 * (1.0 - c1 - c2);
        mu[i] = 12.0 / D * bulk - 0.75 * D * lam[i] * lap[i];
    }
}

/* Eq. 42: offset c_ghost - c_f of the three order parameters on a link into a
 * wetting wall, with c at the wall taken equal to c at the fluid node. */
void orc_wet_offset(double cos12, double cos13, double cos23, double D,
                    double c1, double c2, double off[3])
{
    double c3 = 1.0 - c1 - c2;
    double dx = 1.0;
    off[0] = 4.0 * dx / D * (cos13 * c1 * c3 + cos12 * c1 * c2);
    off[1] = 4.0 * dx / D * (-cos12 * c1 * c2 + cos23 * c2 * c3);
    off[2] = 4.0 * dx / D * (-cos23 * c2 * c3 - cos13 * c1 * c3);
}

/* Eq. 20a: isotropic gradient from the 9 values v[k] = chi(x + e_k). */
void orc_grad(const double v[9], double g[2])
{
    g[0] = 0.0;
    g[1] = 0.0;
    for (int k = 1; k < 9; k++) {
        g[0] += WK[k] * EX[k] * v[k] / CS2;
        g[1] += WK[k] * EY[k] * v[k] / CS2;
    }
}

/* Eq. 20b: isotropic Laplacian from the 9 values v[k] = chi(x + e_k). */
double orc_lap(const double v[9])
{
    double s = 0.0;
    for (int k = 1; k < 9; k++)
        s += 2.0 * WK[k] * (v[k] - v[0]) / CS2;
    return s;
}

/* Eq. 4. */
double orc_sk(int k, double ux, double uy)
{
    double eu = EX[k] * ux + EY[k] * uy;
    double uu = ux * ux + uy * uy;
    return WK[k] * (eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. 2a: order-parameter equilibrium. */
double orc_feq(int k, double c, double mu, double eta, double ux, double uy)
{
    if (k == 0)
        return c + (WK[0] - 1.0) * eta * mu;
    double eu = EX[k] * ux + EY[k] * uy;
    return WK[k] * eta * mu + WK[k] * c * eu / CS2;
}

/* Eq. 2b: hydrodynamic equilibrium. */
double orc_geq(int k, double p, double rho, double ux, double uy)
{
    double s = orc_sk(k, ux, uy);
    if (k == 0)
        return p / CS2 * (WK[0] - 1.0) + rho * s;
    return p / CS2 * WK[k] + rho * s;
}

/* Eq. 11a: order-parameter source, given d/dt (c_i u) (Eq. 19). */
double orc_src_f(int k, double tau, double dtcux, double dtcuy)
{
    return (1.0 - 1.0 / (2.0 * tau)) * WK[k] * (EX[k] * dtcux + EY[k] * dtcuy) / CS2;
}

/* Eq. 11b: hydrodynamic forcing; Ft = F_s + G, Fa the interfacial force. */
double orc_src_g(int k, double taug, double ux, double uy, double grx,
                 double gry, double Ftx, double Fty, double Fax, double Fay)
{
    double s = orc_sk(k, ux, uy);
    double bx = s * grx + (s + WK[k]) * Ftx / CS2;
    double by = s * gry + (s + WK[k]) * Fty / CS2;
    return (1.0 - 1.0 / (2.0 * taug)) * ((EX[k] - ux) * bx + (EY[k] - uy) * by) +
           WK[k] * (EX[k] * Fax + EY[k] * Fay) / CS2;
}

/* Number of OpenMP threads the passes use (1 without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of OpenMP threads of the passes (no effect without OpenMP);
 * results do not depend on it (each pass writes per-node outputs only). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---- MRT option (reading R8) ---------------------------------------------- */
/* Moment matrix: rows are 1, e = -4 + 3|e_k|^2, eps = 4 - 21/2 |e_k|^2 + 9/2 |e_k|^4,
 * j_x = e_kx, q_x = (-5 + 3|e_k|^2) e_kx, j_y, q_y, p_xx = e_kx^2 - e_ky^2, p_xy = e_kx e_ky. */
static const double MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};
/* squared row norms: the rows are orthogonal, so M^-1 = M^T diag(1 / norm) */
static const double MNORM[9] = {9, 36, 36, 6, 12, 6, 12, 4, 4};

void orc_mrt_matrix(double out[81])
{
    for (int r = 0; r < 9; r++)
        for (int k = 0; k < 9; k++)
            out[9 * r + k] = MM[r][k];
}

void orc_mrt_inverse(double out[81])
{
    for (int k = 0; k < 9; k++)
        for (int r = 0; r < 9; r++)
            out[9 * k + r] = MM[r][k] / MNORM[r];
}

/* f' = f - M^-1 S (M f - M feq) + M^-1 (I - S/2) M src for one distribution. */
static void mrt_relax(const double f[9], const double feq[9], const double src[9], const double s[9],
                      double out[9])
{
    double mp[9];
    for (int r = 0; r < 9; r++) {
        double m = 0.0, meq = 0.0, ms = 0.0;
        for (int k = 0; k < 9; k++) {
            m += MM[r][k] * f[k];
            meq += MM[r][k] * feq[k];
            ms += MM[r][k] * src[k];
        }
        mp[r] = m - s[r] * (m - meq) + (1.0 - s[r] / 2.0) * ms;
    }
    for (int k = 0; k < 9; k++) {
        double v = 0.0;
        for (int r = 0; r < 9; r++)
            v += MM[r][k] * mp[r] / MNORM[r];
        out[k] = v;
    }
}

/* Exported for the tests: one MRT relaxation with the given rates. */
void orc_mrt_relax(const double f[9], const double feq[9], const double src[9], const double s[9],
                   double out[9])
{
    mrt_relax(f, feq, src, s, out);
}

int orc_ex(int k) { return EX[k]; }
int orc_ey(int k) { return EY[k]; }
double orc_w(int k) { return WK[k]; }
int orc_opp(int k) { return OPP[k]; }

/* ---- lattice ------------------------------------------------------------- */

static void *zalloc(size_t n) { return calloc(n, 1); }

orc_lattice *orc_create(int nx, int ny, const int edge[4])
{
    if (nx < 3 || ny < 3)
        return NULL;
    orc_lattice *L = (orc_lattice *)zalloc(sizeof(orc_lattice));
    size_t n = (size_t)nx * ny;
    L->nx = nx;
    L->ny = ny;
    for (int e = 0; e < 4; e++)
        L->edge[e] = edge[e];
    L->mask = (unsigned char *)zalloc(n);
    L->kind = (unsigned char *)zalloc(n);
    L->nbk = (unsigned char *)zalloc(9 * n);
    L->nbi = (long *)zalloc(9 * n * sizeof(long));
    L->f = (double *)zalloc(NPL * n * sizeof(double));
    L->fn = (double *)zalloc(NPL * n * sizeof(double));
    L->cu = (double *)zalloc(4 * n * sizeof(double));
    double **fields[] = {&L->c1,   &L->c2,   &L->rho,  &L->mu1, &L->mu2,
                         &L->mu3,  &L->gc1x, &L->gc1y, &L->gc2x, &L->gc2y,
                         &L->grx,  &L->gry,  &L->lm1,  &L->lm2, &L->ux,
                         &L->uy,   &L->p};
    for (size_t i = 0; i < sizeof(fields) / sizeof(fields[0]); i++)
        *fields[i] = (double *)zalloc(n * sizeof(double));
    return L;
}

void orc_destroy(orc_lattice *L)
{
    if (!L)
        return;
    double *fields[] = {L->c1,   L->c2,   L->rho,  L->mu1, L->mu2, L->mu3,
                        L->gc1x, L->gc1y, L->gc2x, L->gc2y, L->grx, L->gry,
                        L->lm1,  L->lm2,  L->ux,   L->uy,  L->p};
    for (size_t i = 0; i < sizeof(fields) / sizeof(fields[0]); i++)
        free(fields[i]);
    free(L->mask);
    free(L->kind);
    free(L->nbk);
    free(L->nbi);
    free(L->f);
    free(L->fn);
    free(L->cu);
    free(L);
}


/* Derived constants: Eqs. 7, 9 (R2), 12, 18a (R1), 38. */
void orc_set_params(orc_lattice *L, const orc_params *P)
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

/* Classify the lattice site (x, y), which may lie outside the lattice; on
 * success *idx is the wrapped linear index of an inside site. */
static int site(const orc_lattice *L, int x, int y, long *idx)
{
    int nx = L->nx, ny = L->ny;
    if (x < 0 || x >= nx) {
        int e = x < 0 ? E_LEFT : E_RIGHT;
        if (L->edge[e] != EDGE_PERIODIC)
            return L->edge[e] == EDGE_WETTING ? SITE_WET : SITE_NEUTRAL;
        x = (x + nx) % nx;
    }
    if (y < 0 || y >= ny) {
        int e = y < 0 ? E_BOTTOM : E_TOP;
        if (L->edge[e] == EDGE_LID)
            return SITE_VOID;
        if (L->edge[e] != EDGE_PERIODIC)
            return L->edge[e] == EDGE_WETTING ? SITE_WET : SITE_NEUTRAL;
        y = (y + ny) % ny;
    }
    *idx = (long)y * nx + x;
    if (L->mask[*idx] == 1)
        return SITE_WET;
    if (L->mask[*idx] == 2)
        return SITE_NEUTRAL;
    if (L->edge[E_TOP] == EDGE_LID && y == ny - 1)
        return SITE_LID;
    return SITE_FLUID;
}

static int is_fluidlike(int s) { return s == SITE_FLUID || s == SITE_LID; }

/* Store the solid mask and tabulate site() for every node and neighbour. */
void orc_set_geometry(orc_lattice *L, const unsigned char *mask)
{
    long n = (long)L->nx * L->ny;
    memcpy(L->mask, mask, (size_t)n);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        int x = (int)(i % L->nx), y = (int)(i / L->nx);
        long j = i;
        L->kind[i] = (unsigned char)site(L, x, y, &j);
        for (int k = 0; k < 9; k++) {
            j = -1;
            L->nbk[(long)k * n + i] = (unsigned char)site(L, x + EX[k], y + EY[k], &j);
            L->nbi[(long)k * n + i] = j;
        }
    }
}

/* Kind of neighbour k of node i, and its index (valid when inside). */
static int nbr(const orc_lattice *L, int k, long i, long *j)
{
    long n = (long)L->nx * L->ny;
    *j = L->nbi[(long)k * n + i];
    return L->nbk[(long)k * n + i];
}

/* Index of the lid node's neighbour x_f (directly below), R5. */
static long below(const orc_lattice *L, long idx) { return idx - L->nx; }

/* Stage 1 (Eqs. 13a, 3, 14): c_1, c_2 and rho at every fluid node; the lid
 * row copies c from the node below (R5). */
static void stage_order_parameters(orc_lattice *L, const double *f)
{
    long n = (long)L->nx * L->ny;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        L->c1[i] = L->c2[i] = L->rho[i] = 0.0;
        if (L->kind[i] != SITE_FLUID)
            continue;
        double a = 0.0, b = 0.0;
        for (int k = 0; k < 9; k++) {
            a += f[(long)k * n + i];
            b += f[(long)(9 + k) * n + i];
        }
        L->c1[i] = a;
        L->c2[i] = b;
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        if (L->kind[i] == SITE_LID) {
            L->c1[i] = L->c1[below(L, i)];
            L->c2[i] = L->c2[below(L, i)];
        }
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        if (!is_fluidlike(L->kind[i]))
            continue;
        double c1 = L->c1[i], c2 = L->c2[i];
        L->rho[i] = c1 * L->P.rho1 + c2 * L->P.rho2 + (1.0 - c1 - c2) * L->P.rho3;
    }
}

/* Stage 2 (Eqs. 8, 20b, 42): chemical potentials with wetting ghosts. */
static void stage_chemical_potentials(orc_lattice *L)
{
    long n = (long)L->nx * L->ny;
    double lam4[4] = {L->lam[0], L->lam[1], L->lam[2], L->lamT};
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        L->mu1[i] = L->mu2[i] = L->mu3[i] = 0.0;
        if (L->kind[i] != SITE_FLUID)
            continue;
        double v1[9], v2[9];
        v1[0] = L->c1[i];
        v2[0] = L->c2[i];
        for (int k = 1; k < 9; k++) {
            long nb;
            int s = nbr(L, k, i, &nb);
            if (is_fluidlike(s)) {
                v1[k] = L->c1[nb];
                v2[k] = L->c2[nb];
            } else if (s == SITE_WET) {
                double off[3];
                orc_wet_offset(L->cos12, L->cos13, L->cos23, L->P.D, L->c1[i],
                               L->c2[i], off);
                v1[k] = L->c1[i] + off[0];
                v2[k] = L->c2[i] + off[1];
            } else { /* neutral wall: cos = 0 (R3) */
                v1[k] = L->c1[i];
                v2[k] = L->c2[i];
            }
        }
        double mu[3];
        orc_chem_pot(lam4, L->P.D, L->c1[i], L->c2[i], orc_lap(v1), orc_lap(v2), mu);
        L->mu1[i] = mu[0];
        L->mu2[i] = mu[1];
        L->mu3[i] = mu[2];
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        if (L->kind[i] == SITE_LID) {
            L->mu1[i] = L->mu1[below(L, i)];
            L->mu2[i] = L->mu2[below(L, i)];
            L->mu3[i] = L->mu3[below(L, i)];
        }
    }
}

/* Stage 3 (Eqs. 20a, 20b, 43): grad c_i, grad rho, lap mu_i with symmetric
 * ghosts; the lid row copies them from the node below (R5). */
static void stage_gradients(orc_lattice *L)
{
    long n = (long)L->nx * L->ny;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        L->gc1x[i] = L->gc1y[i] = L->gc2x[i] = L->gc2y[i] = 0.0;
        L->grx[i] = L->gry[i] = L->lm1[i] = L->lm2[i] = 0.0;
        if (L->kind[i] != SITE_FLUID)
            continue;
        double vc1[9], vc2[9], vr[9], vm1[9], vm2[9];
        for (int k = 0; k < 9; k++) {
            long nb = i;
            int s = k == 0 ? SITE_FLUID : nbr(L, k, i, &nb);
            long src = is_fluidlike(s) ? nb : i; /* Eq. 43 */
            vc1[k] = L->c1[src];
            vc2[k] = L->c2[src];
            vr[k] = L->rho[src];
            vm1[k] = L->mu1[src];
            vm2[k] = L->mu2[src];
        }
        double g[2];
        orc_grad(vc1, g);
        L->gc1x[i] = g[0];
        L->gc1y[i] = g[1];
        orc_grad(vc2, g);
        L->gc2x[i] = g[0];
        L->gc2y[i] = g[1];
        orc_grad(vr, g);
        L->grx[i] = g[0];
        L->gry[i] = g[1];
        L->lm1[i] = orc_lap(vm1);
        L->lm2[i] = orc_lap(vm2);
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        if (L->kind[i] != SITE_LID)
            continue;
        long b = below(L, i);
        L->gc1x[i] = L->gc1x[b];
        L->gc1y[i] = L->gc1y[b];
        L->gc2x[i] = L->gc2x[b];
        L->gc2y[i] = L->gc2y[b];
        L->grx[i] = L->grx[b];
        L->gry[i] = L->gry[b];
        L->lm1[i] = L->lm1[b];
        L->lm2[i] = L->lm2[b];
    }
}

/* Surface-tension force F_s = sum_{i=1..3} mu_i grad c_i (text below Eq. 11),
 * with grad c_3 = -grad c_1 - grad c_2 (Eq. 3). */
static void surface_force(const orc_lattice *L, long i, double F[2])
{
    double g3x = -L->gc1x[i] - L->gc2x[i], g3y = -L->gc1y[i] - L->gc2y[i];
    F[0] = L->mu1[i] * L->gc1x[i] + L->mu2[i] * L->gc2x[i] + L->mu3[i] * g3x;
    F[1] = L->mu1[i] * L->gc1y[i] + L->mu2[i] * L->gc2y[i] + L->mu3[i] * g3y;
}

/* Stage 4 (Eqs. 13b, 13c): velocity and pressure. */
static void stage_velocity_pressure(orc_lattice *L, const double *f)
{
    long n = (long)L->nx * L->ny;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        L->ux[i] = L->uy[i] = L->p[i] = 0.0;
        if (L->kind[i] != SITE_FLUID)
            continue;
        const double *g = f + 18 * n;
        double Fs[2];
        surface_force(L, i, Fs);
        double rho = L->rho[i];
        double Gx = rho * L->P.gx, Gy = rho * L->P.gy;
        double mx = 0.0, my = 0.0, sum = 0.0;
        for (int k = 0; k < 9; k++) {
            mx += EX[k] * g[(long)k * n + i];
            my += EY[k] * g[(long)k * n + i];
            if (k != 0)
                sum += g[(long)k * n + i];
        }
        double ux = (mx + 0.5 * (Fs[0] + Gx)) / rho;
        double uy = (my + 0.5 * (Fs[1] + Gy)) / rho;
        double p = CS2 / (1.0 - WK[0]) *
                   (sum + 0.5 * (ux * L->grx[i] + uy * L->gry[i]) + rho * orc_sk(0, ux, uy));
        L->ux[i] = ux;
        L->uy[i] = uy;
        L->p[i] = p;
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        if (L->kind[i] != SITE_LID)
            continue;
        L->ux[i] = L->P.lid_u; /* Eq. 53: u(x_u) = (U0, 0) */
        L->uy[i] = 0.0;
        L->p[i] = L->p[below(L, i)];
    }
}

/* Surface-tension force F_s and interfacial force F_a = u sum_{i=1,2}
 * (rho_i - rho_3) M_i lap mu_i (Eq. 12) at node i. */
static void node_forces(const orc_lattice *L, long i, double Fs[2], double Fa[2])
{
    surface_force(L, i, Fs);
    double a = (L->P.rho1 - L->P.rho3) * L->M[0] * L->lm1[i] +
               (L->P.rho2 - L->P.rho3) * L->M[1] * L->lm2[i];
    Fa[0] = L->ux[i] * a;
    Fa[1] = L->uy[i] * a;
}

static void compute_macros(orc_lattice *L, const double *f)
{
    stage_order_parameters(L, f);
    stage_chemical_potentials(L);
    stage_gradients(L);
    stage_velocity_pressure(L, f);
}

/* One time step: stages 1-4, then forces, collision (Eqs. 1a, 1b, 45) and
 * streaming with half-way bounce-back (Eq. 44). */
int orc_step(orc_lattice *L, long nsteps)
{
    if (!L->have_params)
        return -1;
    long n = (long)L->nx * L->ny;
    const double tau[2] = {L->P.tau1, L->P.tau2};
    for (long step = 0; step < nsteps; step++) {
        compute_macros(L, L->f);
        memset(L->fn, 0, NPL * n * sizeof(double));
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; i++) {
            int s = L->kind[i];
            if (!is_fluidlike(s))
                continue;
            double c[2] = {L->c1[i], L->c2[i]};
            double mu[2] = {L->mu1[i], L->mu2[i]};
            double ux = L->ux[i], uy = L->uy[i], p = L->p[i], rho = L->rho[i];
            double c3 = 1.0 - c[0] - c[1];
            /* Eq. 15 and Eq. 18b: local viscosity and tau_g. */
            double nu = c[0] * L->P.nu1 + c[1] * L->P.nu2 + c3 * L->P.nu3;
            double taug = nu / CS2 + 0.5;
            double Fs[2], Fa[2];
            node_forces(L, i, Fs, Fa);
            double Gx = rho * L->P.gx, Gy = rho * L->P.gy;
            double Fax = Fa[0], Fay = Fa[1];
            /* Eq. 19: explicit Euler time derivative of c_i u. */
            double dcu[2][2];
            for (int q = 0; q < 2; q++) {
                dcu[q][0] = c[q] * ux - L->cu[(long)(2 * q) * n + i];
                dcu[q][1] = c[q] * uy - L->cu[(long)(2 * q + 1) * n + i];
            }
            /* Pre-collision distributions; Eq. 51 on the lid row (R5). */
            double fin[NPL];
            for (int m = 0; m < NPL; m++)
                fin[m] = L->f[(long)m * n + i];
            if (s == SITE_LID) {
                long b = below(L, i);
                for (int k = 0; k < 9; k++) {
                    for (int q = 0; q < 2; q++) {
                        double cb = q == 0 ? L->c1[b] : L->c2[b];
                        double mb = q == 0 ? L->mu1[b] : L->mu2[b];
                        double eq_u = orc_feq(k, cb, mb, L->eta[q], ux, uy);   /* Eq. 53a */
                        double eq_f = orc_feq(k, cb, mb, L->eta[q], L->ux[b], L->uy[b]);
                        fin[9 * q + k] = eq_u + (L->f[(long)(9 * q + k) * n + b] - eq_f); /* Eqs. 51, 52 */
                    }
                    double geq_u = orc_geq(k, L->p[b], L->rho[b], ux, uy);   /* Eq. 53b */
                    double geq_f = orc_geq(k, L->p[b], L->rho[b], L->ux[b], L->uy[b]);
                    fin[18 + k] = geq_u + (L->f[(long)(18 + k) * n + b] - geq_f);
                }
            }
            /* Collision, Eqs. 1a, 1b and 45 (BGK), or the MRT option (R8). */
            double fpost[NPL];
            if (L->P.collision != 0.0) {
                for (int q = 0; q < 2; q++) {
                    double eq[9], src[9], s[9], out[9];
                    for (int k = 0; k < 9; k++) {
                        eq[k] = orc_feq(k, c[q], mu[q], L->eta[q], ux, uy);
                        /* Eq. 11a without its (1 - 1/(2 tau_i)) factor */
                        src[k] = orc_src_f(k, tau[q], dcu[q][0], dcu[q][1]) / (1.0 - 1.0 / (2.0 * tau[q]));
                        s[k] = L->P.mrt_s_f;
                    }
                    s[0] = s[3] = s[5] = 1.0 / tau[q];
                    mrt_relax(&fin[9 * q], eq, src, s, out);
                    for (int k = 0; k < 9; k++)
                        fpost[9 * q + k] = out[k];
                }
                double eq[9], src[9], s[9], out[9];
                for (int k = 0; k < 9; k++) {
                    eq[k] = orc_geq(k, p, rho, ux, uy);
                    /* Eq. 11b: the bracket without (1 - 1/(2 tau_g)); F_a added below */
                    double with_fa = orc_src_g(k, taug, ux, uy, L->grx[i], L->gry[i], Fs[0] + Gx,
                                               Fs[1] + Gy, Fax, Fay);
                    double fa = WK[k] * (EX[k] * Fax + EY[k] * Fay) / CS2;
                    src[k] = (with_fa - fa) / (1.0 - 1.0 / (2.0 * taug));
                    s[k] = 1.0 / taug;
                }
                s[1] = s[2] = s[4] = s[6] = L->P.mrt_s_g;
                mrt_relax(&fin[18], eq, src, s, out);
                for (int k = 0; k < 9; k++)
                    fpost[18 + k] = out[k] + WK[k] * (EX[k] * Fax + EY[k] * Fay) / CS2;
            } else
            for (int k = 0; k < 9; k++) {
                for (int q = 0; q < 2; q++) {
                    double eq = orc_feq(k, c[q], mu[q], L->eta[q], ux, uy);
                    double src = orc_src_f(k, tau[q], dcu[q][0], dcu[q][1]);
                    double fk = fin[9 * q + k];
                    fpost[9 * q + k] = fk - (fk - eq) / tau[q] + src;
                }
                double geq = orc_geq(k, p, rho, ux, uy);
                double src = orc_src_g(k, taug, ux, uy, L->grx[i], L->gry[i],
                                       Fs[0] + Gx, Fs[1] + Gy, Fax, Fay);
                double gk = fin[18 + k];
                fpost[18 + k] = gk - (gk - geq) / taug + src;
            }
            /* Streaming (Eq. 1) and half-way bounce-back (Eq. 44). */
            for (int k = 0; k < 9; k++) {
                long dst = i;
                int sd = k == 0 ? SITE_FLUID : nbr(L, k, i, &dst);
                for (int q = 0; q < 3; q++) {
                    double v = fpost[9 * q + k];
                    if (is_fluidlike(sd))
                        L->fn[(long)(9 * q + k) * n + dst] = v;
                    else if (sd == SITE_WET || sd == SITE_NEUTRAL)
                        L->fn[(long)(9 * q + OPP[k]) * n + i] = v;
                    /* SITE_VOID: leaves the lattice through the lid (R5) */
                }
            }
            /* Store c_i u for the next step's Eq. 19. */
            for (int q = 0; q < 2; q++) {
                L->cu[(long)(2 * q) * n + i] = c[q] * ux;
                L->cu[(long)(2 * q + 1) * n + i] = c[q] * uy;
            }
        }
        double *t = L->f;
        L->f = L->fn;
        L->fn = t;
    }
    return 0;
}

/* Initial state (reading of the silent set-up): f = f^eq(c, mu(c), u),
 * g = g^eq(p, rho(c), u), c_i u stored for Eq. 19.  Inputs are node arrays
 * of length nx*ny; p may be NULL (zero). */
int orc_set_fields(orc_lattice *L, const double *c1, const double *c2,
                   const double *ux, const double *uy, const double *p)
{
    if (!L->have_params)
        return -1;
    long n = (long)L->nx * L->ny;
    /* Load c into a scratch state whose f_0 carries c, so that stage 1 gives
     * back exactly the requested fields. */
    memset(L->fn, 0, NPL * n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        L->fn[i] = c1[i];
        L->fn[9 * n + i] = c2[i];
    }
    stage_order_parameters(L, L->fn);
    stage_chemical_potentials(L);
    memset(L->f, 0, NPL * n * sizeof(double));
    memset(L->fn, 0, NPL * n * sizeof(double));
    memset(L->cu, 0, 4 * n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        if (!is_fluidlike(L->kind[i]))
            continue;
        double c[2] = {L->c1[i], L->c2[i]};
        double mu[2] = {L->mu1[i], L->mu2[i]};
        double pi = p ? p[i] : 0.0;
        for (int k = 0; k < 9; k++) {
            for (int q = 0; q < 2; q++)
                L->f[(long)(9 * q + k) * n + i] = orc_feq(k, c[q], mu[q], L->eta[q], ux[i], uy[i]);
            L->f[(long)(18 + k) * n + i] = orc_geq(k, pi, L->rho[i], ux[i], uy[i]);
        }
        for (int q = 0; q < 2; q++) {
            L->cu[(long)(2 * q) * n + i] = c[q] * ux[i];
            L->cu[(long)(2 * q + 1) * n + i] = c[q] * uy[i];
        }
    }
    return 0;
}

/* Macroscopic fields of the current state, 10 planes of nx*ny in the order
 * c1, c2, c3, rho, ux, uy, p, mu1, mu2, mu3 (zero at solid nodes). */
int orc_read_fields(orc_lattice *L, double *out)
{
    if (!L->have_params)
        return -1;
    long n = (long)L->nx * L->ny;
    compute_macros(L, L->f);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        int fl = is_fluidlike(L->kind[i]);
        double v[10] = {L->c1[i], L->c2[i], 1.0 - L->c1[i] - L->c2[i], L->rho[i],
                        L->ux[i], L->uy[i], L->p[i], L->mu1[i], L->mu2[i], L->mu3[i]};
        for (int q = 0; q < 10; q++)
            out[(long)q * n + i] = fl ? v[q] : 0.0;
    }
    return 0;
}

/* Raw state: 27 distribution planes followed by the 4 c_i u planes. */
void orc_get_state(const orc_lattice *L, double *out)
{
    long n = (long)L->nx * L->ny;
    memcpy(out, L->f, NPL * n * sizeof(double));
    memcpy(out + NPL * n, L->cu, 4 * n * sizeof(double));
}

void orc_set_state(orc_lattice *L, const double *in)
{
    long n = (long)L->nx * L->ny;
    memcpy(L->f, in, NPL * n * sizeof(double));
    memcpy(L->cu, in + NPL * n, 4 * n * sizeof(double));
}

/* Forces and gradients of the current state, 8 planes of nx*ny in the order
 * Fs_x, Fs_y, Fa_x, Fa_y, lap mu1, lap mu2, d rho/dx, d rho/dy. */
int orc_read_aux(orc_lattice *L, double *out)
{
    if (!L->have_params)
        return -1;
    long n = (long)L->nx * L->ny;
    compute_macros(L, L->f);
    memset(out, 0, 8 * n * sizeof(double));
    for (long i = 0; i < n; i++) {
        if (!is_fluidlike(L->kind[i]))
            continue;
        double Fs[2], Fa[2];
        node_forces(L, i, Fs, Fa);
        double v[8] = {Fs[0], Fs[1], Fa[0], Fa[1], L->lm1[i], L->lm2[i], L->grx[i], L->gry[i]};
        for (int q = 0; q < 8; q++)
            out[(long)q * n + i] = v[q];
    }
    return 0;
}

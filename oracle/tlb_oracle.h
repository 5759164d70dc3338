/*
 * Declarations shared by the two source files of the FP64 oracle
 * (tlb_oracle.c: the D2Q9 lattice of the paper's experiments;
 * tlb_oracle3d.c: the D3Q19 form of the same model).
 *
 * TEST INFRASTRUCTURE ONLY (see tlb_oracle.c).
 */
#ifndef TLB_ORACLE_H
#define TLB_ORACLE_H

typedef struct {
    double sigma12, sigma13, sigma23;          /* surface tensions, Eq. 7 */
    double theta12_deg, theta13_deg, theta23_deg; /* contact angles, Eq. 38 */
    double rho1, rho2, rho3;                   /* densities, Eq. 14 */
    double nu1, nu2, nu3;                      /* viscosities, Eq. 15 */
    double M0;                                 /* M_i = M0 / lambda_i, Eq. 12 */
    double D;                                  /* interface thickness, Eq. 8 */
    double tau1, tau2;                         /* relaxation times, Eq. 1a */
    double gx, gy;                             /* body force per unit mass (R7) */
    double lid_u;                              /* U0 of the velocity lid, Eq. 53 */
    double collision;                          /* 0 BGK (Eqs. 1a, 1b), 1 MRT (R8) */
    double mrt_s_f;                            /* MRT rate of the non-flux moments of f^i */
    double mrt_s_g;                            /* MRT rate of e, eps, q_x, q_y of g */
} orc_params;

/* Eq. 7 and Eq. 9 (reading R2): lam[0..2] = lambda_1..3, lam[3] = lambda_T. */
void orc_lambdas(double s12, double s13, double s23, double lam[4]);
/* Eq. 8: mu_1..3 from c_1, c_2 and their Laplacians. */
void orc_chem_pot(const double lam[4], double D, double c1, double c2, double lap1, double lap2, double mu[3]);
/* Eq. 42: c_ghost - c_f of c_1..3 on a link into a wetting wall. */
void orc_wet_offset(double cos12, double cos13, double cos23, double D, double c1, double c2, double off[3]);

#endif

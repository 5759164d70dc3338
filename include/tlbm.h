/*
 * tlbm.h -- C ABI of the GB300 lattice library for the phase-field lattice
 * Boltzmann ternary-fluid model with ternary wetting boundaries of
 * Liang, Li, Shi and Chai, "Lattice Boltzmann modeling of wall-bounded ternary
 * fluid flows" (arXiv:1710.09534), Sec. II.
 *
 * One call of tlb_step advances one D2Q9 lattice by n time steps on the
 * caller's CUDA stream: two order-parameter distributions f^1, f^2 and one
 * hydrodynamic distribution g (Eqs. 1a, 1b) with BGK collision, equilibria
 * (Eqs. 2a, 2b, 4), sources (Eqs. 11a, 11b, 12, 19), moments (Eqs. 13-15),
 * chemical potentials (Eqs. 8, 9) from the isotropic stencils (Eqs. 20a, 20b),
 * the ternary wetting ghost values (Eq. 42), symmetric ghosts (Eq. 43),
 * half-way bounce-back (Eq. 44) and the non-equilibrium-extrapolation velocity
 * lid (Eqs. 51-53).
 *
 * Conventions shared by every call
 *   - Node arrays are row-major [ny][nx] (x fastest); node (i, j) sits at
 *     (x, y) = (i, j).  Host arrays are copied, never retained.
 *   - Edges are given as int32 edges[4] = {left, right, bottom, top}, each one
 *     of TLB_EDGE_*.  A periodic edge must be paired with a periodic opposite
 *     edge.  Half-way walls sit half a spacing outside the lattice.  The lid is
 *     allowed on the top edge only; it turns row ny-1 into the boundary row
 *     x_u of Eq. 51, whose neighbour x_f is the node directly below.  At a
 *     corner outside in both x and y, the x edge decides the kind of site.
 *   - Readings of the paper that both this library and its FP64 oracle follow:
 *     eta_i = M_i / (cs^2 (tau_i - 1/2)) per component with M_i = M0/lambda_i;
 *     lambda_T = 3 l1 l2 l3 / (l1 l2 + l1 l3 + l2 l3); the Eq. 42 offset on
 *     every solid link (axis or diagonal), used only for lap c_i inside mu_i;
 *     a neutral wall is cos = 0; body force G = rho (gx, gy).
 *   - Every call returns TLB_OK or a negative TLB_E* code and sets a
 *     thread-local message readable with tlb_last_error().  No call aborts
 *     or throws.  Device work is asynchronous on the stream given at creation
 *     unless a call says that it synchronizes.
 *   - Memory ownership: the caller allocates the device workspace
 *     (tlb_workspace_bytes) and keeps it and the stream alive until
 *     tlb_destroy.  The library itself never allocates device memory.
 */
#ifndef TLBM_H
#define TLBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tlb_lattice tlb_lattice;
typedef struct tlb_batch tlb_batch;

/* Storage precision of the distributions.  TLB_FP64 computes in FP64;
 * TLB_FP32 stores and computes in FP32 (diagnostic sums in FP64).  TLB_FP16
 * and TLB_BF16 compute in FP32 and store every population except the two rest
 * populations f^i_0 in 16 bits, after subtracting its equilibrium at rest
 * (u = 0, mu = 0, p = 0: zero for all of them in this model, Eqs. 2a, 2b) and,
 * for FP16, scaling by 2^12 so that small populations stay normal numbers; the
 * rest populations (equilibrium at rest c_i) and the c_i u planes of Eq. 19 stay
 * FP32, and the rest populations absorb the 16-bit rounding of the moving ones,
 * so each component's mass is conserved as in FP32 storage.  In all precisions
 * the rest populations of f^1, f^2 in the FP32 and 16-bit formats are float
 * pairs hi + lo. */
enum { TLB_FP64 = 0, TLB_FP32 = 1, TLB_FP16 = 2, TLB_BF16 = 3 };

/* In-place streaming, OR-ed into the precision of tlb_workspace_bytes and
 * tlb_create_lattice (beyond the paper, which does not discuss storage): the
 * lattice keeps ONE distribution buffer instead of two and streams in place
 * with the AA pattern -- an even step reads each node's own slots k and
 * writes f'_k into its own slot k-bar; an odd step reads f_k from slot k-bar
 * of x - e_k and writes f'_k into slot k of x + e_k (the half-way
 * bounce-back of Eq. 44 becomes own-slot reads and writes on wall links).
 * Because the chemical potentials need the order parameters of neighbours
 * (Eqs. 8, 20), a first pass per step writes c_1, c_2 of every node to two
 * planes of the arithmetic type, which the update then reads.  Workspace:
 * 0.57 (FP64, FP32) and 0.62 (FP16, BF16) of the two-buffer size at
 * 2048x2048; each step also moves the order-parameter pass.  The results equal
 * the two-buffer update's up to rounding order.  Every call sees the usual
 * layout (a call that ends on an even step streams its result in place), so
 * all reads, diagnostics and state export work as for two buffers; such a
 * lattice cannot join a batch (TLB_EINVAL from tlb_batch_add).  tlb_set_fields
 * stages the host arrays through the order-parameter planes in bands of rows
 * (one set-up launch per band). */
enum { TLB_INPLACE = 0x100 };

enum { TLB_EDGE_PERIODIC = 0, TLB_EDGE_WETTING = 1, TLB_EDGE_NEUTRAL = 2, TLB_EDGE_LID = 3 };

/* Solid mask values for tlb_set_geometry. */
enum { TLB_NODE_FLUID = 0, TLB_NODE_WETTING_SOLID = 1, TLB_NODE_NEUTRAL_SOLID = 2 };

enum {
    TLB_OK = 0,
    TLB_EINVAL = -1,    /* invalid argument or parameter set */
    TLB_ENOMEM = -2,    /* workspace too small */
    TLB_ECUDA = -3,     /* a CUDA runtime call failed (message has the CUDA error) */
    TLB_EUNSTABLE = -4, /* non-finite values found in the state */
    TLB_ETIMEOUT = -5,  /* tlb_sync deadline passed with work still pending */
    TLB_ESTATE = -6     /* call out of order (e.g. step before set_fields) */
};

/* Field selection bits for tlb_read_fields; planes are written in bit order. */
enum {
    TLB_F_C1 = 1u << 0, TLB_F_C2 = 1u << 1, TLB_F_C3 = 1u << 2, TLB_F_RHO = 1u << 3,
    TLB_F_UX = 1u << 4, TLB_F_UY = 1u << 5, TLB_F_P = 1u << 6, TLB_F_MU1 = 1u << 7,
    TLB_F_MU2 = 1u << 8, TLB_F_MU3 = 1u << 9, TLB_F_ALL = (1u << 10) - 1u
};

/* Model parameters (Sec. II).  sigma_ij: surface tensions (Eq. 7);
 * theta_ij: static contact angles measured through fluid i (Eq. 38), which
 * must satisfy Eq. 39; rho_i, nu_i: phase densities and viscosities (Eqs. 14,
 * 15); M0: M_i = M0 / lambda_i (Eq. 12); D: interface thickness (Eq. 8);
 * tau1, tau2: relaxation times of Eq. 1a; gx, gy: body force per unit mass;
 * lid_u: U0 of Eq. 53 for a TLB_EDGE_LID top edge.
 * collision: 0 = the BGK operators of Eqs. 1a, 1b (the paper's model); 1 = a
 * multiple-relaxation-time option beyond the paper, which uses BGK only:
 * every distribution is relaxed in the orthogonal D2Q9 moment basis of
 * Lallemand and Luo, f' = f - M^-1 S (M f - M f^eq) + M^-1 (I - S/2) M F with
 * F the source of Eq. 11a/11b without its (1 - 1/(2 tau)) factor (the F_a part
 * of Eq. 11b is added unrelaxed).  Rates: for f^i the conserved and flux
 * moments (rows rho, j_x, j_y) relax at 1/tau_i and the rest at mrt_s_f; for g
 * the rows rho, j_x, j_y, p_xx, p_xy relax at 1/tau_g (so that Eq. 15 sets the
 * shear viscosity) and the energy rows e, eps, q_x, q_y at mrt_s_g.  With
 * mrt_s_f = 1/tau_i and mrt_s_g = 1/tau_g the update equals BGK.  Ignored by
 * BGK; with collision = 1, 0 < mrt_s_f, mrt_s_g < 2. */
typedef struct {
    double sigma12, sigma13, sigma23;
    double theta12_deg, theta13_deg, theta23_deg;
    double rho1, rho2, rho3;
    double nu1, nu2, nu3;
    double M0;
    double D;
    double tau1, tau2;
    double gx, gy;
    double lid_u;
    double collision;
    double mrt_s_f, mrt_s_g;
} tlb_params;

/* FP64 diagnostics of the current state (Sec. III.A measures; reduced on
 * the device in a fixed order).  mass[i] = sum over fluid nodes of c_{i+1}
 * (the lid row counts with the values of the row below it); nonfinite =
 * number of fluid nodes whose c1, c2 or g-moments are not finite. */
typedef struct {
    double mass[3];
    int64_t nonfinite;
} tlb_diag;

/* Bytes of device workspace one lattice needs (the state of Eqs. 1a/1b
 * double-buffered -- one buffer plus the order-parameter planes with
 * TLB_INPLACE -- the c_i u planes of Eq. 19, node classes and the near-wall
 * list).  precision: TLB_FP64 .. TLB_BF16, optionally | TLB_INPLACE.  Returns a
 * negative TLB_E* code for invalid sizes or precision. */
int64_t tlb_workspace_bytes(int nx, int ny, int precision);

/* Create a lattice of nx*ny nodes (nx, ny >= 3 and <= 32768) with the
 * storage precision (| TLB_INPLACE for in-place streaming).  The handle owns
 * one CUDA stream and a few events of its own (no device memory), released
 * by tlb_destroy.  dev_workspace:
 * caller-owned device memory of at least tlb_workspace_bytes, 256-byte aligned.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  *out receives
 * the handle.  The lattice starts all-fluid; parameters and fields must be set
 * before stepping. */
int tlb_create_lattice(int nx, int ny, int precision, const int32_t edges[4],
                       void *dev_workspace, int64_t ws_bytes, void *cuda_stream,
                       tlb_lattice **out);

/* Solid geometry: host_mask[ny*nx] of TLB_NODE_* values (NULL = all fluid).
 * A solid node is never updated; its fluid neighbours use the wetting ghost
 * rule (Eq. 42, wetting solids) or the symmetric rule (neutral solids) and
 * bounce back on links into it (Eq. 44).  With a lid, rows ny-2 and ny-1 must
 * be fluid.  Builds the node classes and the compacted near-wall list on the
 * host and uploads them (synchronizes the stream).  Must be followed by
 * tlb_set_fields before the next step. */
int tlb_set_geometry(tlb_lattice *lat, const uint8_t *host_mask);

/* Model parameters.  TLB_EINVAL if: any sigma_ij <= 0, lambda_1 or lambda_2
 * <= 0, lambda_3 < 0 (Eq. 7); D <= 0; rho_i <= 0; nu_i <= 0; tau_i <= 1/2;
 * M0 <= 0; the Eq. 39 residual |s12 cos t12 - s13 cos t13 + s23 cos t23| >
 * 1e-6 max(sigma); a non-finite value; collision not 0 or 1; with collision
 * = 1, an MRT rate outside (0, 2).  Changing the collision model of a batch
 * member makes the next batch step fail unless every member agrees.  lambda_i <= lambda_T / 2 (outside the
 * well-posed range stated after Eq. 7) is accepted; the message then says so. */
int tlb_set_params(tlb_lattice *lat, const tlb_params *params);

/* Initial state from host node arrays (length nx*ny each; p may be NULL for
 * p = 0): f^i = f^{i,eq}(c_i, mu_i(c), u) (Eq. 2a with mu from Eq. 8),
 * g = g^eq(p, rho(c), u) (Eq. 2b), stored c_i u = c_i u (so the first Eq. 19
 * derivative is zero for a still start).  Solid nodes get zero.  The lid row
 * takes c and mu from the row below.  Synchronizes the stream. */
int tlb_set_fields(tlb_lattice *lat, const double *c1, const double *c2, const double *ux,
                   const double *uy, const double *p);

/* The same from device FP64 arrays (length nx*ny each, p may be NULL);
 * asynchronous; the arrays must stay valid until the stream reaches it. */
int tlb_set_fields_device(tlb_lattice *lat, const double *c1, const double *c2,
                          const double *ux, const double *uy, const double *p);

/* Advance n >= 0 time steps, asynchronously on the stream: per step one fused
 * interior kernel and one near-wall kernel (in-place lattices: the
 * order-parameter pass, the interior kernel, the lid row if any, the
 * near-wall kernel, and after a last even step the in-place streaming).  The
 * near-wall launches run on a stream the lattice owns, ordered after the
 * step's earlier work and joined back into the caller's stream before the
 * step ends, so work the caller queues after tlb_step sees the whole step.
 * TLB_ESTATE before set_fields. */
int tlb_step(tlb_lattice *lat, int64_t n);

/* Wait for the stream with a deadline (timeout_ms < 0: no deadline).
 * TLB_ETIMEOUT if work is still pending at the deadline (nothing is
 * cancelled), TLB_ECUDA if the stream reported an error. */
int tlb_sync(tlb_lattice *lat, int64_t timeout_ms);

/* Macroscopic fields of the current state as FP64 planes of nx*ny, in the
 * order of the set bits of field_mask (TLB_F_*): c1, c2, c3, rho, ux, uy, p,
 * mu1, mu2, mu3.  Solid nodes read 0; the lid row reads the row below it with
 * u = (U0, 0).  host_out receives popcount(field_mask)*nx*ny doubles.
 * Synchronizes the stream. */
int tlb_read_fields(tlb_lattice *lat, uint32_t field_mask, double *host_out);

/* The same into device memory (dev_out: popcount(field_mask)*nx*ny doubles);
 * asynchronous. */
int tlb_read_fields_device(tlb_lattice *lat, uint32_t field_mask, double *dev_out);

/* FP64 mass totals and non-finite count (see tlb_diag); synchronizes.
 * Returns TLB_EUNSTABLE (with *out filled) if nonfinite > 0. */
int tlb_diagnostics(tlb_lattice *lat, tlb_diag *out);

/* Contact-line diagnostic of a drop of fluid `component` (1 or 2) on the
 * bottom wall, in FP64 on the device (Sec. III.A: theta_n = 2 atan(2 H_d /
 * L_s)).  A drop is a run of wall-row nodes (row y = 0, periodic in x) with
 * c >= 1/2; L_s is the distance between its two c = 1/2 crossings on that row
 * (linear interpolation); H_d is the largest, over the run's columns, of the
 * c = 1/2 crossing reached by walking up from the wall through c >= 1/2
 * (linear interpolation) plus 1/2 for the half-way wall.  host_out receives
 * 4 doubles per drop {L_s, H_d, theta_n in degrees, x of the base centre} for
 * up to min(max_drops, 256) drops; *n_drops = number of drops found.
 * Synchronizes. */
int tlb_contact_angles(tlb_lattice *lat, int component, double *host_out, int max_drops, int *n_drops);

/* Film thickness on top of a solid (Sec. III.D: the film of the impacting
 * compound drop on the cylinder, Fig. 14's h), in FP64 on the device.  In
 * column x (0 <= x < nx), from the fluid node above the solid node y_top
 * (-1 <= y_top <= ny - 2; -1 is the bottom edge wall), walk up through nodes
 * whose order-parameter sum selected by comps (1: c1, 2: c2, 3: c1 + c2) is
 * >= 1/2.  *h_out = the height of the c = 1/2 crossing (linear interpolation)
 * above the half-way wall at y_top + 1/2; 0 if the first node is below 1/2;
 * measured to row ny - 1 if the sum never drops below 1/2.  No wrap in y.
 * Synchronizes. */
int tlb_film_thickness(tlb_lattice *lat, int x, int y_top, int comps, double *h_out);

/* Raw state as FP64 host planes [31][ny][nx]: f^1_k (k = 0..8), f^2_k,
 * g_k, then c1 ux, c1 uy, c2 ux, c2 uy of the previous step (Eq. 19).
 * Synchronizes. */
int tlb_read_state(tlb_lattice *lat, double *host_out);

/* Checkpoint: bytes needed, export into a host buffer and import from one
 * (the exact storage-precision state, so a resumed run is bit-identical).
 * Both synchronize.  Import requires a lattice of the same size, precision,
 * edges and geometry (TLB_EINVAL on a size mismatch). */
int64_t tlb_state_bytes(tlb_lattice *lat);
int tlb_export_state(tlb_lattice *lat, void *host_buf, int64_t bytes);
int tlb_import_state(tlb_lattice *lat, const void *host_buf, int64_t bytes);

/* theta_12 from Eq. 39 given the tensions, theta_13 and theta_23 (degrees):
 * the paper's convention when the two fluid-3 angles are prescribed
 * (Sec. III.A).  TLB_EINVAL if no angle satisfies it. */
int tlb_theta12_from(double sigma12, double sigma13, double sigma23, double theta13_deg,
                     double theta23_deg, double *theta12_deg);

/* Per-kernel timing with CUDA events on the lattice's stream.  enable = 1
 * starts recording events around the fused interior launch and the
 * near-wall launch of every step (and clears the totals); enable = 0 stops.
 * tlb_profile_read synchronizes and returns the summed device milliseconds
 * ms[0] (interior kernel), ms[1] (near-wall kernel) and the launch counts. */
int tlb_profile(tlb_lattice *lat, int enable);
int tlb_profile_read(tlb_lattice *lat, double ms[2], int64_t launches[2]);

/* Number of nodes in the near-wall list (handled by the near-wall kernel). */
int64_t tlb_wall_nodes(tlb_lattice *lat);

/* ---- Batches: many lattices advanced together -------------------------
 * A batch steps all its member lattices in lockstep: per step, one
 * persistent kernel whose blocks take (member, strip, segment) tiles of the
 * fused interior update from a shared counter and, concurrently on a stream
 * the batch owns, one loop over all the members' near-wall nodes (same
 * per-node arithmetic as tlb_step, so a member's result does not depend on
 * the rest of the batch).  Pairs of steps run as one captured CUDA graph on
 * the batch's stream (the side stream's launches are captured with it).
 * In-place lattices (TLB_INPLACE) cannot be members.  Members keep their
 * own workspaces; the batch workspace holds the device descriptors and work
 * lists.  Not in the paper: it serves many independent simulations.
 *
 * tlb_batch_workspace_bytes: bytes for up to max_lattices members, max_tiles
 * tiles (sum of tlb_batch_tiles_needed over the members) and max_wall_nodes
 * (sum of tlb_wall_nodes).  tlb_batch_create: the stream must not be the
 * legacy default stream.  tlb_batch_add: the lattice must have the batch's
 * precision and device and not belong to another batch; its own stream is
 * synchronized; while it is a member, tlb_step on it returns TLB_ESTATE.
 * tlb_batch_remove synchronizes the batch stream.  tlb_batch_step advances
 * every member n steps, asynchronously.  tlb_batch_config sets the tile shape
 * (threads 64 or 128; row segments rows_small for members with ny <=
 * small_ny, rows_large otherwise).
 *
 * tlb_batch_tune times 8 candidate shapes on the batch's own members,
 * trial_steps + 2 trial steps each, keeps the fastest and reports {threads,
 * rows_small, rows_large, small_ny} and its time per step.  It leaves every
 * member's state as it was: each trial step reads the members' current
 * distributions and writes their spare buffer without making it current, and
 * the c_i u planes of Eq. 19 (the only state a step updates in place) are
 * saved to dev_scratch before the trials and restored after them.
 * dev_scratch: caller-owned device memory, 256-byte aligned, of at least
 * tlb_batch_tune_scratch_bytes(batch) bytes for the current members (the
 * library does not allocate it).  Synchronizes the batch stream.  TLB_ESTATE
 * for an empty batch or a member without state; TLB_ENOMEM for too little
 * scratch.  On failure the previous shape is kept. */
int64_t tlb_batch_workspace_bytes(int max_lattices, int64_t max_tiles, int64_t max_wall_nodes);
int64_t tlb_batch_tiles_needed(int nx, int ny);
int tlb_batch_create(int precision, int max_lattices, int64_t max_tiles, int64_t max_wall_nodes,
                     void *dev_workspace, int64_t ws_bytes, void *cuda_stream, tlb_batch **out);
int tlb_batch_add(tlb_batch *batch, tlb_lattice *lat);
int tlb_batch_remove(tlb_batch *batch, tlb_lattice *lat);
int tlb_batch_size(tlb_batch *batch);
int tlb_batch_step(tlb_batch *batch, int64_t n);
int tlb_batch_config(tlb_batch *batch, int threads, int rows_small, int rows_large, int small_ny);
int64_t tlb_batch_tune_scratch_bytes(tlb_batch *batch);
int tlb_batch_tune(tlb_batch *batch, int trial_steps, void *dev_scratch, int64_t scratch_bytes,
                   int out_config[4], double *out_ms_per_step);
void tlb_batch_destroy(tlb_batch *batch);

/* ---- D3Q19: the same model on a three-dimensional lattice ---------------
 * Sec. II.A states the model for D dimensions; these calls run it on the
 * D3Q19 velocity set (e_0 = 0; e_1..6 = +x, -x, +y, -y, +z, -z; e_7..18 the 12
 * face diagonals (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1),
 * (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1); weights 1/3,
 * 1/18, 1/36): Eqs. 1-20 with the Eq. 20 stencils over its 18 links, the
 * Eq. 42 wetting ghost on every link into a wetting solid (Eq. 43 otherwise),
 * half-way bounce-back (Eq. 44), BGK collision.  precision: TLB_FP64 (FP64
 * storage and arithmetic) or TLB_FP32 (FP32 storage and arithmetic, the rest
 * populations as float pairs hi + lo so that each component's mass is
 * conserved to round-off, as for the 2D FP32 storage); TLB_EINVAL otherwise.
 * Body force G = rho (gx, gy, 0).  Node arrays are [nz][ny][nx], x fastest;
 * nx, ny, nz >= 3 and nx*ny*nz < 2^31 (TLB_EINVAL otherwise).
 * edges[6] = {x-, x+, y-, y+, z-, z+}, each TLB_EDGE_PERIODIC, _WETTING or
 * _NEUTRAL (no lid); a periodic edge needs a periodic opposite edge; at a
 * site outside in several axes the first outside axis in x, y, z order
 * whose edge is not periodic decides.  Mask values as for tlb_set_geometry.
 * One step is three launches on the lattice's stream (order parameters into
 * two planes, chemical potentials into two planes, then the fused update and
 * push; equal densities and viscosities in the three fluids select an update
 * without the terms that then vanish).  Ownership and errors as for the 2D calls; the library allocates no
 * device memory (workspace from tlb3_workspace_bytes, 256-byte aligned).
 *   tlb3_set_params: TLB_EINVAL as tlb_set_params, and for collision != 0 or
 *     lid_u != 0.
 *   tlb3_set_fields: host arrays of nx*ny*nz (p may be NULL); f = f^eq(c,
 *     mu(c), u), g = g^eq(p, rho, u), c_i u stored; synchronizes.
 *   tlb3_step: n steps, asynchronous.  tlb3_sync: waits for the stream.
 *   tlb3_read_fields: field_mask bits 0..10 select c1, c2, c3, rho, ux, uy,
 *     uz, p, mu1, mu2, mu3 (in that order) as FP64 planes of nx*ny*nz;
 *     synchronizes.
 *   tlb3_read_state: 63 FP64 planes: f^1_k, f^2_k, g_k (k = 0..18), then c1
 *     ux, c1 uy, c1 uz, c2 ux, c2 uy, c2 uz of the previous step (Eq. 19); zero on solid nodes.
 *   tlb3_diagnostics: FP64 mass totals of c1, c2, c3 over fluid nodes and
 *     the non-finite count (TLB_EUNSTABLE if any). */
typedef struct tlb3_lattice tlb3_lattice;
int64_t tlb3_workspace_bytes(int nx, int ny, int nz, int precision);
int tlb3_create(int nx, int ny, int nz, int precision, const int32_t edges[6], void *dev_workspace, int64_t ws_bytes,
                void *cuda_stream, tlb3_lattice **out);
int tlb3_set_geometry(tlb3_lattice *lat, const uint8_t *host_mask);
int tlb3_set_params(tlb3_lattice *lat, const tlb_params *params);
int tlb3_set_fields(tlb3_lattice *lat, const double *c1, const double *c2, const double *ux, const double *uy,
                    const double *uz, const double *p);
int tlb3_step(tlb3_lattice *lat, int64_t n);
int tlb3_sync(tlb3_lattice *lat);
int tlb3_read_fields(tlb3_lattice *lat, uint32_t field_mask, double *host_out);
int tlb3_read_state(tlb3_lattice *lat, double *host_out);
int tlb3_diagnostics(tlb3_lattice *lat, tlb_diag *out);
/* Per-kernel timing with CUDA events on the lattice's stream, as tlb_profile:
 * ms[0..2] and launches[0..2] for the order-parameter, chemical-potential and
 * update launches of the steps run since tlb3_profile(lat, 1).  With FP32
 * storage and equal densities and viscosities the update forms the chemical
 * potentials itself (no second launch): ms[1] is then the empty interval. */
int tlb3_profile(tlb3_lattice *lat, int enable);
int tlb3_profile_read(tlb3_lattice *lat, double ms[3], int64_t launches[3]);
void tlb3_destroy(tlb3_lattice *lat);

/* Allocation-free variant of the tlb_diagnostics reduction.  The paper has
 * no counterpart: this exists for callers that cannot allocate device memory
 * where they need the totals (code living in a fixed arena it does not own,
 * or a loop that must not stall on an allocation).  It reads the lattice's
 * current state, writes 4 doubles {sum c1, sum c2, sum c3, non-finite count}
 * to dev_out (caller-owned device memory) asynchronously on the lattice's
 * stream, and keeps its partial sums in a static 32 KiB device array that
 * every GPU loading the library holds until process exit.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   - Limit: lattices of at most 16,777,216 nodes (4096 x 4096); larger ones
 *     get TLB_EINVAL with a message (use tlb_diagnostics for those).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Each device holds its own copy of the array, and every call on that
 *     device shares it: calls on the same device whose work overlaps (for
 *     example on different streams) race and may return wrong totals; order
 *     them on one stream.  Calls on different devices do not interfere.
 *     Each call overwrites every partial it reads, so nothing needs
 *     clearing.
 * TLB_ESTATE before set_fields; TLB_EINVAL for a null dev_out. */
int tlb_diagnostics_noalloc(tlb_lattice *lat, double *dev_out);

/* Arithmetic ceiling of the FP64 (or FP32) update, for its roofline.  The
 * paper has no counterpart; it is a measurement aid.  Launches a kernel of
 * independent fused-multiply-add chains on every SM of the current device
 * (one warm-up launch, then the fastest of five, timed with CUDA events on a
 * stream the call creates and destroys) and returns the achieved rate in
 * *tflops (an FMA counts as 2 flops) and the kernel time in *ms (may be
 * NULL).  precision: TLB_FP64 or TLB_FP32.  dev_sink: caller-owned device
 * memory of at least 8 bytes; the kernel writes it only in a case that does
 * not occur, so that the chains are not optimised away.  Synchronizes.
 * TLB_EINVAL for a null pointer or another precision. */
int tlb_fma_peak(int precision, void *dev_sink, double *tflops, double *ms);

/* Release the host handle (the workspace stays the caller's). */
void tlb_destroy(tlb_lattice *lat);

/* Message of the last failed call on this thread ("" if none). */
const char *tlb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TLBM_H */

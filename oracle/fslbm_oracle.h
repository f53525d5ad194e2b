/*
 * Plain FP64 CPU oracle of the free-surface lattice Boltzmann (FSLBM) time step
 * of Schwarzmeier & Ruede, "Analysis and comparison of boundary condition
 * variants in the free-surface lattice Boltzmann method" (arXiv 2207.13962).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path (the
 * CUDA library under paper_2207_13962_gb300/) never calls it and shares no
 * code, header or table with it.
 *
 * Every routine is a literal, single-threaded, cell-by-cell restatement of the
 * paper's Section 2 (LBM, Eqs. nm-lbm-*) and Section 3 (boundary-condition
 * variants, Eqs. fsbcv-*), with the readings of ambiguous passages listed in
 * the C file's header comment.
 */
#ifndef FSLBM_ORACLE_H
#define FSLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc orc;

/* q = 19 or 27 for whole-domain runs (9 is accepted only by the unit helpers).
 * per_x, per_y, per_z: boundary of each axis, 0 no-slip walls, 1 periodic,
 * 2 free-slip walls.  collision: 0 SRT, 1 TRT.  variant: 1 NBRC, 2 NBKC,
 * 3 OM, 4 OM3.  om3_fallback: 1 NBRC or 2 NBKC.  bubble_model: 0 constant
 * p_v0, 1 per-bubble volume tracking.  cs: Smagorinsky constant (0: no LES).
 * Returns NULL on bad arguments. */
orc* orc_create(int nx, int ny, int nz, int per_x, int per_y, int per_z, int q,
                int collision, int variant, int om3_fallback, int bubble_model,
                double omega, double trt_magic, double gx, double gy, double gz,
                double sigma, double eps_phi, double p_v0, double cs);
void orc_destroy(orc* o);

/* fill[N], flags[N] (0 gas 1 interface 2 liquid 3 obstacle), velocity[3N]
 * (component-major: ux[N] uy[N] uz[N]) or NULL, density[N] or NULL (=1).
 * Returns 0 on success, 1 on invalid input (closure broken, bad flag). */
int orc_init(orc* o, const double* fill, const unsigned char* flags,
             const double* velocity, const double* density);
void orc_step(orc* o, int n);
/* Bubble coalescence and segmentation (reading R24) every `every` steps
 * after init (0, the default: the labels of the initial state stay). */
void orc_set_bubble_relabel(orc* o, int every);
/* The same relabelling once, now (bubble model only). */
void orc_relabel_bubbles(orc* o);
long orc_steps_done(const orc* o);

/* Any pointer may be NULL.  pdf[q*N] direction-major post-collision PDFs. */
void orc_read(const orc* o, double* pdf, double* fill, unsigned char* flags,
              double* mass);
/* rho[N], u[3N] of each liquid/interface cell evaluated from its current
 * post-collision PDFs (rho = sum f*, rho u = sum c f* - F/2); 0 elsewhere. */
void orc_read_moments(const orc* o, double* rho, double* u);
/* Geometry of the current state (before the next step): nhat[3N], kappa[N]
 * (kappa only meaningful on interface cells), phis[N] smoothed fill. */
void orc_geometry(orc* o, double* nhat, double* kappa, double* phis);
/* Bubble table: returns the number of bubbles; fills up to cap entries. */
int orc_bubbles(const orc* o, double* volume, double* pressure, int* ids_cell,
                int cap);
/* Total liquid mass: sum of rho over liquid cells + m over interface cells. */
double orc_total_mass(const orc* o);

/* ---- unit helpers (lattice-level, no domain) ---- */
/* Direction table: c[3*q] ints, w[q], opp[q]. Returns 0 or 1 on bad q. */
int orc_lattice(int q, int* c, double* w, int* opp);
void orc_feq(int q, double rho, const double* u, double* feq);
/* One collision of a single cell: fin[q] -> fout[q]; rho and u (with the
 * force shift) are returned in rho_u[4]. */
void orc_collide(int q, int collision, double omega, double trt_magic,
                 double cs, const double* g, const double* fin, double* fout,
                 double* rho_u);
/* Reconstruction set R of one interface cell: miss[q] (1 = PDF streams from a
 * gas cell), nhat[3]; recon[q] receives 1 for i in R. */
void orc_select(int q, int variant, int om3_fallback, const double* nhat,
                const int* miss, int* recon);
/* Free-surface BC (Eq. nm-fslbm-boundary-condition) on one cell:
 * fin[q] streamed PDFs (entries with recon[i] are overwritten),
 * fstar_x[q] post-collision PDFs of the cell itself. */
void orc_reconstruct(int q, const int* recon, double rho_g, const double* u,
                     const double* fstar_x, double* fin);
/* Geometry stencils on one 3x3x3 block b[(dx+1) + 3 (dy+1) + 9 (dz+1)]:
 * the K8-smoothed value at its centre (reading R16) and the raw
 * Parker-Youngs gradient there (Eq. nm-fslbm-normal, reading R17; n3[3],
 * not normalised).  The step's geometry evaluates every cell with them. */
double orc_k8_smooth(const double* block27);
void orc_py_gradient(const double* block27, double* n3);

/* ---- observables on a flags array (caller order x + nx (y + ny z)) ---- */
/* Seed-fill front of the layer z = layer (reading R23): front[nx*ny]
 * (optional) gets 1 for front cells; stats[4] = count, min, max and mean of
 * their radius about (xc, yc).  Returns 0, or 1 on bad arguments. */
int orc_seed_fill_front(int nx, int ny, int nz, int per_x, int per_y, const unsigned char* flags,
                        int layer, double xc, double yc, unsigned char* front, double* stats);

#ifdef __cplusplus
}
#endif
#endif

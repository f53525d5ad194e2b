/*
 * Plain FP64 CPU oracle of the FSLBM time step (arXiv 2207.13962).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  Single thread,
 * whole-grid loops over cells, neighbour loops in direction order i = 0..q-1.
 * Compile without floating-point contraction (-ffp-contract=off) so that each
 * expression rounds exactly as written.
 *
 * Passages followed (section / equation of the paper):
 *   Sec. 2.1  lattice, Eq. nm-lbm-collision, nm-lbm-streaming,
 *             nm-lbm-collision-operator (SRT), nm-lbm-equilibrium,
 *             nm-lbm-density, nm-lbm-velocity (force shift), nm-lbm-force-guo,
 *             no-slip bounce-back.
 *   Sec. 2.2  cell types, Eq. nm-fslbm-mass, nm-fslbm-mass-flux, conversion
 *             thresholds, conflict rule, Eq. nm-fslbm-excess-mass, Thuerey
 *             flux adjustment, PDF initialisation of new interface cells,
 *             Eq. nm-fslbm-boundary-condition, nm-fslbm-pressure-gas,
 *             nm-fslbm-pressure-volume, nm-fslbm-pressure-laplace, curvature
 *             by FDM, Eq. nm-fslbm-normal (Parker-Youngs), K8 smoothing.
 *   Sec. 3    sets K/R of the variants: Eq. fsbcv-nbrc, fsbcv-nbkc,
 *             fsbcv-om-sets, fsbcv-om3.
 *
 * Readings taken where the paper is silent, garbled or inconsistent:
 *   R1  BGK sign: Omega_i = -(f_i - f_i^eq)/tau (relaxation towards f^eq).
 *   R2  c_s^2 = 1/3 (p0 = c_s^2 rho0 = 1/3).
 *   R3  n = grad(phi~) points into the liquid; NBRC/NBKC use n.c_i >= 0 / > 0.
 *   R4  NBRC/NBKC also reconstruct every missing PDF (i in G-) outside the
 *       normal-based set.
 *   R5  ties: a direction with |n^.c_i| <= 2^-20 on the normalised normal
 *       counts as n.c_i = 0 (Appendix A assumes that only c_0 ties; at mirror
 *       planes of the interface a component of n^ is zero in exact
 *       arithmetic and rounding-sized otherwise, so an exact sign test would
 *       decide by rounding noise).  NBRC reconstructs ties, NBKC only missing
 *       ones.
 *   R6  OM3 falls back to NBKC (selectable NBRC) when |G-| < 3.
 *   R7  gas density rho^G = 3 (p^V + sigma kappa), kappa = -div(n^) with n^
 *       pointing into the liquid (sum of principal curvatures).
 *   R8  the density and velocity of a cell at time t are evaluated from its
 *       post-collision PDFs: rho = sum f*_i, rho u = sum c_i f*_i - F/2 (equal
 *       to the moments of its last collision, which conserves rho and adds F
 *       to the momentum).  The BC uses this u(x,t); new interface cells
 *       average these values over their neighbours at t+1.
 *   R9  force density F = rho g, not weighted by the fill level.
 *   R10 TRT: omega+ = omega, 1/omega- = 1/2 + Lambda/(1/omega+ - 1/2); Guo
 *       source split into symmetric (omega+) and antisymmetric (omega-) parts.
 *   R11 mass flux uses post-collision PDFs, fill levels and flags of time t.
 *   R12 Thuerey classes: NF (no liquid nb), NE (no gas nb), else STD;
 *       interface-interface flux table (see mass_flux()).
 *   R13 conversion conflicts: an interface cell marked for gas stays
 *       interface when a neighbour is marked for liquid.
 *   R14 new interface cells from gas: f* = f^eq(mean rho, mean u) over
 *       neighbours that are liquid or old interface after conversion.
 *   R15 excess mass m_ex = m - rho (to liquid) or m (to gas), split evenly over
 *       neighbours that are interface after conversion; no receiver -> the
 *       conversion is deferred, and the cell stays interface with its mass
 *       (it was not counted as a receiver, so it takes no share).  Receivers
 *       sum shares in direction order.
 *   R16 K8 kernel (1 - r^2/4)^4 on the 3x3x3 block (zero at r >= 2), weights
 *       normalised by their sum; obstacle / out-of-domain -> centre value.
 *   R17 Parker-Youngs weights 4 (face centre), 2 (edge), 1 (corner); obstacle
 *       neighbour -> centre value; n = 0 -> n^ = 0.
 *   R18 kappa = -(1/2) sum_a (n^_a(x+e_a) - n^_a(x-e_a)); obstacle -> centre.
 *   R19 bubbles: connected gas components (lattice neighbourhood), labelled in
 *       order of their lowest cell index; interface cells take the lowest id
 *       of their gas neighbours; volume V = #gas + sum over interface (1-phi)
 *       accumulated in fixed point with 2^-32 resolution.
 *   R20 cells outside a non-periodic boundary act as no-slip obstacle cells,
 *       unless the face is a free-slip wall (R22).
 *   R21 Smagorinsky LES (Sec. 2.1, Eqs. nm-lbm-turbulence-viscosity to
 *       nm-lbm-turublence-relaxation-time): tau = tau0 + tau_t with
 *       tau_t = (sqrt(tau0^2 + 2 sqrt(2) (C_S dx)^2 Qbar / (rho c_s^4)) - tau0)/2,
 *       the printed form "1/2 sqrt(...) - tau0" read with the 1/2 over both
 *       terms (as printed, tau would be tau0/2 at zero strain);
 *       Qbar = sqrt(2 sum_ab Q_ab Q_ab), Q_ab = sum_i c_ia c_ib (f_i - f^eq_i)
 *       from the PDFs entering the collision; dx_LES = 1.  TRT keeps its
 *       magic parameter: omega- follows from the adjusted omega+.  The Guo
 *       prefactors use the adjusted rates.
 *   R22 free-slip faces (Sec. 2.1: PDFs reflected specularly, the normal
 *       component reversed): a PDF whose pull source lies across a free-slip
 *       face comes from the mirror cell, whose coordinates along those axes
 *       are the cell's own, with the direction's components along them
 *       reversed.  If the mirror cell is gas, the PDF is missing and the
 *       free-surface BC reconstructs it (Sec. 2.2, the paragraph after
 *       Eq. nm-fslbm-boundary-condition); if it is an obstacle, it bounces
 *       back.  The mass exchange (Eq. nm-fslbm-mass-flux) of an interface
 *       cell runs over these wall links like over lattice links, so the
 *       masses of interface cells keep track of the PDFs that move between
 *       cells along a wall.
 *   R23 seed-fill front (Sec. 4.3, cylindrical dam break: the front radius
 *       is taken over the interface cells that a seed fill started at a
 *       domain boundary reaches): the fill runs in one z-layer, through the
 *       cells that are gas or obstacle, over in-plane face neighbours
 *       (across periodic faces too), seeded with every such cell on the
 *       layer's edge (x = 0, nx-1 or y = 0, ny-1).  A front cell is an
 *       interface cell of the layer with a reached gas cell among its
 *       in-plane face neighbours.  Its radius is the distance of its cell
 *       centre (x + 1/2, y + 1/2) to the given centre (xc, yc).
 *   R24 bubble coalescence and segmentation (Sec. 2.2 cites a bubble model
 *       that follows them, without the algorithm): every K steps (K = 0, the
 *       default, keeps the labels of the initial state) the bubbles are
 *       relabelled from the current flags as at init (R19), and each old
 *       bubble's gas, whose amount is p^V V = p^V(0) V0, is divided over the
 *       new bubbles in proportion to the fixed-point volume of its cells that
 *       each holds (a bubble none of whose cells is in a new bubble has
 *       vanished with its gas).  Merging bubbles so keep the sum of p^V V
 *       (Boyle's law at equal temperature), and the parts of a split bubble
 *       keep its pressure.  Cells without an old id (gas or interface cells
 *       outside every bubble, which the step gives the pressure p^V(0)) bring
 *       their volume at p^V(0), so a new gas region starts at p^V(0).
 *
 * R8 has one exception: a gas cell that becomes interface gets f^eq of the
 * mean density and velocity of its neighbours (R14), with no collision, so
 * R8 evaluates its velocity as that mean minus g/2 until its first collision.
 */
#include "fslbm_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { GAS = 0, IFACE = 1, LIQ = 2, OBST = 3 };
enum { STD = 0, NF = 1, NE = 2 };
enum { C_NONE = 0, C_TOL = 1, C_TOG = 2 };

/* ------------------------------------------------------------------ lattices */
/* Direction order: rest, 6 faces, 12 edges, 8 corners; i odd/even pairs are
 * opposite (opp(i) = i+1 for odd i, i-1 for even i > 0). */
static const int C27[27][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},   {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1},  {1, 1, 1},
    {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1},
    {-1, 1, 1},  {1, -1, -1}};
static const int C9[9][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},
                             {0, 1, 0},  {0, -1, 0}, {1, 1, 0},
                             {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

typedef struct {
  int q;
  int c[27][3];
  double w[27];
  int opp[27];
} lattice;

static int make_lattice(int q, lattice* L) {
  int i;
  if (q != 9 && q != 19 && q != 27) return 1;
  L->q = q;
  for (i = 0; i < q; ++i) {
    const int* ci = (q == 9) ? C9[i] : C27[i];
    int n2 = ci[0] * ci[0] + ci[1] * ci[1] + ci[2] * ci[2];
    L->c[i][0] = ci[0];
    L->c[i][1] = ci[1];
    L->c[i][2] = ci[2];
    L->opp[i] = (i == 0) ? 0 : ((i % 2 == 1) ? i + 1 : i - 1);
    if (q == 9) {
      L->w[i] = (n2 == 0) ? 4.0 / 9.0 : (n2 == 1) ? 1.0 / 9.0 : 1.0 / 36.0;
    } else if (q == 19) {
      L->w[i] = (n2 == 0) ? 1.0 / 3.0 : (n2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
    } else {
      L->w[i] = (n2 == 0)   ? 8.0 / 27.0
                : (n2 == 1) ? 2.0 / 27.0
                : (n2 == 2) ? 1.0 / 54.0
                            : 1.0 / 216.0;
    }
  }
  return 0;
}

/* Index of the direction (cx, cy, cz) in L, -1 if absent. */
static int dir_of(const lattice* L, int cx, int cy, int cz) {
  int i;
  for (i = 0; i < L->q; ++i)
    if (L->c[i][0] == cx && L->c[i][1] == cy && L->c[i][2] == cz) return i;
  return -1;
}

int orc_lattice(int q, int* c, double* w, int* opp) {
  lattice L;
  int i;
  if (make_lattice(q, &L)) return 1;
  for (i = 0; i < q; ++i) {
    if (c) {
      c[3 * i] = L.c[i][0];
      c[3 * i + 1] = L.c[i][1];
      c[3 * i + 2] = L.c[i][2];
    }
    if (w) w[i] = L.w[i];
    if (opp) opp[i] = L.opp[i];
  }
  return 0;
}

/* --------------------------------------------------------- LBM cell algebra */
/* Eq. nm-lbm-equilibrium with c_s^2 = 1/3 (R2):
 * f_i^eq = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u). */
static double feq_i(const lattice* L, int i, double rho, double ux, double uy,
                    double uz) {
  double cu = (double)L->c[i][0] * ux + (double)L->c[i][1] * uy +
              (double)L->c[i][2] * uz;
  double usq = ux * ux + uy * uy + uz * uz;
  double t = 1.0 + 3.0 * cu;
  t = t + 4.5 * cu * cu;
  t = t - 1.5 * usq;
  return L->w[i] * rho * t;
}

void orc_feq(int q, double rho, const double* u, double* feq) {
  lattice L;
  int i;
  if (make_lattice(q, &L)) return;
  for (i = 0; i < q; ++i) feq[i] = feq_i(&L, i, rho, u[0], u[1], u[2]);
}

/* Guo source without the (1 - omega/2) prefactor (Eq. nm-lbm-force-guo):
 * w_i [ 3 (c_i - u).F + 9 (c_i.u)(c_i.F) ]. */
static double guo_i(const lattice* L, int i, double ux, double uy, double uz,
                    double Fx, double Fy, double Fz) {
  double cx = L->c[i][0], cy = L->c[i][1], cz = L->c[i][2];
  double cu = cx * ux + cy * uy + cz * uz;
  double cF = cx * Fx + cy * Fy + cz * Fz;
  double uF = ux * Fx + uy * Fy + uz * Fz;
  double t = 3.0 * (cF - uF) + 9.0 * cu * cF;
  return L->w[i] * t;
}

/* Moments of streamed PDFs: rho (Eq. nm-lbm-density), u with the force shift
 * u = j/rho + g/2 (Eq. nm-lbm-velocity with F = rho g, R9). */
static void moments(const lattice* L, const double* f, const double* g,
                    double* rho, double* u) {
  double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  int i;
  for (i = 0; i < L->q; ++i) r = r + f[i];
  for (i = 0; i < L->q; ++i) {
    if (L->c[i][0] != 0) jx = jx + (double)L->c[i][0] * f[i];
  }
  for (i = 0; i < L->q; ++i) {
    if (L->c[i][1] != 0) jy = jy + (double)L->c[i][1] * f[i];
  }
  for (i = 0; i < L->q; ++i) {
    if (L->c[i][2] != 0) jz = jz + (double)L->c[i][2] * f[i];
  }
  *rho = r;
  u[0] = jx / r + 0.5 * g[0];
  u[1] = jy / r + 0.5 * g[1];
  u[2] = jz / r + 0.5 * g[2];
}

/* Density and velocity of a cell from its post-collision PDFs (R8):
 * rho = sum f*_i, u = (sum c_i f*_i)/rho - g/2. */
static void post_moments(const lattice* L, const double* f, long stride,
                         const double* g, double* rho, double* u) {
  double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  int i;
  for (i = 0; i < L->q; ++i) r = r + f[i * stride];
  for (i = 0; i < L->q; ++i) {
    if (L->c[i][0] != 0) jx = jx + (double)L->c[i][0] * f[i * stride];
  }
  for (i = 0; i < L->q; ++i) {
    if (L->c[i][1] != 0) jy = jy + (double)L->c[i][1] * f[i * stride];
  }
  for (i = 0; i < L->q; ++i) {
    if (L->c[i][2] != 0) jz = jz + (double)L->c[i][2] * f[i * stride];
  }
  *rho = r;
  u[0] = jx / r - 0.5 * g[0];
  u[1] = jy / r - 0.5 * g[1];
  u[2] = jz / r - 0.5 * g[2];
}

/* Relaxation rate adjusted by the Smagorinsky model (R21) from the
 * non-equilibrium part of the PDFs entering the collision. */
static double les_omega(const lattice* L, double omega, double cs,
                        const double* fin, const double* feq, double rho) {
  double qxx = 0.0, qyy = 0.0, qzz = 0.0, qxy = 0.0, qxz = 0.0, qyz = 0.0;
  double q2, qbar, tau0, tau;
  int i;
  for (i = 0; i < L->q; ++i) {
    double cx = L->c[i][0], cy = L->c[i][1], cz = L->c[i][2];
    double d = fin[i] - feq[i];
    qxx = qxx + cx * cx * d;
    qyy = qyy + cy * cy * d;
    qzz = qzz + cz * cz * d;
    qxy = qxy + cx * cy * d;
    qxz = qxz + cx * cz * d;
    qyz = qyz + cy * cz * d;
  }
  q2 = qxx * qxx + qyy * qyy + qzz * qzz + 2.0 * (qxy * qxy + qxz * qxz + qyz * qyz);
  qbar = sqrt(2.0 * q2);
  tau0 = 1.0 / omega;
  tau = 0.5 * (tau0 + sqrt(tau0 * tau0 + 2.0 * sqrt(2.0) * (cs * cs) * qbar /
                                               (rho * (1.0 / 9.0))));
  return 1.0 / tau;
}

/* Collision (Eq. nm-lbm-collision with R1, R9, R10; LES R21 when cs > 0). */
static void collide(const lattice* L, int collision, double omega,
                    double trt_magic, double cs, const double* g,
                    const double* fin, double* fout, double* rho_out,
                    double* u_out) {
  double rho, u[3];
  double feq[27], src[27];
  int i;
  moments(L, fin, g, &rho, u);
  {
    double Fx = rho * g[0], Fy = rho * g[1], Fz = rho * g[2];
    for (i = 0; i < L->q; ++i) {
      feq[i] = feq_i(L, i, rho, u[0], u[1], u[2]);
      src[i] = guo_i(L, i, u[0], u[1], u[2], Fx, Fy, Fz);
    }
  }
  if (cs > 0.0) omega = les_omega(L, omega, cs, fin, feq, rho);
  if (collision == 0) {
    double pref = 1.0 - 0.5 * omega;
    for (i = 0; i < L->q; ++i)
      fout[i] = fin[i] - omega * (fin[i] - feq[i]) + pref * src[i];
  } else {
    double om_p = omega;
    double om_m = 1.0 / (0.5 + trt_magic / (1.0 / om_p - 0.5));
    double pref_p = 1.0 - 0.5 * om_p;
    double pref_m = 1.0 - 0.5 * om_m;
    for (i = 0; i < L->q; ++i) {
      int j = L->opp[i];
      double fp = 0.5 * (fin[i] + fin[j]);
      double fm = 0.5 * (fin[i] - fin[j]);
      double ep = 0.5 * (feq[i] + feq[j]);
      double em = 0.5 * (feq[i] - feq[j]);
      double sp = 0.5 * (src[i] + src[j]);
      double sm = 0.5 * (src[i] - src[j]);
      fout[i] = fin[i] - om_p * (fp - ep) - om_m * (fm - em) + pref_p * sp +
                pref_m * sm;
    }
  }
  *rho_out = rho;
  u_out[0] = u[0];
  u_out[1] = u[1];
  u_out[2] = u[2];
}

void orc_collide(int q, int collision, double omega, double trt_magic,
                 double cs, const double* g, const double* fin, double* fout,
                 double* rho_u) {
  lattice L;
  double rho, u[3];
  if (make_lattice(q, &L)) return;
  collide(&L, collision, omega, trt_magic, cs, g, fin, fout, &rho, u);
  rho_u[0] = rho;
  rho_u[1] = u[0];
  rho_u[2] = u[1];
  rho_u[3] = u[2];
}

/* ------------------------------------------------- boundary-condition sets */
static double ndot(const lattice* L, int i, const double* n) {
  return (double)L->c[i][0] * n[0] + (double)L->c[i][1] * n[1] +
         (double)L->c[i][2] * n[2];
}

/* Width of the tie band of reading R5: |n^.c_i| <= TIE counts as a tie. */
#define TIE 0x1p-20

/* Sets R of Sec. 3 (Eqs. fsbcv-nbrc, fsbcv-nbkc, fsbcv-om-sets, fsbcv-om3)
 * with readings R3-R6: NBRC takes n.c_i >= 0 (ties included), NBKC
 * n.c_i > 0 (ties excluded), both with every missing PDF. */
static void select_R(const lattice* L, int variant, int om3_fallback,
                     const double* nhat, const int* miss, int* recon) {
  int i, nmiss = 0, v = variant;
  for (i = 0; i < L->q; ++i) nmiss += miss[i] ? 1 : 0;
  if (v == 4) v = (nmiss >= 3) ? 3 : om3_fallback;
  for (i = 0; i < L->q; ++i) {
    int r = miss[i] ? 1 : 0;
    double d = ndot(L, i, nhat);
    if (v == 1 && d >= -TIE) r = 1;
    if (v == 2 && d > TIE) r = 1;
    recon[i] = r;
  }
}

void orc_select(int q, int variant, int om3_fallback, const double* nhat,
                const int* miss, int* recon) {
  lattice L;
  if (make_lattice(q, &L)) return;
  select_R(&L, variant, om3_fallback, nhat, miss, recon);
}

/* Eq. nm-fslbm-boundary-condition:
 * f_i(x) = f_i^eq(rho^G,u) + f_ibar^eq(rho^G,u) - f*_ibar(x). */
static void reconstruct(const lattice* L, const int* recon, double rho_g,
                        const double* u, const double* fstar_x, double* fin) {
  int i;
  for (i = 0; i < L->q; ++i) {
    if (recon[i]) {
      int j = L->opp[i];
      fin[i] = (feq_i(L, i, rho_g, u[0], u[1], u[2]) +
                feq_i(L, j, rho_g, u[0], u[1], u[2])) -
               fstar_x[j];
    }
  }
}

void orc_reconstruct(int q, const int* recon, double rho_g, const double* u,
                     const double* fstar_x, double* fin) {
  lattice L;
  if (make_lattice(q, &L)) return;
  reconstruct(&L, recon, rho_g, u, fstar_x, fin);
}

/* ------------------------------------------------------------------ domain */
struct orc {
  lattice L;
  int nx, ny, nz, per[3], slip[3];
  double cs; /* Smagorinsky constant, 0: no LES */
  long N;
  int collision, variant, om3_fallback, bubble_model;
  double omega, trt_magic, g[3], sigma, eps, pv0;
  double* f;    /* post-collision PDFs f*(t), direction-major [q][N] */
  double* fn;   /* next buffer */
  unsigned char* flag;
  double *phi, *m;
  double* rho;               /* density of this step's collision (scratch) */
  int* bid;                  /* bubble id (gas/interface), -1 otherwise */
  int nb;                    /* number of bubbles */
  int relabel_every;         /* steps between bubble relabellings (R24), 0: never */
  double *V0, *pV;           /* per bubble */
  long step;
  /* scratch */
  double *phis, *nhat, *kappa, *rhog;
  unsigned char *cls, *mark, *conv, *nflag, *isnew, *dfr;
  double *phin, *mn, *share;
};

/* Neighbour of cell (x,y,z) at offset d; -1 outside a non-periodic boundary. */
static long nbr(const orc* o, int x, int y, int z, int dx, int dy, int dz) {
  int X = x + dx, Y = y + dy, Z = z + dz;
  if (X < 0 || X >= o->nx) {
    if (!o->per[0]) return -1;
    X = (X + o->nx) % o->nx;
  }
  if (Y < 0 || Y >= o->ny) {
    if (!o->per[1]) return -1;
    Y = (Y + o->ny) % o->ny;
  }
  if (Z < 0 || Z >= o->nz) {
    if (!o->per[2]) return -1;
    Z = (Z + o->nz) % o->nz;
  }
  return (long)X + (long)o->nx * ((long)Y + (long)o->ny * (long)Z);
}

static void coords(const orc* o, long c, int* x, int* y, int* z) {
  *x = (int)(c % o->nx);
  *y = (int)((c / o->nx) % o->ny);
  *z = (int)(c / ((long)o->nx * o->ny));
}

/* flag of a neighbour, OBST outside the domain (R20) */
static int nflag_of(const orc* o, long n) { return n < 0 ? OBST : o->flag[n]; }

/* Pull source of direction k of cell (x, y, z) (Eq. nm-lbm-streaming): the
 * cell x - c_k, whose PDF k arrives (*j = k).  Across a periodic face the
 * source wraps; across a free-slip face it is the mirror image (R22): the
 * coordinate along that axis stays the cell's own and the arriving PDF is
 * the one with that component of c_k reversed.  -1 across a no-slip face. */
static long pull_source(const orc* o, int x, int y, int z, int k, int* j) {
  const lattice* L = &o->L;
  int p[3], c[3], n[3], a;
  p[0] = x;
  p[1] = y;
  p[2] = z;
  n[0] = o->nx;
  n[1] = o->ny;
  n[2] = o->nz;
  for (a = 0; a < 3; ++a) {
    int s = p[a] - L->c[k][a];
    c[a] = L->c[k][a];
    if (s < 0 || s >= n[a]) {
      if (o->per[a]) {
        s = (s + n[a]) % n[a];
      } else if (o->slip[a]) {
        s = p[a];
        c[a] = -c[a];
      } else {
        return -1;
      }
    }
    p[a] = s;
  }
  *j = dir_of(L, c[0], c[1], c[2]);
  return (long)p[0] + (long)o->nx * ((long)p[1] + (long)o->ny * (long)p[2]);
}

orc* orc_create(int nx, int ny, int nz, int per_x, int per_y, int per_z, int q,
                int collision, int variant, int om3_fallback, int bubble_model,
                double omega, double trt_magic, double gx, double gy, double gz,
                double sigma, double eps_phi, double p_v0, double cs) {
  orc* o;
  long N;
  if (nx < 1 || ny < 1 || nz < 1 || (q != 19 && q != 27)) return NULL;
  if (per_x < 0 || per_x > 2 || per_y < 0 || per_y > 2 || per_z < 0 || per_z > 2) return NULL;
  if (!(cs >= 0.0)) return NULL;
  if (variant < 1 || variant > 4 || (om3_fallback != 1 && om3_fallback != 2))
    return NULL;
  o = (orc*)calloc(1, sizeof(orc));
  if (!o) return NULL;
  make_lattice(q, &o->L);
  o->nx = nx;
  o->ny = ny;
  o->nz = nz;
  o->per[0] = per_x == 1;
  o->per[1] = per_y == 1;
  o->per[2] = per_z == 1;
  o->slip[0] = per_x == 2;
  o->slip[1] = per_y == 2;
  o->slip[2] = per_z == 2;
  o->cs = cs;
  N = (long)nx * ny * nz;
  o->N = N;
  o->collision = collision;
  o->variant = variant;
  o->om3_fallback = om3_fallback;
  o->bubble_model = bubble_model;
  o->omega = omega;
  o->trt_magic = trt_magic;
  o->g[0] = gx;
  o->g[1] = gy;
  o->g[2] = gz;
  o->sigma = sigma;
  o->eps = eps_phi;
  o->pv0 = p_v0;
  o->f = (double*)calloc((size_t)q * N, sizeof(double));
  o->fn = (double*)calloc((size_t)q * N, sizeof(double));
  o->flag = (unsigned char*)calloc(N, 1);
  o->phi = (double*)calloc(N, sizeof(double));
  o->m = (double*)calloc(N, sizeof(double));
  o->rho = (double*)calloc(N, sizeof(double));
  o->bid = (int*)calloc(N, sizeof(int));
  o->phis = (double*)calloc(N, sizeof(double));
  o->nhat = (double*)calloc(3 * N, sizeof(double));
  o->kappa = (double*)calloc(N, sizeof(double));
  o->rhog = (double*)calloc(N, sizeof(double));
  o->cls = (unsigned char*)calloc(N, 1);
  o->mark = (unsigned char*)calloc(N, 1);
  o->conv = (unsigned char*)calloc(N, 1);
  o->nflag = (unsigned char*)calloc(N, 1);
  o->isnew = (unsigned char*)calloc(N, 1);
  o->dfr = (unsigned char*)calloc(N, 1);
  o->phin = (double*)calloc(N, sizeof(double));
  o->mn = (double*)calloc(N, sizeof(double));
  o->share = (double*)calloc(N, sizeof(double));
  if (!o->f || !o->fn || !o->flag || !o->phi || !o->m || !o->rho ||
      !o->bid || !o->phis || !o->nhat || !o->kappa || !o->rhog || !o->cls ||
      !o->mark || !o->conv || !o->nflag || !o->isnew || !o->dfr || !o->phin || !o->mn ||
      !o->share) {
    orc_destroy(o);
    return NULL;
  }
  return o;
}

void orc_destroy(orc* o) {
  if (!o) return;
  free(o->f);
  free(o->fn);
  free(o->flag);
  free(o->phi);
  free(o->m);
  free(o->rho);
  free(o->bid);
  free(o->V0);
  free(o->pV);
  free(o->phis);
  free(o->nhat);
  free(o->kappa);
  free(o->rhog);
  free(o->cls);
  free(o->mark);
  free(o->conv);
  free(o->nflag);
  free(o->isnew);
  free(o->dfr);
  free(o->phin);
  free(o->mn);
  free(o->share);
  free(o);
}

/* Fixed-point bubble volume term (R19): round((1 - phi) * 2^32). */
static int64_t vol_fix(double one_minus_phi) {
  return (int64_t)llrint(one_minus_phi * 4294967296.0);
}

/* Bubble volumes V_b = #gas + sum_interface (1 - phi) (R19). */
static void bubble_volumes(const orc* o, double* V) {
  int64_t* acc = (int64_t*)calloc(o->nb > 0 ? o->nb : 1, sizeof(int64_t));
  long c;
  int b;
  for (c = 0; c < o->N; ++c) {
    b = o->bid[c];
    if (b < 0) continue;
    if (o->flag[c] == GAS)
      acc[b] += (int64_t)4294967296LL;
    else if (o->flag[c] == IFACE)
      acc[b] += vol_fix(1.0 - o->phi[c]);
  }
  for (b = 0; b < o->nb; ++b) V[b] = (double)acc[b] / 4294967296.0;
  free(acc);
}

/* Bubble labels of the current flags (R19): the connected gas components
 * (lattice neighbourhood, periodic wrap) numbered in the order of their
 * lowest cell index; an interface cell takes the lowest id among its gas
 * neighbours (-1 without one); every other cell -1.  Returns the count. */
static int label_bubbles(orc* o) {
  const lattice* L = &o->L;
  const long N = o->N;
  long c;
  int i, x, y, z, nb = 0;
  long* stack = (long*)malloc(sizeof(long) * (size_t)(N > 0 ? N : 1));
  for (c = 0; c < N; ++c) o->bid[c] = -1;
  for (c = 0; c < N; ++c) {
    long sp = 0;
    if (o->flag[c] != GAS || o->bid[c] >= 0) continue;
    o->bid[c] = nb;
    stack[sp++] = c;
    while (sp > 0) {
      long a = stack[--sp];
      coords(o, a, &x, &y, &z);
      for (i = 1; i < L->q; ++i) {
        long n = nbr(o, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
        if (n >= 0 && o->flag[n] == GAS && o->bid[n] < 0) {
          o->bid[n] = nb;
          stack[sp++] = n;
        }
      }
    }
    ++nb;
  }
  free(stack);
  for (c = 0; c < N; ++c) {
    int best = -1;
    if (o->flag[c] != IFACE) continue;
    coords(o, c, &x, &y, &z);
    for (i = 1; i < L->q; ++i) {
      long n = nbr(o, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
      if (n >= 0 && o->flag[n] == GAS && (best < 0 || o->bid[n] < best)) best = o->bid[n];
    }
    o->bid[c] = best;
  }
  return nb;
}

int orc_init(orc* o, const double* fill, const unsigned char* flags,
             const double* velocity, const double* density) {
  const lattice* L = &o->L;
  long N = o->N, c;
  int i, x, y, z;
  for (c = 0; c < N; ++c)
    if (flags[c] > OBST) return 1;
  memcpy(o->flag, flags, (size_t)N);
  /* closure: no liquid cell next to a gas cell */
  for (c = 0; c < N; ++c) {
    if (o->flag[c] != LIQ) continue;
    coords(o, c, &x, &y, &z);
    for (i = 1; i < L->q; ++i) {
      long n = nbr(o, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
      if (n >= 0 && o->flag[n] == GAS) return 1;
    }
  }
  for (c = 0; c < N; ++c) {
    double r = density ? density[c] : 1.0;
    double ux = velocity ? velocity[c] : 0.0;
    double uy = velocity ? velocity[N + c] : 0.0;
    double uz = velocity ? velocity[2 * N + c] : 0.0;
    int fl = o->flag[c];
    o->phi[c] = (fl == LIQ) ? 1.0 : (fl == IFACE) ? fill[c] : 0.0;
    o->m[c] = (fl == LIQ) ? r : (fl == IFACE) ? fill[c] * r : 0.0;
    o->rho[c] = 0.0;
    if (fl == LIQ || fl == IFACE) {
      for (i = 0; i < L->q; ++i) o->f[i * N + c] = feq_i(L, i, r, ux, uy, uz);
    } else {
      for (i = 0; i < L->q; ++i) o->f[i * N + c] = 0.0;
    }
  }
  /* bubble labels: connected gas components in order of lowest index (R19) */
  {
    const int nb = label_bubbles(o);
    o->nb = nb;
    free(o->V0);
    free(o->pV);
    o->V0 = (double*)calloc(nb > 0 ? nb : 1, sizeof(double));
    o->pV = (double*)calloc(nb > 0 ? nb : 1, sizeof(double));
    bubble_volumes(o, o->V0);
    for (i = 0; i < nb; ++i) o->pV[i] = o->pv0;
  }
  o->step = 0;
  return 0;
}

/* --------------------------------------------------------------- geometry */
/* K8 kernel of radius 2 on integer offsets (R16). */
static double k8(int dx, int dy, int dz) {
  double r2 = (double)(dx * dx + dy * dy + dz * dz);
  double t = 1.0 - r2 / 4.0;
  if (r2 >= 4.0) return 0.0;
  return t * t * t * t;
}

/* Blocks of 3x3x3 values around a cell, b[(dx+1) + 3 (dy+1) + 9 (dz+1)]. */
#define BLK(dx, dy, dz) ((dx) + 1 + 3 * ((dy) + 1) + 9 * ((dz) + 1))

/* Smoothed fill level at the centre of a block of fill levels (R16):
 * sum K8(r) phi / sum K8(r), summed over dz, dy, dx in that order. */
static double k8_smooth(const double* b) {
  double s = 0.0, wsum = 0.0;
  int dx, dy, dz;
  for (dz = -1; dz <= 1; ++dz)
    for (dy = -1; dy <= 1; ++dy)
      for (dx = -1; dx <= 1; ++dx) wsum = wsum + k8(dx, dy, dz);
  for (dz = -1; dz <= 1; ++dz)
    for (dy = -1; dy <= 1; ++dy)
      for (dx = -1; dx <= 1; ++dx) s = s + k8(dx, dy, dz) * b[BLK(dx, dy, dz)];
  return s / wsum;
}

/* Parker-Youngs gradient at the centre of a block of smoothed fill levels
 * (Eq. nm-fslbm-normal, R17): for axis a, the differences across the two
 * faces normal to a, weighted 4 (face centre), 2 (edge), 1 (corner); p runs
 * over the slower, r over the faster of the two other axes. */
static void py_gradient(const double* b, double* n3) {
  int a;
  for (a = 0; a < 3; ++a) {
    double s = 0.0;
    int p, r;
    for (p = -1; p <= 1; ++p)
      for (r = -1; r <= 1; ++r) {
        int d1[3], d2[3];
        double w;
        if (a == 0) {
          d1[0] = 1; d1[1] = r; d1[2] = p;
        } else if (a == 1) {
          d1[0] = r; d1[1] = 1; d1[2] = p;
        } else {
          d1[0] = r; d1[1] = p; d1[2] = 1;
        }
        d2[0] = d1[0];
        d2[1] = d1[1];
        d2[2] = d1[2];
        d2[a] = -1;
        w = (p == 0 && r == 0) ? 4.0 : (p == 0 || r == 0) ? 2.0 : 1.0;
        s = s + w * (b[BLK(d1[0], d1[1], d1[2])] - b[BLK(d2[0], d2[1], d2[2])]);
      }
    n3[a] = s;
  }
}

double orc_k8_smooth(const double* block27) { return k8_smooth(block27); }
void orc_py_gradient(const double* block27, double* n3) { py_gradient(block27, n3); }

/* The per-cell loops below (and those of classify() and stream_collide())
 * write only their own cell's entries; built with -fopenmp they are shared
 * out over threads with the same results. */
static void geometry(orc* o) {
  long N = o->N, c;
  /* smoothed fill level on every non-obstacle cell; obstacle and
   * out-of-domain stencil points take the centre's value */
#pragma omp parallel for schedule(static)
  for (c = 0; c < N; ++c) {
    int x, y, z, dx, dy, dz;
    double b[27];
    if (o->flag[c] == OBST) continue;
    coords(o, c, &x, &y, &z);
    for (dz = -1; dz <= 1; ++dz)
      for (dy = -1; dy <= 1; ++dy)
        for (dx = -1; dx <= 1; ++dx) {
          long n = nbr(o, x, y, z, dx, dy, dz);
          b[BLK(dx, dy, dz)] = (nflag_of(o, n) == OBST) ? o->phi[c] : o->phi[n];
        }
    o->phis[c] = k8_smooth(b);
  }
  /* Parker-Youngs normal n = grad(phi~) and n^ = n/|n| (R17) */
#pragma omp parallel for schedule(static)
  for (c = 0; c < N; ++c) {
    double n3[3], len, b[27];
    int a, x, y, z, dx, dy, dz;
    if (o->flag[c] == OBST) continue;
    coords(o, c, &x, &y, &z);
    for (dz = -1; dz <= 1; ++dz)
      for (dy = -1; dy <= 1; ++dy)
        for (dx = -1; dx <= 1; ++dx) {
          long n = nbr(o, x, y, z, dx, dy, dz);
          b[BLK(dx, dy, dz)] = (nflag_of(o, n) == OBST) ? o->phis[c] : o->phis[n];
        }
    py_gradient(b, n3);
    len = sqrt(n3[0] * n3[0] + n3[1] * n3[1] + n3[2] * n3[2]);
    for (a = 0; a < 3; ++a) o->nhat[a * N + c] = (len > 0.0) ? n3[a] / len : 0.0;
  }
  /* curvature kappa = -div(n^) by central differences (R18) and rho^G (R7) */
#pragma omp parallel for schedule(static)
  for (c = 0; c < N; ++c) {
    double s = 0.0, pv;
    int a, x, y, z;
    if (o->flag[c] != IFACE) {
      o->kappa[c] = 0.0;
      o->rhog[c] = 0.0;
      continue;
    }
    coords(o, c, &x, &y, &z);
    for (a = 0; a < 3; ++a) {
      int d[3] = {0, 0, 0};
      long np, nm;
      double vp, vm;
      d[a] = 1;
      np = nbr(o, x, y, z, d[0], d[1], d[2]);
      nm = nbr(o, x, y, z, -d[0], -d[1], -d[2]);
      vp = (nflag_of(o, np) == OBST) ? o->nhat[a * N + c] : o->nhat[a * N + np];
      vm = (nflag_of(o, nm) == OBST) ? o->nhat[a * N + c] : o->nhat[a * N + nm];
      s = s + (vp - vm);
    }
    o->kappa[c] = -0.5 * s;
    pv = (o->bubble_model && o->bid[c] >= 0) ? o->pV[o->bid[c]] : o->pv0;
    o->rhog[c] = 3.0 * (pv + o->sigma * o->kappa[c]);
  }
}

void orc_geometry(orc* o, double* nhat, double* kappa, double* phis) {
  geometry(o);
  if (nhat) memcpy(nhat, o->nhat, sizeof(double) * 3 * (size_t)o->N);
  if (kappa) memcpy(kappa, o->kappa, sizeof(double) * (size_t)o->N);
  if (phis) memcpy(phis, o->phis, sizeof(double) * (size_t)o->N);
}

/* Thuerey class of an interface cell (R12). */
static void classify(orc* o) {
  long c;
#pragma omp parallel for schedule(static)
  for (c = 0; c < o->N; ++c) {
    int i, x, y, z;
    int has_l = 0, has_g = 0;
    o->cls[c] = STD;
    if (o->flag[c] != IFACE) continue;
    coords(o, c, &x, &y, &z);
    for (i = 1; i < o->L.q; ++i) {
      long n = nbr(o, x, y, z, o->L.c[i][0], o->L.c[i][1], o->L.c[i][2]);
      int fl = nflag_of(o, n);
      if (fl == LIQ) has_l = 1;
      if (fl == GAS) has_g = 1;
    }
    if (!has_l && has_g) o->cls[c] = NF;
    if (has_l && !has_g) o->cls[c] = NE;
  }
}

/* Interface-interface mass flux with the Thuerey adjustment (R12);
 * a = f*_ibar(y) (incoming), b = f*_i(x) (outgoing). */
static double thuerey(int cx, int cy, double a, double b) {
  if (cx == cy) return a - b;
  if (cx == STD) return (cy == NF) ? a : -b;
  if (cx == NF) return -b;
  return a; /* cx == NE */
}

/* ----------------------------------------------------------- stream-collide */
static void stream_collide(orc* o) {
  const lattice* L = &o->L;
  const int q = L->q;
  long N = o->N, c;
#pragma omp parallel for schedule(static)
  for (c = 0; c < N; ++c) {
    double fin[27], fout[27], fx[27], rho, u[3];
    int miss[27], recon[27];
    int i, x, y, z;
    int fl = o->flag[c];
    if (fl != LIQ && fl != IFACE) continue;
    coords(o, c, &x, &y, &z);
    for (i = 0; i < q; ++i) fx[i] = o->f[i * N + c];
    /* pull streaming (Eq. nm-lbm-streaming) with bounce-back at obstacles
     * and no-slip faces, specular reflection at free-slip faces (R22) */
    for (i = 0; i < q; ++i) {
      int j = i;
      long s = pull_source(o, x, y, z, i, &j);
      int sf = nflag_of(o, s);
      miss[i] = 0;
      if (sf == OBST) {
        fin[i] = fx[L->opp[i]];
      } else if (sf == GAS) {
        if (fl == IFACE) {
          miss[i] = 1;
          fin[i] = 0.0;
        } else {
          fin[i] = fx[L->opp[i]]; /* unreachable while the layer is closed */
        }
      } else {
        fin[i] = o->f[j * N + s];
      }
    }
    if (fl == IFACE) {
      double dm = 0.0;
      double nh[3] = {o->nhat[c], o->nhat[N + c], o->nhat[2 * N + c]};
      double rc, uc[3];
      post_moments(L, o->f + c, N, o->g, &rc, uc);
      select_R(L, o->variant, o->om3_fallback, nh, miss, recon);
      reconstruct(L, recon, o->rhog[c], uc, fx, fin);
      /* mass exchange (Eq. nm-fslbm-mass-flux, R11, R12) with the cell n
       * whose PDF arrives in direction ibar: the neighbour x + c_i, or its
       * mirror image across a free-slip face (R22) */
      for (i = 1; i < q; ++i) {
        int j = L->opp[i];
        long n = pull_source(o, x, y, z, L->opp[i], &j);
        int nf = nflag_of(o, n);
        double a, b;
        if (nf == GAS || nf == OBST) continue;
        a = o->f[j * N + n];
        b = fx[i];
        if (nf == LIQ) {
          dm = dm + (a - b);
        } else {
          double v = thuerey(o->cls[c], o->cls[n], a, b);
          dm = dm + 0.5 * (o->phi[c] + o->phi[n]) * v;
        }
      }
      o->mn[c] = o->m[c] + dm;
    }
    collide(L, o->collision, o->omega, o->trt_magic, o->cs, o->g, fin, fout, &rho, u);
    for (i = 0; i < q; ++i) o->fn[i * N + c] = fout[i];
    o->rho[c] = rho;
    if (fl == IFACE) o->phin[c] = o->mn[c] / rho;
  }
}

/* -------------------------------------------------------------- conversion */
static void convert(orc* o) {
  const lattice* L = &o->L;
  const int q = L->q;
  long N = o->N, c;
  int i, x, y, z;
  /* commit mass and fill of interface cells; raw marks */
  for (c = 0; c < N; ++c) {
    o->mark[c] = C_NONE;
    if (o->flag[c] != IFACE) continue;
    o->m[c] = o->mn[c];
    o->phi[c] = o->phin[c];
    if (o->phi[c] > 1.0 + o->eps) o->mark[c] = C_TOL;
    else if (o->phi[c] < -o->eps) o->mark[c] = C_TOG;
  }
  /* conflicts: liquid-gas separation first (R13) */
  for (c = 0; c < N; ++c) {
    o->conv[c] = o->mark[c];
    if (o->mark[c] != C_TOG) continue;
    coords(o, c, &x, &y, &z);
    for (i = 1; i < q; ++i) {
      long n = nbr(o, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
      if (n >= 0 && o->flag[n] == IFACE && o->mark[n] == C_TOL)
        o->conv[c] = C_NONE;
    }
  }
  /* new flags before deferral */
  for (c = 0; c < N; ++c) {
    int fl = o->flag[c];
    o->nflag[c] = (unsigned char)fl;
    o->isnew[c] = 0;
    if (fl == IFACE) {
      if (o->conv[c] == C_TOL) o->nflag[c] = LIQ;
      if (o->conv[c] == C_TOG) o->nflag[c] = GAS;
    } else if (fl == GAS || fl == LIQ) {
      int want = (fl == GAS) ? C_TOL : C_TOG;
      coords(o, c, &x, &y, &z);
      for (i = 1; i < q; ++i) {
        long n = nbr(o, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
        if (n >= 0 && o->flag[n] == IFACE && o->conv[n] == want) {
          o->nflag[c] = IFACE;
          o->isnew[c] = (unsigned char)(fl == GAS ? 1 : 2);
        }
      }
    }
  }
  /* receivers and deferral (R15) */
  for (c = 0; c < N; ++c) {
    int nrecv = 0;
    o->share[c] = 0.0;
    o->dfr[c] = 0;
    if (o->flag[c] != IFACE || o->conv[c] == C_NONE) continue;
    coords(o, c, &x, &y, &z);
    for (i = 1; i < q; ++i) {
      long n = nbr(o, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
      if (n >= 0 && o->nflag[n] == IFACE) ++nrecv;
    }
    if (nrecv == 0) {
      o->dfr[c] = 1; /* deferred: stays interface, keeps its mass */
    } else {
      double mex = (o->conv[c] == C_TOL) ? (o->m[c] - o->rho[c]) : o->m[c];
      o->share[c] = mex / (double)nrecv;
    }
  }
  for (c = 0; c < N; ++c) {
    if (o->dfr[c]) {
      o->conv[c] = C_NONE;
      o->nflag[c] = IFACE;
    }
  }
  /* new interface cells from gas: f* = f^eq(mean rho, mean u) (R14);
   * from liquid: m = rho, phi = 1 */
  for (c = 0; c < N; ++c) {
    if (o->isnew[c] == 1) {
      double sr = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, rb, ub[3];
      int cnt = 0;
      coords(o, c, &x, &y, &z);
      for (i = 1; i < q; ++i) {
        long n = nbr(o, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
        if (n < 0) continue;
        if (o->nflag[n] == LIQ || (o->nflag[n] == IFACE && !o->isnew[n])) {
          double rn, un[3];
          post_moments(L, o->fn + n, N, o->g, &rn, un);
          sr = sr + rn;
          sx = sx + un[0];
          sy = sy + un[1];
          sz = sz + un[2];
          ++cnt;
        }
      }
      if (cnt > 0) {
        rb = sr / (double)cnt;
        ub[0] = sx / (double)cnt;
        ub[1] = sy / (double)cnt;
        ub[2] = sz / (double)cnt;
      } else {
        rb = 1.0;
        ub[0] = ub[1] = ub[2] = 0.0;
      }
      for (i = 0; i < q; ++i) o->fn[i * N + c] = feq_i(L, i, rb, ub[0], ub[1], ub[2]);
      o->rho[c] = rb;
      o->m[c] = 0.0;
      o->phi[c] = 0.0;
    } else if (o->isnew[c] == 2) {
      int best = -1;
      double rn, un[3];
      post_moments(L, o->fn + c, N, o->g, &rn, un);
      o->rho[c] = rn;
      o->m[c] = rn;
      o->phi[c] = 1.0;
      coords(o, c, &x, &y, &z);
      for (i = 1; i < q; ++i) {
        long n = nbr(o, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
        if (n >= 0 && o->nflag[n] == GAS && o->bid[n] >= 0 &&
            (best < 0 || o->bid[n] < best))
          best = o->bid[n];
      }
      o->bid[c] = best;
    }
  }
  /* excess mass: receivers gather shares in direction order (R15).  The
   * receivers are the cells counted above; a deferred cell was not counted
   * (its flag was not interface then), so it keeps its mass. */
  for (c = 0; c < N; ++c) {
    double s = 0.0;
    if (o->nflag[c] != IFACE || o->dfr[c]) continue;
    coords(o, c, &x, &y, &z);
    for (i = 1; i < q; ++i) {
      long n = nbr(o, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
      if (n >= 0 && o->flag[n] == IFACE && o->conv[n] != C_NONE)
        s = s + o->share[n];
    }
    o->m[c] = o->m[c] + s;
    o->phi[c] = o->m[c] / o->rho[c];
  }
  /* converted cells */
  for (c = 0; c < N; ++c) {
    if (o->flag[c] != IFACE || o->conv[c] == C_NONE) continue;
    if (o->conv[c] == C_TOL) {
      o->phi[c] = 1.0;
      o->m[c] = o->rho[c];
    } else {
      o->phi[c] = 0.0;
      o->m[c] = 0.0;
    }
  }
  for (c = 0; c < N; ++c) o->flag[c] = o->nflag[c];
  for (c = 0; c < N; ++c)
    if (o->flag[c] == LIQ) o->bid[c] = -1;
}

static void bubble_pressure(orc* o) {
  double* V;
  int b;
  if (!o->bubble_model || o->nb == 0) return;
  V = (double*)calloc(o->nb, sizeof(double));
  bubble_volumes(o, V);
  for (b = 0; b < o->nb; ++b)
    o->pV[b] = (V[b] > 0.0) ? (o->pv0 * o->V0[b]) / V[b] : o->pv0;
  free(V);
}

/* Bubble coalescence and segmentation (R24): the bubbles become the
 * connected gas regions of the current flags (label_bubbles), and the gas
 * of every old bubble A, whose amount is proportional to p^V_A V_A =
 * p^V(0) V0_A, goes to the new bubbles in proportion to the volume of A's
 * cells that each holds: V0_C = sum over A (ascending) of
 * V0_A * (vol(A and C) / vol(A handed on)), plus vol(C's cells without an
 * id), volumes in the fixed point of R19, vol(A handed on) over the cells
 * of A that are in a new bubble.  Then p^V = p^V(0) V0 / V. */
static void relabel_bubbles(orc* o) {
  const long N = o->N;
  const int nb_old = o->nb;
  int* old = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
  int64_t *M, *row;
  double *V0n, *pVn;
  int nb_new, A, C, W;
  long c;
  memcpy(old, o->bid, sizeof(int) * (size_t)N);
  nb_new = label_bubbles(o);
  W = nb_new + 1; /* column 0: cells that end in no bubble */
  M = (int64_t*)calloc((size_t)(nb_old > 0 ? nb_old : 1) * (size_t)W, sizeof(int64_t));
  row = (int64_t*)calloc((size_t)(nb_old > 0 ? nb_old : 1), sizeof(int64_t));
  /* free[C]: volume of the cells of new bubble C that carried no id */
  int64_t* fr = (int64_t*)calloc((size_t)(nb_new > 0 ? nb_new : 1), sizeof(int64_t));
  for (c = 0; c < N; ++c) {
    int64_t v;
    A = old[c];
    if (o->flag[c] == GAS)
      v = (int64_t)4294967296LL;
    else if (o->flag[c] == IFACE)
      v = vol_fix(1.0 - o->phi[c]);
    else
      continue;
    if (A < 0) {
      if (o->bid[c] >= 0) fr[o->bid[c]] += v;
      continue;
    }
    M[(size_t)A * W + (size_t)(o->bid[c] + 1)] += v;
    if (o->bid[c] >= 0) row[A] += v; /* the volume A hands on to new bubbles */
  }
  V0n = (double*)calloc((size_t)(nb_new > 0 ? nb_new : 1), sizeof(double));
  pVn = (double*)calloc((size_t)(nb_new > 0 ? nb_new : 1), sizeof(double));
  for (C = 0; C < nb_new; ++C) {
    double s = 0.0;
    for (A = 0; A < nb_old; ++A) {
      const int64_t m = M[(size_t)A * W + (size_t)(C + 1)];
      if (m == 0 || row[A] == 0) continue;
      s = s + o->V0[A] * ((double)m / (double)row[A]);
    }
    /* cells without an id hold gas at p^V(0), like the gas cells outside
       every bubble (their pressure is p^V(0) in the step) */
    V0n[C] = s + (double)fr[C] / 4294967296.0;
  }
  free(fr);
  free(o->V0);
  free(o->pV);
  o->V0 = V0n;
  o->pV = pVn;
  o->nb = nb_new;
  free(M);
  free(row);
  free(old);
  bubble_pressure(o);
}

/* One FSLBM time step: geometry -> stream/BC/mass/collide -> conversion and
 * excess mass -> bubble pressure (and, every relabel_every steps, bubble
 * coalescence and segmentation). */
static void one_step(orc* o) {
  double* t;
  geometry(o);
  classify(o);
  stream_collide(o);
  convert(o);
  t = o->f;
  o->f = o->fn;
  o->fn = t;
  bubble_pressure(o);
  o->step += 1;
  if (o->bubble_model && o->relabel_every > 0 && o->step % o->relabel_every == 0) relabel_bubbles(o);
}

void orc_set_bubble_relabel(orc* o, int every) { o->relabel_every = every > 0 ? every : 0; }

void orc_relabel_bubbles(orc* o) {
  if (o->bubble_model) relabel_bubbles(o);
}

void orc_step(orc* o, int n) {
  int k;
  for (k = 0; k < n; ++k) one_step(o);
}

long orc_steps_done(const orc* o) { return o->step; }

void orc_read(const orc* o, double* pdf, double* fill, unsigned char* flags,
              double* mass) {
  long N = o->N;
  if (pdf) memcpy(pdf, o->f, sizeof(double) * (size_t)o->L.q * N);
  if (fill) memcpy(fill, o->phi, sizeof(double) * (size_t)N);
  if (flags) memcpy(flags, o->flag, (size_t)N);
  if (mass) memcpy(mass, o->m, sizeof(double) * (size_t)N);
}

void orc_read_moments(const orc* o, double* rho, double* u) {
  long c, N = o->N;
  for (c = 0; c < N; ++c) {
    double r = 0.0, v[3] = {0.0, 0.0, 0.0};
    if (o->flag[c] == LIQ || o->flag[c] == IFACE)
      post_moments(&o->L, o->f + c, N, o->g, &r, v);
    if (rho) rho[c] = r;
    if (u) {
      u[c] = v[0];
      u[N + c] = v[1];
      u[2 * N + c] = v[2];
    }
  }
}

int orc_bubbles(const orc* o, double* volume, double* pressure, int* ids_cell,
                int cap) {
  int b;
  if (volume || pressure) {
    double* V = (double*)calloc(o->nb > 0 ? o->nb : 1, sizeof(double));
    bubble_volumes(o, V);
    for (b = 0; b < o->nb && b < cap; ++b) {
      if (volume) volume[b] = V[b];
      if (pressure) pressure[b] = o->bubble_model ? o->pV[b] : o->pv0;
    }
    free(V);
  }
  if (ids_cell) memcpy(ids_cell, o->bid, sizeof(int) * (size_t)o->N);
  return o->nb;
}

/* Total mass: the density of every liquid cell plus the mass of every
 * interface cell.  The cells' contributions are summed with Neumaier's
 * compensated summation, so the result carries no accumulation error that
 * grows with the number of cells (the mass balance is judged at 1e-12). */
double orc_total_mass(const orc* o) {
  long c;
  int i;
  double M = 0.0, comp = 0.0;
  for (c = 0; c < o->N; ++c) {
    double x;
    if (o->flag[c] == LIQ) {
      double r = 0.0;
      for (i = 0; i < o->L.q; ++i) r = r + o->f[i * o->N + c];
      x = r;
    } else if (o->flag[c] == IFACE) {
      x = o->m[c];
    } else {
      continue;
    }
    {
      const double t = M + x;
      if (fabs(M) >= fabs(x))
        comp += (M - t) + x;
      else
        comp += (x - t) + M;
      M = t;
    }
  }
  return M + comp;
}

/* Seed-fill front detection (R23) on the layer z = layer of a flags array
 * (caller order c = x + nx (y + ny z)).  front[nx*ny] (optional) receives 1
 * for front cells; stats[4] = count, minimum, maximum and mean radius
 * (0 when no front cell).  A plain breadth-first fill with a queue. */
int orc_seed_fill_front(int nx, int ny, int nz, int per_x, int per_y, const unsigned char* flags,
                        int layer, double xc, double yc, unsigned char* front, double* stats) {
  long M, c, head = 0, tail = 0;
  int x, y, k;
  unsigned char* reach;
  long* queue;
  const unsigned char* fl;
  double n = 0.0, rmin = 0.0, rmax = 0.0, rsum = 0.0;
  if (nx < 1 || ny < 1 || nz < 1 || layer < 0 || layer >= nz || !flags || !stats) return 1;
  M = (long)nx * ny;
  fl = flags + (long)layer * M;
  reach = (unsigned char*)calloc((size_t)M, 1);
  queue = (long*)malloc(sizeof(long) * (size_t)M);
  if (!reach || !queue) {
    free(reach);
    free(queue);
    return 1;
  }
  /* seeds: gas or obstacle cells on the layer's edge */
  for (y = 0; y < ny; ++y)
    for (x = 0; x < nx; ++x) {
      c = x + (long)nx * y;
      if ((x == 0 || x == nx - 1 || y == 0 || y == ny - 1) && (fl[c] == GAS || fl[c] == OBST)) {
        reach[c] = 1;
        queue[tail++] = c;
      }
    }
  while (head < tail) {
    const long cur = queue[head++];
    const int cx = (int)(cur % nx), cy = (int)(cur / nx);
    for (k = 0; k < 4; ++k) {
      int X = cx + (k == 0) - (k == 1), Y = cy + (k == 2) - (k == 3);
      long nb;
      if (X < 0 || X >= nx) {
        if (!per_x) continue;
        X = (X + nx) % nx;
      }
      if (Y < 0 || Y >= ny) {
        if (!per_y) continue;
        Y = (Y + ny) % ny;
      }
      nb = X + (long)nx * Y;
      if (!reach[nb] && (fl[nb] == GAS || fl[nb] == OBST)) {
        reach[nb] = 1;
        queue[tail++] = nb;
      }
    }
  }
  for (y = 0; y < ny; ++y)
    for (x = 0; x < nx; ++x) {
      int hit = 0;
      c = x + (long)nx * y;
      if (fl[c] == IFACE)
        for (k = 0; k < 4; ++k) {
          int X = x + (k == 0) - (k == 1), Y = y + (k == 2) - (k == 3);
          long nb;
          if (X < 0 || X >= nx) {
            if (!per_x) continue;
            X = (X + nx) % nx;
          }
          if (Y < 0 || Y >= ny) {
            if (!per_y) continue;
            Y = (Y + ny) % ny;
          }
          nb = X + (long)nx * Y;
          if (reach[nb] && fl[nb] == GAS) hit = 1;
        }
      if (front) front[c] = (unsigned char)hit;
      if (hit) {
        const double dx = (x + 0.5) - xc, dy = (y + 0.5) - yc;
        const double r = sqrt(dx * dx + dy * dy);
        if (n == 0.0 || r < rmin) rmin = r;
        if (n == 0.0 || r > rmax) rmax = r;
        rsum += r;
        n += 1.0;
      }
    }
  stats[0] = n;
  stats[1] = rmin;
  stats[2] = rmax;
  stats[3] = n > 0.0 ? rsum / n : 0.0;
  free(reach);
  free(queue);
  return 0;
}


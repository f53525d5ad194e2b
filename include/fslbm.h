/*
 * fslbm.h - C ABI of the GB300 (sm_103a) free-surface lattice Boltzmann step.
 *
 * The library advances the free-surface lattice Boltzmann method (FSLBM) of
 * Schwarzmeier & Ruede, arXiv 2207.13962, Sec. 2 (LBM with SRT/TRT collision
 * and Guo forcing, Eqs. nm-lbm-*; free-surface extension, Eqs. nm-fslbm-*)
 * with the free-surface boundary condition in the four variants of Sec. 3
 * (NBRC Eq. fsbcv-nbrc, NBKC Eq. fsbcv-nbkc, OM Eq. fsbcv-om-sets, OM3
 * Eq. fsbcv-om3).  Every step of the path runs in hand-written CUDA kernels.
 *
 * Conventions shared by all calls
 * -------------------------------
 *  * Cells are indexed c = x + nx * (y + ny * z).
 *  * Cell types (flags): 0 gas, 1 interface, 2 liquid, 3 obstacle (Sec. 2.2).
 *    Cells outside a non-periodic domain face are no-slip walls.
 *  * PDFs are ordered i = 0 rest, 1..6 faces (+x,-x,+y,-y,+z,-z), 7..18 edges,
 *    19..26 corners (D3Q27 only); directions 2k-1 and 2k are opposite.
 *    Full table: (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1)
 *    (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1)
 *    (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1) (1,1,1) (-1,-1,-1) (1,1,-1)
 *    (-1,-1,1) (1,-1,1) (-1,1,-1) (-1,1,1) (1,-1,-1).
 *  * Host arrays passed in are owned by the caller and copied; the context
 *    owns all device memory it allocates.  Nothing is retained after a call.
 *  * Every call returns a status.  A call that fails with FSLBM_EINVAL leaves
 *    the context untouched; the message of the last failure is returned by
 *    fslbm_last_error().
 *  * Work is enqueued on params.stream (a cudaStream_t, NULL = the legacy
 *    default stream).  fslbm_step is asynchronous; fslbm_observables,
 *    fslbm_read_fields and fslbm_sync synchronize that stream.
 */
#ifndef FSLBM_H
#define FSLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fslbm_ctx fslbm_ctx;

typedef enum {
  FSLBM_OK = 0,
  FSLBM_EINVAL = 1,     /* bad argument or initial state; nothing changed   */
  FSLBM_ENOMEM = 2,     /* device or host allocation failed                  */
  FSLBM_ECUDA = 3,      /* a CUDA call failed; see fslbm_last_error()        */
  FSLBM_EUNSTABLE = 4,  /* |u|^2 >= c_s^2, rho <= 0 or a NaN was seen
                           (the instability of Sec. 4.2); fields stay readable */
  FSLBM_ETIMEOUT = 5,   /* a bounded device wait gave up                     */
  FSLBM_ESTATE = 6,     /* call out of order (e.g. step before init)         */
  FSLBM_ECAPACITY = 7   /* a list outgrew its capacity (not returned: the
                           interface and new-cell lists hold every cell) */
} fslbm_status;

/* Velocity sets D3Q19 and D3Q27 (Sec. 2.1). */
typedef enum { FSLBM_D3Q19 = 19, FSLBM_D3Q27 = 27 } fslbm_lattice;

/* Collision: SRT, Eq. nm-lbm-collision-operator (relaxing towards f^eq);
 * TRT: two relaxation rates with the magic parameter trt_magic. */
typedef enum { FSLBM_SRT = 0, FSLBM_TRT = 1 } fslbm_collision;

/* Free-surface boundary-condition variants (i)-(iv) of Sec. 3. */
typedef enum {
  FSLBM_NBRC = 1, /* Eq. fsbcv-nbrc: R = {n.c_i >= 0} (centre included)   */
  FSLBM_NBKC = 2, /* Eq. fsbcv-nbkc: R = {n.c_i > 0} (centre kept)        */
  FSLBM_OM = 3,   /* Eq. fsbcv-om-sets: R = G- (only missing PDFs)        */
  FSLBM_OM3 = 4   /* Eq. fsbcv-om3: OM if |G-| >= 3, else the fallback    */
} fslbm_bc_variant;

/* Storage of the PDFs.  FSLBM_FP64 stores f_i and computes in FP64 with the
 * expressions of the plain CPU oracle.  FSLBM_FP32, FP16S and BF16S store the
 * deviation d_i = f_i - w_i from the rest state (FP16 as d_i * 2^15) and
 * compute in FP32 on deviations, so that rounding is relative to |d| ~ 1e-3
 * rather than to |f|.  Fill level, mass, excess mass, the mass flux between
 * cells and bubble volumes are always FP64.
 * FSLBM_FP32MC and FSLBM_FP16SMC are the mass-conserving forms of FP32 and
 * FP16S: the q - 1 moving deviations lie on a fixed grid (steps of 2^-34 and
 * 2^-30), the rest deviation is stored as an integer number of grid steps
 * and takes up every rounding of the collision, so each liquid cell keeps
 * exactly the mass it received and the liquid mass (Eq. nm-fslbm-mass) does
 * not drift with the storage rounding.  FP32MC stores as many bytes as FP32,
 * FP16SMC 2 more per cell and buffer than FP16S; deviations are bounded by
 * |f_i - w_i| < 2^-3 (FP32MC) and < 2 (FP16SMC), beyond which a step reports
 * FSLBM_EUNSTABLE. */
typedef enum {
  FSLBM_FP64 = 0,
  FSLBM_FP32 = 1,
  FSLBM_FP16S = 2,
  FSLBM_BF16S = 3,
  FSLBM_FP32MC = 4,
  FSLBM_FP16SMC = 5
} fslbm_precision;

/* Boundary of each axis of the domain (the faces at its two ends).  Walls
 * lie outside the domain: FSLBM_NO_SLIP bounces PDFs back (Sec. 2.1),
 * FSLBM_FREE_SLIP reflects them specularly, reversing the wall-normal
 * component (Sec. 2.1); a reflected PDF that comes from a gas cell is
 * missing and the free-surface BC reconstructs it (Sec. 2.2, the paragraph
 * after Eq. nm-fslbm-boundary-condition), and interface cells exchange mass
 * with the mirror cell along the wall (Eq. nm-fslbm-mass-flux).  Obstacle
 * cells inside the domain are always no-slip. */
typedef enum { FSLBM_NO_SLIP = 0, FSLBM_PERIODIC = 1, FSLBM_FREE_SLIP = 2 } fslbm_boundary;

typedef struct {
  int nx, ny, nz;     /* cells per axis, each >= 1                             */
  int periodic[3];    /* fslbm_boundary of each axis (1 = periodic; 0 = no-slip
                         and 2 = free-slip walls outside the domain)          */
} fslbm_domain;

typedef struct {
  double omega;       /* relaxation rate 1/tau, 0 < omega < 2 (Eq. nm-lbm-viscosity) */
  double trt_magic;   /* TRT magic parameter Lambda (3/16 recommended)          */
  double g[3];        /* gravitational acceleration; F = rho g (Sec. 2.2)       */
  double sigma;       /* surface tension (Eq. nm-fslbm-pressure-laplace)        */
  double eps_phi;     /* conversion threshold epsilon_phi, paper: 1e-2          */
  double p_v0;        /* initial volume pressure p^V(0), paper: p0 = 1/3        */
  int precision;      /* fslbm_precision                                        */
  int om3_fallback;   /* FSLBM_NBKC (paper's text) or FSLBM_NBRC (its equation) */
  int bubble_model;   /* 0: all gas at p_v0; 1: per-bubble volume tracking
                         (Eq. nm-fslbm-pressure-volume)                         */
  void* stream;       /* cudaStream_t for all work, NULL = default stream       */
  double smagorinsky_cs; /* Smagorinsky constant C_S of the LES model of Sec. 2.1
                         (Eqs. nm-lbm-turbulence-viscosity to
                         nm-lbm-turublence-relaxation-time; paper: 0.1), 0: off.
                         The local relaxation time is
                         tau = (tau0 + sqrt(tau0^2 + 18 sqrt(2) C_S^2 Qbar / rho)) / 2
                         from the non-equilibrium momentum flux Qbar of the
                         PDFs entering the collision; TRT keeps trt_magic  */
  int bubble_relabel_every; /* bubble coalescence and segmentation (the bubble
                         model Sec. 2.2 cites follows them), every K steps
                         after init; 0 (default): the bubbles stay those of
                         the initial state.  With the bubble model on, the
                         bubbles become the connected gas regions of the
                         current flags (as at init), and each old bubble's
                         gas, whose amount is p^V V = p^V(0) V(0), goes to
                         the new bubbles in proportion to the volume of its
                         cells that each holds (fixed point, exact sums; a
                         bubble none of whose cells is in a new one has
                         vanished with its gas):
                         merging bubbles keep sum p^V V, the parts of a split
                         bubble keep its pressure, and gas or interface cells
                         outside every bubble bring their volume at p^V(0).
                         Single-domain contexts only (batches reject it). */
} fslbm_params;

/* Whole-domain observables (FP64 reductions on the device). */
typedef struct {
  int64_t step;        /* steps done since init                              */
  double total_mass;   /* sum rho (liquid) + sum m (interface), Eq. nm-fslbm-mass */
  int64_t n_liquid, n_interface, n_gas, n_obstacle;
  double max_u;        /* max |u| over liquid and interface cells            */
  int nan_seen;        /* a non-finite value or rho <= 0 was seen            */
  int n_bubbles;       /* bubbles tracked (connected gas regions at init)    */
  double liquid_volume;/* sum of fill levels over liquid and interface cells */
} fslbm_obs;

/* Defaults: omega 1, Lambda 3/16, g 0, sigma 0, eps_phi 1e-2, p_v0 1/3,
 * FP32, OM3 fallback NBKC, no bubble model, default stream, no LES. */
void fslbm_params_default(fslbm_params* p);

/* Create a context for one domain (Sec. 2; Sec. 3 for bc_variant).
 * Allocates all device memory for the domain; returns FSLBM_EINVAL for bad
 * sizes/enums (out untouched), FSLBM_ENOMEM if the device is full. */
fslbm_status fslbm_create(const fslbm_domain* domain, fslbm_lattice lattice,
                          fslbm_collision collision, fslbm_bc_variant bc_variant,
                          const fslbm_params* params, fslbm_ctx** out);

/* Storage order of the cells inside the context (a storage choice: results
 * are the same for every order, bitwise in FP64).  The caller's cell index
 * c = x + nx * (y + ny * z) of every host array in and out of the library
 * never changes.  order[k] is the axis (0 x, 1 y, 2 z) held at storage
 * position k, order[0] the contiguous one.  The bulk stream-collide sweeps
 * 32-cell groups of consecutive storage positions, so it keeps more lanes
 * busy when liquid runs are long along the contiguous axis (a tube along z
 * wants z contiguous).  order == NULL (the default) lets fslbm_init choose:
 * the axis with the fewest liquid-holding groups for the initial flags, x
 * unless another axis needs at most 95 % of x's groups.  Takes effect at the
 * next fslbm_init.  FSLBM_EINVAL unless order is a permutation of 0, 1, 2. */
fslbm_status fslbm_set_axis_order(fslbm_ctx* ctx, const int* order);
/* The storage order in use (order[3]); identity until the first init. */
fslbm_status fslbm_get_axis_order(const fslbm_ctx* ctx, int* order);

/* Initial state (Sec. 2.2).  fill[N] fill levels (used on interface cells;
 * liquid 1, gas 0), flags[N] cell types 0..3, velocity[3N] component-major
 * (ux[N], uy[N], uz[N]) or NULL for rest, density[N] or NULL for rho = 1.
 * PDFs start at f^eq(rho, u) (Eq. nm-lbm-equilibrium); mass m = phi rho
 * (Eq. nm-fslbm-mass).  Gas bubbles are the connected gas regions, labelled
 * in the order of their lowest cell index.  Host pointers, copied.
 * FSLBM_EINVAL if a flag is > 3 or a liquid cell touches a gas cell (the
 * interface layer must be closed). */
fslbm_status fslbm_init(fslbm_ctx* ctx, const double* fill, const uint8_t* flags,
                        const double* velocity, const double* density);

/* Advance n >= 0 time steps: geometry (K8 smoothing, Parker-Youngs normal,
 * FDM curvature), stream-collide with the free-surface BC of the chosen
 * variant, mass exchange and fill update, conversion with neighbour fix-up,
 * excess-mass redistribution and the bubble-pressure update (Sec. 2.2, 3).
 * Asynchronous on params.stream; launch errors are returned, device-side
 * instability is reported by fslbm_sync / fslbm_observables. */
fslbm_status fslbm_step(fslbm_ctx* ctx, int n);

/* Wait for the stream; FSLBM_EUNSTABLE if an instability was flagged,
 * FSLBM_ETIMEOUT if a bounded device wait gave up (only the TMA-staged bulk
 * sweep waits on the device; it is not built by default). */
fslbm_status fslbm_sync(fslbm_ctx* ctx);

/* Whole-domain observables; synchronizes.  Returns FSLBM_EUNSTABLE (with
 * *out filled) when max |u| >= c_s or a NaN was seen. */
fslbm_status fslbm_observables(fslbm_ctx* ctx, fslbm_obs* out);

/* Liquid-front radius statistics of one z-layer. */
typedef struct {
  int64_t count;   /* front cells                                        */
  double r_min, r_max, r_mean; /* radius of their cell centres about the
                                  centre; 0 when count is 0              */
} fslbm_front_stats;

/* Seed-fill front detection (Sec. 4.3, cylindrical dam break: the front
 * radius is taken over the interface cells that a seed fill started at a
 * domain boundary reaches, i.e. the outermost ones).  In the z-layer
 * `layer`, the fill runs through the cells that are gas or obstacle, over
 * in-plane face neighbours (across periodic x/y faces too), seeded with
 * every such cell on the layer's edge (x = 0, nx-1 or y = 0, ny-1).  A front
 * cell is an interface cell of the layer with a reached gas cell among its
 * in-plane face neighbours; its radius is the distance of its centre
 * (x + 1/2, y + 1/2) to (xc, yc).  front_mask (optional, host, nx*ny bytes,
 * index x + nx*y) receives 1 for front cells.  Synchronizes.  FSLBM_EINVAL
 * for a layer outside [0, nz) or a non-finite centre; FSLBM_ESTATE before
 * init.  r_mean sums the radii with device atomics (order not fixed); the
 * count, mask, r_min and r_max do not depend on the order. */
fslbm_status fslbm_front(fslbm_ctx* ctx, int layer, double xc, double yc, fslbm_front_stats* out,
                         uint8_t* front_mask);

/* Copy fields to host buffers (any pointer may be NULL); synchronizes.
 * pdf[q*N] direction-major post-collision PDFs as FP64, fill[N], flags[N]
 * (0..3), mass[N] (meaningful on interface cells; 0 on gas). */
fslbm_status fslbm_read_fields(fslbm_ctx* ctx, double* pdf, double* fill,
                               uint8_t* flags, double* mass);

/* Per-bubble volume V_b and volume pressure p^V_b (Eq. nm-fslbm-pressure-volume);
 * writes min(cap, n) entries, *n_out = number of bubbles.  Synchronizes. */
fslbm_status fslbm_bubbles(fslbm_ctx* ctx, double* volume, double* pressure,
                           int cap, int* n_out);

/* Opt-in per-stage CUDA-event timing of the next steps (0 disables).  While
 * enabled, fslbm_step launches kernels one by one (no CUDA graph). */
fslbm_status fslbm_set_timing(fslbm_ctx* ctx, int enable);
/* Accumulated milliseconds per stage since timing was enabled, one stage per
 * kernel of the step in the order geometry, bulk, interface, resolve, count,
 * apply, finalize (with the rebuild of the interface list in cell order),
 * bubbles; writes min(cap, 8) values.  The FP32 and 16-bit engines run the
 * geometry inside the bulk launch, so their geometry stage is empty. */
fslbm_status fslbm_stage_times(fslbm_ctx* ctx, double* ms, int cap, int* n_launches);

/* Checkpoint of the full state (PDFs, flags, fill, mass, bubbles, step) into
 * a caller buffer.  With buf == NULL only *size is returned.  The arrays are
 * kept in the context's storage order; fslbm_load accepts a checkpoint only
 * in a context with the same sizes, lattice, precision, bubble count and
 * storage order (FSLBM_EINVAL otherwise). */
fslbm_status fslbm_save(fslbm_ctx* ctx, void* buf, size_t* size);
fslbm_status fslbm_load(fslbm_ctx* ctx, const void* buf, size_t size);

/* Number of interface cells of the current state (synchronizes). */
fslbm_status fslbm_interface_count(fslbm_ctx* ctx, int64_t* n);

/* Sizes of the work lists of the next step (synchronizes; any pointer may be
 * NULL): interface cells, 32-cell groups swept by the bulk kernel (those
 * that hold or held liquid) and 8^3 geometry tiles holding interface cells. */
fslbm_status fslbm_work_counts(fslbm_ctx* ctx, int64_t* interface_cells,
                               int64_t* liquid_segments, int64_t* geometry_tiles);

/* Whole-domain observables of a state held in caller-provided device memory,
 * for callers that may not allocate device memory (their device memory is
 * owned by another allocator, or an allocation would stall a latency-critical
 * loop).  The paper has no counterpart: this is a service of the library.
 * Same results as fslbm_observables on the same state.
 *   domain: sizes (periodic flags unused); q: 19 or 27; g[3]: gravity (host).
 *   pdf: device, q*N FP64 post-collision PDFs, direction-major and unpadded:
 *        PDF i of cell c at pdf[i * N + c] (contexts pad their own direction
 *        slices, so pass an array like the one fslbm_read_fields returns).
 *   flags, fill, mass: device, N entries each (flags 0..3, higher bits ignored).
 *   out: host; stream: cudaStream_t or NULL.  Synchronizes the stream.
 * Allocates nothing: the block partials live in a fixed 66 KB device array
 * of the library (held by every GPU that loads it until the process exits).
 * The first call on a device looks up that array's device address and keeps
 * it for the life of the process; make that call before any stream capture.
 * The kept address does not survive cudaDeviceReset: after a reset of the
 * device in the same process, this entry point must not be used again.  All
 * calls share the array, so calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialized by the caller.
 * FSLBM_EINVAL for q not 19/27, empty domains or more than 2^31 - 1 cells;
 * FSLBM_ECUDA if a CUDA call fails. */
fslbm_status fslbm_observables_noalloc(const fslbm_domain* domain, int q, const double* g,
                                       const double* pdf, const uint8_t* flags,
                                       const double* fill, const double* mass,
                                       fslbm_obs* out, void* stream);

void fslbm_destroy(fslbm_ctx* ctx);
const char* fslbm_last_error(const fslbm_ctx* ctx);
const char* fslbm_version(void);

/* ------------------------------------------------------------------ batches
 * Many domains of different sizes advance together: each phase of the step
 * (geometry, bulk stream-collide, interface update, conversion, excess mass,
 * bubbles; Sec. 2.2, 3) runs as ONE launch over a block table of all member
 * domains, captured once in a CUDA graph.  Results are those of stepping
 * each member alone: bitwise in FP64 (compiled without multiply-add
 * contraction), to FP32 rounding otherwise (the compiler may contract the
 * shared per-cell code differently in the batched kernels).
 *
 * Members are initialized contexts of the same lattice, precision and
 * collision operator (variant, omega, g, sigma, eps_phi, bubble model and
 * sizes may differ).  They stay owned by the caller, must outlive the batch,
 * and keep working with every single-context call between batch steps
 * (fslbm_step, fslbm_read_fields, ...): a batch step is ordered after the
 * members' pending work and their later work after it. */
typedef struct fslbm_batch fslbm_batch;

/* Launch shape of a batch step: persistent bulk-sweep blocks per SM and
 * interface-band blocks per SM; ms_per_step is the time measured for it by
 * fslbm_batch_autotune (0 if not measured). */
typedef struct {
  int bulk_blocks_per_sm;
  int band_blocks_per_sm;
  double ms_per_step;
} fslbm_tuning;

/* Group n >= 1 members (host array of context pointers, copied).  Work is
 * enqueued on stream (cudaStream_t, NULL = legacy default).  FSLBM_ESTATE if
 * a member is not initialized; FSLBM_EINVAL for mixed lattice, precision or
 * collision, or a member listed twice. */
fslbm_status fslbm_batch_create(fslbm_ctx* const* members, int n, void* stream, fslbm_batch** out);

/* Advance every member n >= 0 steps (asynchronous, n graph launches). */
fslbm_status fslbm_batch_step(fslbm_batch* b, int n);

/* Wait for the batch stream; FSLBM_EUNSTABLE if any member flagged an
 * instability.  member_status (n entries, may be NULL) receives each
 * member's status. */
fslbm_status fslbm_batch_sync(fslbm_batch* b, fslbm_status* member_status);

/* Pick the launch shape by measurement: every combination of 1..max bulk
 * blocks per SM and {1, 2, 4, 8} band blocks per SM runs 1 + steps batch
 * steps timed with CUDA events; the fastest is kept and returned in *chosen
 * (may be NULL).  The steps are real steps: every member advances by
 * (steps + 1) x (number of candidates). */
fslbm_status fslbm_batch_autotune(fslbm_batch* b, int steps, fslbm_tuning* chosen);
fslbm_status fslbm_batch_set_tuning(fslbm_batch* b, const fslbm_tuning* t);
fslbm_status fslbm_batch_get_tuning(const fslbm_batch* b, fslbm_tuning* t);
/* Kernels launched by batch steps so far. */
fslbm_status fslbm_batch_launches(const fslbm_batch* b, int64_t* n);
void fslbm_batch_destroy(fslbm_batch* b);
const char* fslbm_batch_last_error(const fslbm_batch* b);

/* Device bytes a context of this domain holds, including the peak of
 * fslbm_init's staging buffers (with_velocity: a velocity field is passed).
 * FSLBM_EINVAL for bad sizes or enums. */
fslbm_status fslbm_memory_estimate(const fslbm_domain* domain, fslbm_lattice lattice, int precision,
                                   int with_velocity, size_t* bytes);

/* ------------------------------------------------------------------ serving
 * A request loop with continuous batching.  Runs of different domain sizes
 * are submitted as they arrive; each poll admits queued runs in arrival
 * order while slots (max_active) and device memory (memory_budget, by
 * fslbm_memory_estimate) allow, keeps the admitted runs' PDFs, flags and
 * fill levels resident, advances all of them together by up to chunk_steps
 * steps in the shared launches of one batch (rebuilt when the membership
 * changes), and retires the runs that are done: their fill levels, flags and
 * observables are copied to the host and their device memory is freed for
 * the next admissions.  A run's result is that of running it alone (bitwise
 * in FP64, to FP32 rounding otherwise; see batches). */
typedef struct fslbm_server fslbm_server;

typedef struct {
  fslbm_lattice lattice;     /* shared by all runs */
  fslbm_collision collision; /* shared by all runs */
  int precision;             /* fslbm_precision, shared by all runs */
  int max_active;            /* resident runs at most (>= 1) */
  int chunk_steps;           /* steps between admission rounds (>= 1) */
  int64_t memory_budget;     /* device bytes for resident runs; 0: 90 % of
                                the memory free when the server is created */
  void* stream;              /* cudaStream_t for all work, NULL = default */
} fslbm_server_config;

typedef struct {
  fslbm_domain domain;
  fslbm_bc_variant bc_variant;
  fslbm_params params;       /* precision must equal the server's; stream ignored */
  const double* fill;        /* host arrays as for fslbm_init, copied at submit */
  const uint8_t* flags;
  const double* velocity;    /* may be NULL */
  const double* density;     /* may be NULL */
  int steps;                 /* steps to run */
} fslbm_request;

typedef struct {
  int64_t id;
  int status;                /* fslbm_status of the run (init or final state) */
  int64_t steps;             /* steps done */
  int64_t cells;
  fslbm_obs obs;             /* observables of the final state */
  double t_queue;            /* seconds from submit to admission */
  double t_result;           /* seconds from submit to the result (time-to-result) */
} fslbm_result;

typedef struct {
  int64_t submitted, admitted, completed;
  int queued, active, max_active_seen;
  int64_t batch_rebuilds, batch_steps;
  double cell_updates;       /* cells x steps of the completed runs */
  int64_t memory_used, memory_budget;
} fslbm_server_stats;

fslbm_status fslbm_server_create(const fslbm_server_config* cfg, fslbm_server** out);
/* Queue a run (host arrays copied); *id identifies its result.  FSLBM_ENOMEM
 * if the run alone exceeds the memory budget. */
fslbm_status fslbm_server_submit(fslbm_server* s, const fslbm_request* rq, int64_t* id);
/* One round: admit, step the resident runs by up to chunk_steps (synchronous),
 * retire finished runs.  *n_active (may be NULL): runs resident afterwards. */
fslbm_status fslbm_server_poll(fslbm_server* s, int* n_active);
/* Result of a finished run (FSLBM_ESTATE while it is not finished); fill[N]
 * and flags[N] (may be NULL) receive its final fields.  The result is
 * released by this call. */
fslbm_status fslbm_server_result(fslbm_server* s, int64_t id, fslbm_result* res, double* fill,
                                 uint8_t* flags);
fslbm_status fslbm_server_stats_get(const fslbm_server* s, fslbm_server_stats* out);
void fslbm_server_destroy(fslbm_server* s);
const char* fslbm_server_last_error(const fslbm_server* s);

#ifdef __cplusplus
}
#endif
#endif /* FSLBM_H */

/*
 * fv.h -- C ABI of libfv, a GB300 (sm_103a) solver for the reduced
 * Baer-Nunziato diffuse-interface model with the second-order well-balanced
 * path-conservative finite-volume scheme of Gaburro, Castro & Dumbser,
 * "A well balanced diffuse interface method for complex nonhydrostatic free
 * surface flows" (Section 3: Eq. (Scheme) with the Osher x fluctuation, the
 * well-balanced Osher-Romberg y fluctuation, the fluctuation reconstruction of
 * Section 3.4 and the free-surface detector of Section 3.5).
 *
 * Conventions shared by every entry point
 *   - State layout: four structure-of-arrays planes, in this order,
 *       m = alpha*rho, mu = alpha*rho*u, mv = alpha*rho*v, a = alpha,
 *     each ny*nx doubles with the x index fastest: q[v*nx*ny + j*nx + i].
 *     The 5th variable of the paper (the gravity potential y) is static and is
 *     not stored.  Solid (removed) cells are ignored on input and are 0 on
 *     output.
 *   - Cell (i, j) covers [x0 + i dx, x0 + (i+1) dx] x [y0 + j dy, y0 + (j+1) dy];
 *     gravity acts along -y.
 *   - Ownership: the library owns every device buffer it allocates; the caller
 *     owns every array it passes in and may free it when the call returns.
 *   - Streams: all device work is enqueued on the stream given to fv_create
 *     (NULL = legacy default stream).  Calls that return host data synchronise
 *     that stream first.
 *   - Errors: every call returns an fv_status; no C++ exception crosses the
 *     ABI.  fv_last_error() gives a thread-local message for the last failure.
 *   - Threads: one handle must not be used from two threads at once.
 */
#ifndef FV_H
#define FV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FV_OK = 0,
  FV_EINVAL = 1,      /* invalid argument (null pointer, bad size, gamma != 1, ...) */
  FV_ENOMEM = 2,      /* device or host allocation failed */
  FV_ECUDA = 3,       /* a CUDA runtime call failed */
  FV_ENONFINITE = 4,  /* a step produced a non-finite state or alpha <= 0 or alpha*rho <= 0 */
  FV_ETIMEOUT = 5     /* a bounded device wait gave up */
} fv_status;

/* Arithmetic of the step.
 *   FV_FP64     : state and all arithmetic in double.
 *   FV_FP32_DEV : deviation form of Section 3.4 in float.  The stored state is
 *                 m^f = m - alpha rho^E(y; y0_i) (deviation from the cell's own
 *                 water-at-rest profile), mu, mv, alpha; fluxes, reconstruction
 *                 and update run in float; the dt reduction, the detector
 *                 column sums and the equilibrium table are double. */
typedef enum { FV_FP64 = 0, FV_FP32_DEV = 1 } fv_prec;

enum { FV_BC_WALL = 0, FV_BC_TRANSMISSIVE = 1 };

/* Uniform Cartesian grid of nx x ny cells T_ij (Section 3: rectangular grid). */
typedef struct {
  int32_t nx, ny;     /* >= 1 each; nx*ny <= 2^31 - 1 */
  double x0, y0;      /* lower-left corner */
  double dx, dy;      /* > 0 */
} fv_grid;

/* Tait liquid (Eq. (TaitLaw)) and model constants (Section 5 preamble). */
typedef struct {
  double rho0;        /* reference density, > 0 */
  double k0;          /* Tait constant, > 0 */
  double gamma;       /* Tait exponent; must be 1 (all of the paper's tests) */
  double g;           /* gravity, >= 0 (0 switches gravity off) */
  double eps_gas;     /* gas volume fraction eps, in (0, 0.1) */
} fv_eos;

/* Boundaries: side[0..3] = West, East, South, North, each FV_BC_WALL (reflective
 * wall, the mirror state with u.n negated, Section 5 preamble) or
 * FV_BC_TRANSMISSIVE.  solid: nullable host pointer to nx*ny bytes (x fastest),
 * 1 = cell removed from the domain (obstacle, Section 5.1), copied at create. */
typedef struct {
  int32_t side[4];
  const uint8_t* solid;
} fv_bc;

typedef struct fv_handle fv_handle;

/* Diagnostics of the current state (fv_get_diag). */
typedef struct {
  double t;           /* simulated time since fv_set_state */
  int64_t steps;      /* steps taken since fv_set_state */
  double dt_next;     /* dt the next step will use (CFL of the last fv_step) */
  double mass;        /* sum over fluid cells of m dx dy, fixed-order double sum */
  int32_t status;     /* FV_OK or FV_ENONFINITE if any step since set_state failed */
} fv_diag;

/* Create a solver for one domain.  cuda_stream: a cudaStream_t (may be NULL).
 * Allocates all device memory for the grid (about 80 bytes per cell in FP64).
 * Returns FV_EINVAL for bad sizes or parameters, FV_ENOMEM on allocation
 * failure; *out is set only on success. */
fv_status fv_create(const fv_grid* grid, const fv_eos* eos, const fv_bc* bc, fv_prec prec,
                    void* cuda_stream, fv_handle** out);

/* Load Q^0 (layout above).  on_device = 0: q is host memory; 1: q is device
 * memory readable on the handle's stream.  Runs the free-surface detector
 * (Eq. (Free_surf_detector)) and the CFL reduction for the first step, and
 * resets t and the step count.  Non-admissible fluid cells give FV_EINVAL. */
fv_status fv_set_state(fv_handle* h, const double* q, int on_device);

/* Advance n >= 0 time steps of Eq. (Scheme), each with
 * dt = cfl / max over fluid cells of ((|u|+c)/dx + (|v|+c)/dy), cfl in (0, 1].
 * Asynchronous on the handle's stream unless t_out is non-null, in which case
 * the stream is synchronised, *t_out receives the simulated time and the
 * device status is checked (FV_ENONFINITE if a step produced a bad state). */
fv_status fv_step(fv_handle* h, int32_t n, double cfl, double* t_out);

/* Scheme used by the following fv_step / fv_step_timed calls: 2 (default) =
 * Eq. (Scheme) with the second-order well-balanced reconstruction of Section
 * 3.4; 1 = the first-order scheme of Sections 3.2-3.3 (Eq.
 * (SemidiscreteScheme_2)): cell averages as face states, y faces along the
 * well-balanced path between the two cell centres, no interior term.  Both
 * precisions.  fv_adjoint, the batch and fv_step_static are second order
 * only.  FV_EINVAL for another value. */
fv_status fv_set_order(fv_handle* h, int32_t order);

/* x-face viscosity used by the following fv_step / fv_step_timed calls:
 * FV_XFACE_GL (default) = the Osher viscosity with 3-point Gauss-Legendre
 * quadrature of |A1| (Eq. (OsherMatrixFormal_approx)); FV_XFACE_OR = the
 * conservative Osher-Romberg viscosity of Section 3.1 (Eq. (OR_cons)) with the
 * Romberg nodes of Eq. (RombergWeights), b4x = u Delta alpha on each
 * sub-segment.  Both orders and precisions; fv_adjoint, the batch and
 * fv_step_static use Gauss-Legendre.  FV_EINVAL for another value. */
#define FV_XFACE_GL 0
#define FV_XFACE_OR 1
fv_status fv_set_xface(fv_handle* h, int32_t solver);

/* Staging of the second-order step kernel used by the following fv_step,
 * fv_step_timed and fv_adjoint calls.  The arithmetic of a step (Eq. (Scheme))
 * is the same in every staging and the results are bitwise identical; only
 * the speed differs.  FV_TILING_TILE = one CTA per 32 x 8 tile of cells;
 * FV_TILING_STRIP = one CTA per 32-column strip marching upwards in blocks of
 * 8 rows, sharing the reconstructed rows and y faces between blocks
 * (faster in both precisions); FV_TILING_AUTO (default) = the strip kernel.
 * The batch (fv_batch_*) stages by strips.  FV_EINVAL for another value. */
#define FV_TILING_AUTO 0
#define FV_TILING_TILE 1
#define FV_TILING_STRIP 2
fv_status fv_set_tiling(fv_handle* h, int32_t tiling);

/* Rows per strip of the strip kernel (a positive multiple of 8), or 0
 * (default) for the built-in choice from the grid and the device's occupancy.
 * Results do not depend on it; speed does.  FV_EINVAL for a negative value or
 * one that is not a multiple of 8. */
fv_status fv_set_strip_height(fv_handle* h, int32_t rows);

/* Autotuner: times the strip kernel of the current order-2 step from the
 * current state with strip heights of 32, 48, 64, 96, 128, 160, 192 and 256 rows
 * (those not above the grid, rounded up to 8), three launches each after one
 * warm-up, on the handle's stream, and keeps the fastest (fv_set_strip_height).
 * The state, time, levels and accumulators are left as they were (the trial
 * launches write only the other state buffer, which the next step
 * overwrites).  *rows_out (nullable) receives the chosen height.  A no-op for
 * the first-order scheme and the tile staging.  Synchronises the stream.
 * FV_EINVAL without a state; FV_ECUDA on a CUDA error (the previous height is
 * kept). */
fv_status fv_tune(fv_handle* h, int32_t* rows_out);

/* fv_step plus timing: CUDA events recorded on the handle's stream around
 * every launch of the fused step kernel give *kernel_ms, the summed device
 * time of those launches, and *total_ms, the device time of the whole call
 * (step kernels plus the per-step finalize kernel).  Synchronises the stream;
 * either output pointer may be null.  Errors as fv_step. */
fv_status fv_step_timed(fv_handle* h, int32_t n, double cfl, double* kernel_ms, double* total_ms);

/* Copy the current state out in the layout above (double).  on_device as in
 * fv_set_state.  Synchronises the stream. */
fv_status fv_get_state(fv_handle* h, double* q, int on_device);

/* Detected free-surface levels K_i (y0_i = y0 + K_i dy) the next step will
 * use; K: host array of nx int32.  Synchronises the stream. */
fv_status fv_get_levels(fv_handle* h, int32_t* K);

/* Time, step count, next dt, fluid mass and status.  Synchronises. */
fv_status fv_get_diag(fv_handle* h, fv_diag* d);

/* Release the handle and its device memory (synchronises; NULL is a no-op). */
void fv_destroy(fv_handle* h);

/* ---- Discrete adjoint (reverse mode) of n time steps.
 *
 * Loss of a gauge record: L = sum_{n=1..N} dt_n sum_g (m_g^n - T_g^n)^2, m =
 * alpha rho at gauge cell g after step n, dt_n the step's dt.  fv_adjoint runs
 * the N steps from the handle's current state Q^0 (like fv_step(h, N, cfl);
 * the handle holds Q^N afterwards) and returns dL/dQ^0.  The paper computes
 * no gradients; the derivative is that of the scheme of Eq. (Scheme) with the
 * quantities that are piecewise constant in the state held at their forward
 * values: dt_n, the detected levels K_i^n (Eq. (Free_surf_detector)), and each
 * branch of the step (the Barth-Jespersen factor's active face and stencil
 * extremum, |u|, sign(v) with sign(0) = 0, the order switch alpha <= 10 eps,
 * the first-order fallback).  It is evaluated in the handle's arithmetic type
 * (FP64, or FP32 deviation form) and accumulated in double.  States at every
 * checkpoint_every-th step are kept on the device and each segment is
 * replayed once before it is reversed (ceil(sqrt(N)) when 0: about 2 sqrt(N)
 * stored states, one extra forward pass). */
typedef struct {
  int32_t nsteps;           /* N >= 1 */
  double cfl;               /* (0, 1] */
  int32_t ngauges;          /* >= 1 */
  const int64_t* gauges;    /* host, ngauges fluid cell indices j*nx + i (repeats allowed) */
  const double* target;     /* host, N*ngauges: T_g^n at [(n-1)*ngauges + g] */
  int32_t checkpoint_every; /* >= 0; 0 = ceil(sqrt(N)) */
  double* m_series;         /* nullable host, N*ngauges: receives m_g^n */
  /* Obstacle heights (optional; nheights = 0 for none).  The paper removes
   * whole cells for an obstacle, so its height has no derivative in the
   * scheme; the derivative returned is that of the extension in which
   * raising obstacle k by theta dy leaves the fluid cell on each of its top
   * cells a capacity 1 - theta: its x faces open over min(c_left, c_right) dy
   * (a neighbour sees the closed part as a wall), its y fluctuations and the
   * y jump terms of the interior integral divided by the capacity, the
   * gravity integral not.  theta = 0 is the scheme of Eq. (Scheme), and the
   * value is the one-sided derivative d/dh_k at the grid-aligned heights
   * (raising), with dt_n and K_i^n held as for dL_dq0. */
  int32_t nheights;         /* >= 0 */
  const int32_t* height_id; /* host, ny*nx, null iff nheights = 0: k in [0, nheights) at the
                               fluid cells resting on obstacle k (the cell below is solid),
                               -1 elsewhere */
  double* dL_dh;            /* host, nheights, null iff nheights = 0: receives dL/dh_k (per
                               metre of height; 0 for a k with no cells) */
} fv_adjoint_spec;

typedef struct {
  double loss;              /* L */
  double t;                 /* simulated time after the N steps */
  int32_t checkpoints;      /* stored states */
  int32_t recomputed_steps; /* forward steps replayed by the reverse sweep */
  double forward_ms;        /* device time of the forward sweep (CUDA events) */
  double reverse_ms;        /* device time of the reverse sweep, replays included */
} fv_adjoint_info;

/* dL_dq0: 4 planes (alpha rho, alpha rho u, alpha rho v, alpha) of nx*ny
 * doubles, layout of fv_set_state, zero in solid cells; host (on_device = 0)
 * or device memory (1).  info: nullable.  Synchronises.  FV_EINVAL on bad
 * arguments (a gauge outside the grid or in a solid cell, a non-finite
 * target, a height_id entry out of range or on a cell that is not a fluid
 * cell resting on a solid one), FV_ENONFINITE if a forward step produced a non-admissible state,
 * FV_ENOMEM if the workspace (about (2 sqrt(N) + 20) state-sized buffers)
 * cannot be allocated. */
fv_status fv_adjoint(fv_handle* h, const fv_adjoint_spec* spec, double* dL_dq0, int on_device,
                     fv_adjoint_info* info);

/* The map whose derivative fv_adjoint returns (reading R-adj; the paper
 * computes no gradient): n >= 0 steps of Eq. (Scheme) from the handle's state,
 * step k (0-based) taking dt[k] (host, finite, >= 0) and the levels
 * K[k*nx .. k*nx + nx) (host, each in [0, ny]) instead of its own, as
 * fv_adjoint holds them (record them from a free run with fv_get_diag's
 * dt_next and fv_get_levels before each step).  If ngauges > 0, m_series
 * (host, n*ngauges) receives alpha rho at gauges[g] (host, cell indices j*nx
 * + i) after each step, at [k*ngauges + g].  The state advances; the simulated
 * time and step count do not.  Second order with Gauss-Legendre x faces on an
 * undivided grid only.  Allocates device memory for its records; synchronises.
 * FV_EINVAL for bad arguments, FV_ENONFINITE if a step produced a
 * non-admissible state. */
fv_status fv_step_frozen(fv_handle* h, int32_t n, const double* dt, const int32_t* K,
                         int32_t ngauges, const int64_t* gauges, double* m_series);

/* ---- Batched ensemble of independent domains (configs of uneven sizes,
 * parameter sweeps).  Each domain has its own grid, equation of state,
 * boundaries, free-surface levels, dt (its own CFL condition) and time; one
 * ensemble step advances every domain by one of its own steps.  A step is one
 * launch over the strips of all domains (a persistent grid, or one CTA per
 * strip after fv_batch_tune finds that faster) plus one per-domain finalize
 * launch; fv_batch_step captures n steps into a CUDA graph on an internal
 * stream (ordered after and before the stream given at create) and replays it.
 * The paper runs one domain at a time; the per-domain arithmetic is the same as
 * fv_step's. */
typedef struct fv_batch fv_batch;

/* ndom >= 1 domains; grids, eos, bcs: host arrays of ndom entries (each as for
 * fv_create; solid masks are copied).  Errors as fv_create. */
fv_status fv_batch_create(int32_t ndom, const fv_grid* grids, const fv_eos* eos, const fv_bc* bcs,
                          fv_prec prec, void* cuda_stream, fv_batch** out);

/* State of domain dom (layout as fv_set_state; on_device as there).  Every
 * domain needs a state before the first fv_batch_step.  Synchronises. */
fv_status fv_batch_set_state(fv_batch* b, int32_t dom, const double* q, int on_device);

/* n ensemble steps with CFL number cfl (each domain its own dt).
 * Asynchronous with respect to the host. */
fv_status fv_batch_step(fv_batch* b, int32_t n, double cfl);

/* As fv_batch_step; *total_ms receives the device time of the n steps (CUDA
 * events on the internal stream).  Synchronises. */
fv_status fv_batch_step_timed(fv_batch* b, int32_t n, double cfl, double* total_ms);

/* Autotuner of the batch's step launch: times the step kernel from the
 * current states with strips of 32, 48, 64, 96, 128, 160, 192 and 256 rows,
 * each in two work orders (0: domain by domain; 1: longest strips first) and
 * two launch forms (1: a persistent grid of the resident CTAs taking the strips
 * round-robin; 0: one CTA per strip, handed out by the block scheduler as CTAs
 * finish), three launches each after one warm-up at the given cfl, and keeps
 * the fastest (default before tuning: 128 rows, domain order, persistent).
 * Results do not depend on the choice; speed does.  States, times, levels and
 * accumulators are left as they were (the trial launches write only the other
 * state buffers, which the next step overwrites); cached step graphs are
 * dropped when the choice changes.  rows_out, order_out, persistent_out
 * (nullable) receive it.  Synchronises.  FV_EINVAL if a domain has no state or
 * cfl is outside (0, 1]; FV_ECUDA on a CUDA error (the previous choice is
 * kept). */
fv_status fv_batch_tune(fv_batch* b, double cfl, int32_t* rows_out, int32_t* order_out,
                        int32_t* persistent_out);

/* Sets the batch's step launch as fv_batch_tune would: strips of `rows` rows (a
 * positive multiple of 8), work order 0 or 1, persistent 1 or 0 (meanings as
 * above).  Results do not depend on it.  FV_EINVAL on another value; FV_ECUDA
 * if the new work list cannot be placed (the previous launch is kept). */
fv_status fv_batch_set_launch(fv_batch* b, int32_t rows, int32_t order, int32_t persistent);

/* State, diagnostics and domain count (as the single-domain calls). */
fv_status fv_batch_get_state(fv_batch* b, int32_t dom, double* q, int on_device);
fv_status fv_batch_get_diag(fv_batch* b, int32_t dom, fv_diag* d);
int32_t fv_batch_size(const fv_batch* b);

/* Release the ensemble (synchronises; NULL is a no-op). */
void fv_batch_destroy(fv_batch* b);

/* ---------------------------------------------------------------------------
 * Partitioned domains, for one grid over several GPUs (x strips: the scheme's
 * stencil, Eq. (Scheme), reaches two columns to each side of a cell, and the
 * levels of Eq. (Free_surf_detector) are sums over whole columns; the paper
 * runs on one GPU and has no partition of its own).  One grid of NX
 * columns is split into strips owning columns [a_k, b_k); strip k is a handle
 * created (fv_create) on columns [a_k - 2, b_k + 2) of the grid, clipped at the
 * grid's sides (its x0, solid mask and the grid's W/E boundary kinds on the
 * clipped sides accordingly; an inner side's kind is irrelevant).  Its state
 * (fv_set_state) is the grid's state on those columns.  Per step, for every
 * strip: fv_step(h, 1, cfl, NULL); then fv_part_rate into one device double
 * per strip and fv_part_set_rate with all of them (strips on one GPU) or with
 * their all-reduce(max) (strips on several GPUs); then fv_part_pack of both
 * inner sides, the transfer of each buffer to the neighbouring strip (the same
 * device buffer on one GPU, a send/receive between GPUs), and fv_part_unpack
 * there.  After
 * fv_set_state the rate exchange is done once before the first step.  The
 * owned cells then hold bit for bit what one handle on the whole grid
 * computes, in both precisions.  All calls are asynchronous on the handle's
 * stream; the caller orders the transfers between streams. */

/* Owned columns [own_lo, own_hi) of this handle's grid: own_lo is 0 (the grid's
 * W side) or 2 (a strip to the W), nx - own_hi is 0 or 2, own_hi - own_lo >= 2;
 * (0, 0) = not partitioned (the default).  Only owned cells count in the signal
 * rate and the status; fv_step and fv_step_timed then take n <= 1 and
 * fv_adjoint is refused.  FV_EINVAL otherwise. */
fv_status fv_set_partition(fv_handle* h, int32_t own_lo, int32_t own_hi);

/* Bytes of one side's halo buffer: 4 planes x ny rows x 2 columns of the
 * handle's element type (double in FV_FP64, float in FV_FP32_DEV, as stored:
 * alpha rho as its deviation from equilibrium in FP32), plane-major then row
 * then column, followed by 4 int32 (the 2 columns' levels of the stored state
 * and of the next step). */
fv_status fv_part_halo_bytes(const fv_handle* h, int64_t* bytes);

/* Copy the signal rate of the handle's current state (the largest over its
 * owned fluid cells; over all its cells right after fv_set_state, whose halo
 * columns then hold the grid's true values) to rate_dev (one device double). */
fv_status fv_part_rate(fv_handle* h, double* rate_dev);

/* Adopt the largest of the n >= 1 device doubles rates_dev[0..n) (the strips'
 * rates, or one already reduced across GPUs) as the current state's signal
 * rate; the next fv_step takes dt = cfl / rate from it and adds that dt to the
 * simulated time. */
fv_status fv_part_set_rate(fv_handle* h, const double* rates_dev, int32_t n);

/* side 0 (W) / 1 (E): pack the 2 owned columns next to that side into buf_dev
 * (device, fv_part_halo_bytes bytes; the receiving strip's halo on its other
 * side) / unpack buf_dev into the 2 halo columns of that side.  FV_EINVAL if
 * the side has no neighbouring strip or the handle has no state. */
fv_status fv_part_pack(fv_handle* h, int32_t side, void* buf_dev);
fv_status fv_part_unpack(fv_handle* h, int32_t side, const void* buf_dev);

/* Largest grid fv_step_static accepts (size of its static scratch array). */
#define FV_STATIC_MAX_NX 8192
#define FV_STATIC_MAX_NY 8192

/* One FP64 time step that allocates no device memory.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc, such as an
 * application that owns all of its GPU memory through its own pool, or a
 * latency-critical loop where cudaMalloc's implicit synchronisation is not
 * acceptable.  It computes exactly what fv_set_state + one fv_step compute in
 * FV_FP64, from q_in to q_out, keeping its scratch (detector column sums,
 * levels, equilibrium table, step scalars; about 385 KB) in one file-scope
 * device array that every GPU loading the library holds until the process
 * exits.
 *   grid, eos, side[4]: as for fv_create (host pointers); grid must satisfy
 *     nx <= FV_STATIC_MAX_NX and ny <= FV_STATIC_MAX_NY, else FV_EINVAL.
 *   solid: device pointer, nx*ny bytes (1 = removed cell).
 *   q_in, q_out: device pointers to the 4-plane double state (layout above);
 *     they must not alias.  Solid cells of q_out are written as 0.
 *   cfl in (0, 1]; cuda_stream: the stream for all work (NULL = default).
 *   dt_out: nullable host pointer; if given, the stream is synchronised,
 *     *dt_out receives the step's dt and the states are checked: FV_EINVAL if
 *     q_in has a fluid cell with alpha <= 0, alpha*rho <= 0 or a non-finite
 *     value (as fv_set_state), else FV_ENONFINITE if q_out is not admissible.
 *     Without dt_out the call is asynchronous and neither state is checked.
 * Calls no allocating routine.  The first call on a device looks up the
 * array's device address with that device current.  The equilibrium table in the array is copied
 * from a host buffer when ny, dy, rho0 or the gravity constant differ from the
 * previous call's on that device.  Every call reuses the same array, which keeps
 * the previous call's contents (the accumulators are cleared at the start of
 * each call), so calls whose work overlaps on a GPU (other streams, other host
 * threads) race and must be serialised by the caller. */
fv_status fv_step_static(const fv_grid* grid, const fv_eos* eos, const int32_t side[4],
                         const uint8_t* solid, const double* q_in, double* q_out, double cfl,
                         void* cuda_stream, double* dt_out);

/* Measured fused multiply-add peak of the current device (roofline
 * denominator of the step kernels, which run on the plain FP32/FP64 pipes; the
 * paper has no counterpart).  kind 0: FP32 scalar FFMA; 1: FP32 paired FFMA2
 * (two lanes per instruction); 2: FP64 DFMA.  Runs `reps` >= 1 timed launches
 * of 8 CTAs x 256 threads per SM, each thread advancing 8 independent
 * recurrences a <- a b + c (about 30 ms per launch), after one warm-up, on a
 * stream of its own; *tflops receives 2 x FMAs / the fastest launch's CUDA-
 * event time in TFLOP/s, *best_ms (nullable) that time.  Allocates and frees
 * a small output buffer; synchronises.  FV_EINVAL for a bad argument,
 * FV_ECUDA on a CUDA error. */
fv_status fv_measure_fma_peak(int32_t kind, int32_t reps, double* tflops, double* best_ms);

/* The double-precision reciprocal the FP64 device code uses (the hardware
 * approximation r refined by the series r (1 + e + e^2), e = 1 - x r),
 * evaluated at n device doubles
 * x_dev into out_dev on cuda_stream (asynchronous), so that it can be checked
 * against IEEE division; the paper has no counterpart. */
fv_status fv_device_rcp(const double* x_dev, double* out_dev, int64_t n, void* cuda_stream);

/* Message of the last failed call on this thread ("" if none). */
const char* fv_last_error(void);

/* Library version string. */
const char* fv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FV_H */

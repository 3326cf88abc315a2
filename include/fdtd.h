/*
 * fdtd.h -- C ABI of the GB300 fundamental-scheme implicit FDTD library.
 *
 * Method: E. L. Tan, "Fundamental Schemes for Efficient Unconditionally Stable
 * Implicit Finite-Difference Time-Domain Methods" (arXiv 2011.14043).
 * The library advances Maxwell's equations on a 3-D Yee grid with PEC walls
 * using one of the fundamental schemes of Sec. II:
 *   FDTD_FADI   fundamental ADI, Eqs. 7-10 (component form Eqs. 37-44)
 *   FDTD_FLOD   fundamental LOD1/SS1, Eq. 15
 *   FDTD_FSS    fundamental second-order split step (SS2), Eq. 17
 *   FDTD_FLOD2  fundamental LOD2 with input/output processing, Eqs. 21-23
 * Each time step is a sequence of updating procedures.  A procedure is, for
 * each of three (E, H) component pairs, an implicit update with a
 * matrix-operator-free right-hand side (a batch of tridiagonal line solves
 * along x, y or z), an explicit H update from the solved E, and the
 * subtraction E <- w - E (Sec. III, Eqs. 38-44 and 45-52).
 *
 * Conventions shared by every call
 * --------------------------------
 * Errors: every call returns FDTD_OK (0) or a negative FDTD_ERR_* code and
 *   never throws or aborts.  After FDTD_ERR_CUDA the handle is poisoned: every
 *   later call except fdtd_destroy returns FDTD_ERR_STATE.  A device
 *   allocation that fails inside a call on a handle returns FDTD_ERR_OOM and
 *   poisons the handle the same way (the call may have changed part of it);
 *   fdtd_create cleans up and returns FDTD_ERR_OOM.
 * Arrays: component arrays are C-contiguous [k][j][i] (x fastest) in the
 *   compact Yee shapes (nx, ny, nz = cells):
 *     EX (nz+1, ny+1, nx)   EY (nz+1, ny, nx+1)   EZ (nz, ny+1, nx+1)
 *     HX (nz, ny, nx+1)     HY (nz, ny+1, nx)     HZ (nz+1, ny, nx)
 *   Element type is the handle's precision: double for FDTD_F64, float for
 *   FDTD_F32.  Per-cell material arrays are double, shape (nz, ny, nx).
 * Ownership: the library owns all device memory it allocates.  Pointers
 *   passed in are only read (or written, for outputs) during the call; with
 *   on_device != 0 they are device pointers on the handle's device, else
 *   host pointers.
 * Streams: a handle is bound to one CUDA stream (NULL = legacy default
 *   stream) given at creation; device work is enqueued on it.  Calls that
 *   return host data synchronise that stream.  Handles are not thread-safe.
 * Walls: perfect electric conductor on all six walls; tangential E on the
 *   walls is held at zero (values passed in for those samples are ignored).
 * 2-D: nz == 1 gives the 2-D TM case (Ez, Hx, Hy), the CFL limit then uses
 *   dx and dy only.
 */
#ifndef FDTD_H_
#define FDTD_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDTD_OK 0
#define FDTD_ERR_INVALID_ARG (-1)   /* bad pointer, size, index or value */
#define FDTD_ERR_OOM (-2)           /* device or host allocation failed */
#define FDTD_ERR_CUDA (-3)          /* a CUDA call failed; handle poisoned */
#define FDTD_ERR_TIMEOUT (-4)       /* a bounded device wait gave up */
#define FDTD_ERR_UNSTABLE (-5)      /* non-finite field or invariant growth */
#define FDTD_ERR_UNSUPPORTED (-6)   /* valid request this build does not implement */
#define FDTD_ERR_STATE (-7)         /* call not valid in the handle's state */
#define FDTD_ERR_BOUNDS (-8)        /* bounds-checked build (-DFDTD_BOUNDS) only: a kernel
                                       index fell outside its array; the access was
                                       skipped and the results are not valid */

typedef enum { FDTD_FADI = 0, FDTD_FLOD = 1, FDTD_FSS = 2, FDTD_FLOD2 = 3 } fdtd_scheme;
typedef enum { FDTD_F64 = 0, FDTD_F32 = 1 } fdtd_precision;
typedef enum { FDTD_EX = 0, FDTD_EY = 1, FDTD_EZ = 2, FDTD_HX = 3, FDTD_HY = 4, FDTD_HZ = 5 } fdtd_comp;

/* Problem statement (Sec. III: grid, lossless isotropic medium, dt).
 * dt > 0 is used as given; otherwise dt = cfl * dt_CFL with
 * dt_CFL = 1 / (c0 * sqrt(1/dx^2 + 1/dy^2 [+ 1/dz^2 when nz > 1])),
 * c0 = 299792458 m/s.  tune[] are kernel-shape overrides (0 = automatic):
 * tune[0] nodes per thread of the non-persistent y/z-line kernels (8, 16 or
 * 32); tune[1] bit 0 set: do not use the persistent TMA-fed y/z kernel
 * (FP32 fields; FP64 fields always run the direct-load y/z kernel);
 * tune[1] bit 1 set: per-node (inhomogeneous-media) coefficients even when
 * fdtd_set_material receives a uniform eps (needed by fdtd_adj_create);
 * tune[1] bit 2 set: the TMA-fed kernel stages its outputs in shared memory
 * and writes them with TMA stores instead of register stores; tune[1] bit 3
 * set: fdtd_step launches the kernels one by one instead of replaying a
 * captured step graph; tune[1] bit 4 set: lines along x of FP32 fields in
 * homogeneous media (129 to 256 cells) run the persistent TMA-fed kernel
 * instead of the one-warp-per-line kernel (the same results; measured
 * slower at 256^3); tune[1] bits 5-6: ring depth and blocks per SM of the
 * TMA-fed x-line kernel (0: 3 stages x 4 blocks, 1: 2 x 4, 2: 4 x 3,
 * 3: 2 x 6); tune[1] bit 7 set: lines along x of FP32 fields in homogeneous
 * media take the tabulated factors near the walls (lanes that diverge from
 * the rest of their warp) instead of the converged factors on every lane
 * with a rank-one (Sherman-Morrison) wall correction; tune[1] bit 8 set:
 * fields set from page-locked host memory go through a staging copy
 * instead of being read in place by the unpacking kernel; tune[1] bit 9
 * set: with fourth-order differences every line takes the one-thread-per-
 * line kernel instead of the block-tiled kernel (FP32 fields, lines of at
 * most 512 cells; the same arithmetic, the same results); tune[1] bit 10
 * set: lines along y and z of FP64 fields with uniform mu (pairs of at
 * least 32768 lines) take the segmented solve instead of one thread per line
 * walking the Thomas recurrences (equal to rounding; the default needs a
 * scratch of three field arrays, allocated at the first fdtd_step); tune[1]
 * bit 11 set: lines along x of exactly 32 L cells (FP32, homogeneous media,
 * wall-corrected) keep the kernel with end-of-line masks instead of the one
 * without them (the same results). */
typedef struct {
  int32_t nx, ny, nz;        /* cells per axis: 2 <= nx <= 1024, 2 <= ny, 1 <= nz; lines
                                along y and z are solved with at most 32 segments of
                                at most 32 nodes, so ny, nz <= 1024 (else
                                FDTD_ERR_UNSUPPORTED) */
  double dx, dy, dz;         /* cell sizes [m], > 0 */
  double dt;                 /* time step [s] */
  double cfl;                /* CFL number, used when dt <= 0 */
  int32_t scheme;            /* fdtd_scheme */
  int32_t precision;         /* fdtd_precision: FP64, or FP32 fields with
                                coefficients formed in FP64 */
  int32_t tune[2];
} fdtd_desc;

typedef struct fdtd_s fdtd_t;

/* Create a handle: validates desc, allocates the six state arrays (zero
 * fields, vacuum) on the current CUDA device, precomputes in FP64 the
 * factorised tridiagonal coefficients of every procedure (Sec. IV: "5N
 * flops ... with precomputed bidiagonally factorized elements").
 * stream: a cudaStream_t or NULL.  *out receives the handle. */
int fdtd_create(const fdtd_desc* desc, void* stream, fdtd_t** out);

/* Release all device and host memory of the handle (NULL is a no-op). */
int fdtd_destroy(fdtd_t* h);

/* The time step in use [s]. */
int fdtd_get_dt(const fdtd_t* h, double* dt);

/* Per-cell relative permittivity / permeability (host, nz*ny*nx doubles,
 * each > 0 and finite; NULL means 1 everywhere).  eps at an E sample is the
 * mean of the in-domain cells sharing that edge; mu at an H sample the mean
 * of the cells sharing that face.  Non-uniform mu runs the general-media
 * kernels (a coupling and an off-diagonal per H face) and is built for grids
 * with nx, ny, nz <= 256 (FDTD_ERR_UNSUPPORTED otherwise); batches and the
 * reverse pass take uniform mu only.  Only valid before the first
 * fdtd_step. */
int fdtd_set_material(fdtd_t* h, const double* eps_r_cell, const double* mu_r_cell);

/* fdtd_set_material with an electric conductivity: sigma_cell (host,
 * nz*ny*nx doubles, each >= 0 and finite [S/m]; NULL or all zero means a
 * lossless medium).  The paper writes A and B for a lossless medium (Sec.
 * III) but states its splitting formulae (Sec. II) for any linear operators;
 * the loss term -sigma/eps E of dE/dt is split evenly between A and B on the
 * E rows, so every procedure of length h adds b sigma / 4 (b = h/(2 eps)) to
 * the diagonal of its line systems, and the FADI input initialization
 * (I + dt/2 B) takes its half of the loss.  sigma at an E sample is the mean
 * of the cells sharing its edge (as eps).  Only the FP64-formed pivots change:
 * the kernels are those of the lossless case.  FADI and FLOD2 invert
 * (I + dt/2 B) resp. (I + dt/4 B) for their output, whose loss diagonal has
 * the opposite sign: they need sigma dt / eps <= 2 at every E sample
 * (FDTD_ERR_UNSUPPORTED otherwise; FLOD and FSS take any sigma).  The
 * reverse pass takes lossless media only.  Only valid before the first
 * fdtd_step. */
int fdtd_set_media(fdtd_t* h, const double* eps_r_cell, const double* mu_r_cell, const double* sigma_cell);

/* Order of the spatial differences: 2 (the Yee differences of Sec. III,
 * the default) or 4.  The paper names higher-order difference operators as
 * a variant its fundamental schemes leave room for (end of Sec. III-A)
 * without formulae; with order 4 every first difference of A and B is the
 * fourth-order staggered central difference (9/8 (u_{+1/2} - u_{-1/2}) -
 * 1/24 (u_{+3/2} - u_{-3/2})) / d, with PEC images past the walls
 * (tangential E odd, H even).  A and B stay skew in the energy product (the
 * schemes keep their invariants); each line system has bandwidth 3 and is
 * solved by a banded LU formed in FP64, one thread per line (three
 * field-sized device scratch arrays are allocated here).  Uniform lossless media and
 * single grids only: FDTD_ERR_UNSUPPORTED for per-cell media, conductivity,
 * batches and the reverse pass.  Only valid before the first fdtd_step. */
int fdtd_set_order(fdtd_t* h, int order);

/* Set one physical field component at the current time (compact Yee shape,
 * handle precision).  For FADI the auxiliary state (Eq. 10) is formed from
 * the physical fields on the next fdtd_step. */
int fdtd_set_field(fdtd_t* h, int comp, const void* data, int on_device);

/* Read one physical field component at the current time.  FADI applies the
 * output relation u = u~/2 (Eq. 9) in the equivalent state form
 * u = (I + dt/2 B)^{-1} (v - pending source); FLOD2 applies its output
 * processing (Eq. 23); FLOD/FSS return the state. */
int fdtd_get_field(fdtd_t* h, int comp, void* out, int on_device);

/* Raw scheme state (FADI: auxiliary v of Eq. 8; FLOD2: u^{n+1/4} of Eq. 21;
 * else the field) for checkpointing; same layout as fdtd_get_field. */
int fdtd_get_state(fdtd_t* h, int comp, void* out, int on_device);
int fdtd_set_state(fdtd_t* h, int comp, const void* data, int on_device);

/* Point current source on one E sample (comp EX/EY/EZ, sample indices in the
 * component's compact shape, not on a wall).  current[n] (host, n < count)
 * is the current I [A] used by step n, i.e. I(t_n + dt/2); steps beyond
 * count use 0.  It enters as f_E = -I/(A eps) with A the sample's dual-face
 * area; each procedure of length h adds (h/2) f to the original-form
 * right-hand side (the paper omits sources; this is the reading used), with
 * f of the step's own sample, except in FDTD_FLOD2: its B procedure, centred
 * on t_{n+1}, takes the mean of current[n] and current[n+1], and its input
 * and output processing (Eqs. 22, 23) the sample of the step that follows
 * them.  With these placements each scheme converges to the semi-discrete
 * Yee system with its current at the temporal order of Table I.
 * One source per handle; a new call replaces it; count == 0 removes it. */
int fdtd_set_source(fdtd_t* h, int comp, int i, int j, int k, const double* current, int64_t count);

/* Record one physical field sample after every step.  *id receives the
 * probe index (0, 1, ...).  At most 16 probes.  FADI samples its output
 * field w/2 (Eq. 9) from the two solves of the step; FLOD2 applies the
 * output processing (Eq. 23) to the whole state every step while it has
 * probes (one extra procedure per step). */
int fdtd_add_probe(fdtd_t* h, int comp, int i, int j, int k, int* id);

/* Advance nsteps time steps (asynchronous on the handle's stream). */
int fdtd_step(fdtd_t* h, int64_t nsteps);

/* Copy the first n recorded values of a probe (host buffer); n may not
 * exceed the number of steps taken since the probe was added. */
int fdtd_get_probe(fdtd_t* h, int id, double* out, int64_t n);

/* FP64 reductions: out[0] = field energy 1/2 dV sum(eps E^2 + mu H^2) of the
 * physical field; out[1] = the same quadratic form of the scheme state (the
 * exactly conserved invariant of a source-free run: equal to out[0] for
 * FLOD/FSS).  Returns FDTD_ERR_UNSTABLE (out still filled) if either is not
 * finite, or if a run with no source has let out[1] grow past its reference
 * by more than 1e-8 (FDTD_F64) or 1e-2 (FDTD_F32) relative (measured
 * roundoff drift is about 1e-13 / 1e-5 per thousand steps).  The reference
 * is the invariant of the state the run started from: taken at the first
 * fdtd_step or fdtd_energy after fdtd_set_field, fdtd_set_source or
 * fdtd_set_material; fdtd_set_state keeps it (restoring a checkpoint of the
 * same run). */
int fdtd_energy(fdtd_t* h, double out[2]);

/* Number of steps taken. */
int fdtd_steps_done(const fdtd_t* h, int64_t* n);

/* Wait for the handle's stream.  Returns FDTD_ERR_TIMEOUT if a kernel's
 * bounded wait gave up (the context stays usable). */
int fdtd_synchronize(fdtd_t* h);

/* Launch accounting and per-kernel timing.  Launch classes of the
 * line-solve kernels: 0 = lines along y, 1 = lines along z, 2 = lines
 * along x.  bytes_per_launch is the algorithmic traffic of one launch: the
 * pair's E and H samples, each read once and written once. */
typedef struct {
  int64_t launches;              /* all kernels this handle enqueued */
  int64_t timed_launches[3];     /* line-solve launches timed, per class */
  double timed_ms[3];            /* their summed device time [ms] */
  double bytes_per_launch[3];    /* algorithmic bytes of one launch */
} fdtd_stats;

/* enable != 0: record a CUDA event pair around every line-solve launch
 * (on the handle's stream) until disabled.  Costs one event record per
 * launch boundary. */
int fdtd_set_timing(fdtd_t* h, int enable);

/* Fill *out (synchronises the stream to resolve pending events). */
int fdtd_get_stats(fdtd_t* h, fdtd_stats* out);

/* Zero the counters and drop recorded events. */
int fdtd_reset_stats(fdtd_t* h);

/* Field energy 1/2 dV sum(eps E^2 + mu H^2) of six device field arrays,
 * without allocating anything.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory where they need
 * the energy (inside a framework whose caching allocator holds the device's
 * memory, or in a loop that cannot take cudaMalloc's implicit device-wide
 * synchronisation).  Its per-plane partial sums live in a fixed 192 KiB
 * file-scope device array that every GPU loading the library holds until
 * the process exits.
 *   fields[6]: device pointers on the current device, compact Yee shapes
 *     ([k][j][i], x fastest), element type double (FDTD_F64) or float
 *     (FDTD_F32); uniform eps_r and mu_r.
 *   out_device: device pointer to one double that receives the energy.
 *   stream: cudaStream_t or NULL; the call is asynchronous on it.
 * Limit: nz <= 4096 (nz + 1 planes per component); larger nz returns
 * FDTD_ERR_INVALID_ARG with a message on stderr.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and caches it for the process, so make that first
 * call before any stream capture, and do not use this entry point after
 * cudaDeviceReset (the cached address may then be stale).  A CUDA error
 * already pending when the call starts is reported as FDTD_ERR_CUDA and
 * left pending; nothing is launched then.
 * All calls share the array: calls whose kernels overlap on the GPU (other
 * streams or threads) race on it. */
int fdtd_energy_noalloc(int nx, int ny, int nz, double dx, double dy, double dz, double eps_r, double mu_r,
                        int precision, const void* const* fields, double* out_device, void* stream);

/* Batches of many independent cavities.  A batch steps a set of
 * handles together: each procedure of the scheme runs as one launch per
 * launch-shape group (line direction, lanes, segment length and count)
 * covering every grid of the batch; the groups of one procedure run
 * concurrently on parallel graph branches, and one step of the whole batch
 * is captured once as a CUDA graph and replayed.  Every grid runs exactly the arithmetic of its own handle's
 * fdtd_step.  Handles must share scheme, precision and stream, be distinct,
 * and have no source or probe (FDTD_ERR_UNSUPPORTED); they stay owned by
 * the caller, stay usable for set/get/energy, and must outlive the batch.
 * stream: the handles' stream.  Errors as for fdtd_step. */
typedef struct fdtd_batch_s fdtd_batch_t;
int fdtd_batch_create(fdtd_t* const* handles, int count, void* stream, fdtd_batch_t** out);
int fdtd_batch_step(fdtd_batch_t* b, int64_t nsteps);
int fdtd_batch_destroy(fdtd_batch_t* b);
/* Kernel launches per batch step (for accounting; persistent mode: one per
 * procedure, memsets not counted); valid after a step. */
int fdtd_batch_launches(const fdtd_batch_t* b, int64_t* per_step);
/* Launch shape of the batch: cfg = {y lanes, y L, z lanes, z L, x warps per
 * block, x packing} (lanes: lines per tile of the y/z kernels; L: nodes per
 * thread, which sets the carry-chain depth ceil(N/L); grids with uniform
 * media keep the L of their coefficient tables; x packing 1: x lines of up
 * to 256 nodes in grids with per-node media run on 8, 16 or 32 lanes with 8
 * nodes per lane, several short lines per warp; 0: one warp per x line).  By
 * default the first fdtd_batch_step tunes it: each candidate shape is timed
 * on the batch's own data (out of place, into the handles' scratch arrays,
 * so the state is untouched) and the fastest kept; results are cached per
 * device, precision, scheme and grid list for the process, and appended to
 * the file named by the environment variable FDTD_TUNE_CACHE when set.
 * tune_ms (may be NULL) receives the tuned time of each direction's
 * launches for one step.  fdtd_batch_set_config fixes the shape
 * (FDTD_ERR_INVALID_ARG for a shape that is not built); cfg = NULL returns
 * to tuning. */
int fdtd_batch_get_config(const fdtd_batch_t* b, int32_t cfg[6], double tune_ms[3]);
int fdtd_batch_set_config(fdtd_batch_t* b, const int32_t* cfg);
/* How a batch step runs.  mode 0: the graph of shape-uniform launches above
 * (one per launch group, on parallel branches).  mode 1: one persistent
 * launch per procedure: its blocks take work items (y/z tiles of any grid
 * packed side by side into the block's threads, or a block's worth of x
 * lines) from a counter that a memset zeroes before the launch, until the
 * list is exhausted; both are captured in the step graph.  mode -1 (default): the first step times
 * both on the batch's own data (one-step graph replays writing scratch) and
 * keeps the faster (the persistent launches also with both y and z lines
 * at (16, 8) and (16, 16), a persistent win bringing its shape along);
 * cached like the shapes.  Persistent launches run blocks of 256 threads
 * and need per-node media on every grid, y and z lines of one shape with a
 * built kernel ((lanes, L) = (16, 8), and for FP32 fields (16, 16)) whose
 * tiles take at most 256 threads (lines of at most 128 cells at L = 8, 256
 * at L = 16), and x lines packed by 8, 16 or 32 lanes: mode 1 otherwise
 * fails with FDTD_ERR_UNSUPPORTED at the next step, and mode -1 keeps the
 * launches.  Both modes run the same arithmetic per line: the
 * fields agree to the last bit.  fdtd_batch_get_mode (valid after a step)
 * gives the mode in use (1 persistent) and the tuned time of one step in
 * each mode (ms; 0 when not timed). */
int fdtd_batch_set_mode(fdtd_batch_t* b, int mode);
int fdtd_batch_get_mode(const fdtd_batch_t* b, int32_t* persistent, double step_ms[2]);

/* Reverse mode: gradient of a probe-energy objective of FADI with respect to
 * the per-cell permittivity.
 *
 * Objective: J = sum over steps n = 1..nsteps and over the probe samples of
 * (E^n)^2, where E^n is the FADI output field after step n (w_B/2, Eq. 9 with
 * Eqs. 8c-8d) and the probe samples are every interior Ex, Ey and Ez sample
 * whose array index (i, j, k) lies in the cell block
 * block = {i0, i1, j0, j1, k0, k1} (half-open ranges).  The gradient is the
 * exact discrete adjoint of the stepper: each procedure's transpose runs in
 * reverse order (transposed line solves with the procedure's own pivots,
 * transposed stencil), and dJ/d eps is collected per E sample, then carried
 * through the edge averaging of eps to the cells.  Checkpoints of the state
 * are kept every checkpoint_every steps; the backward pass recomputes each
 * segment from its checkpoint before running it in reverse.
 *
 * fdtd_adj_create: h must be a FADI handle with per-node media (eps set by
 *   fdtd_set_material, non-uniform or tune[1] bit 1), fields and source set,
 *   no probes, and not yet stepped (FDTD_ERR_UNSUPPORTED / FDTD_ERR_STATE
 *   otherwise).  Device memory: about (6 nsteps/checkpoint_every +
 *   6 checkpoint_every + 18) state arrays (fdtd_adj_memory gives the bytes);
 *   FDTD_ERR_OOM when it does not fit.  The context borrows h, which must
 *   outlive it.
 * fdtd_adj_forward: runs the nsteps steps on h (h advances; its fields are
 *   afterwards those of step nsteps) and returns J (FP64 sum).  Once only.
 * fdtd_adj_backward: grad_eps_r[nz][ny][nx] (double; host or device) =
 *   jbar * dJ/d eps_r per cell.  Requires the forward pass; may be repeated.
 *   h's own state is not touched. */
typedef struct fdtd_adj_s fdtd_adj_t;
int fdtd_adj_create(fdtd_t* h, const int32_t block[6], int64_t nsteps, int32_t checkpoint_every,
                    fdtd_adj_t** out);
int fdtd_adj_forward(fdtd_adj_t* a, double* objective);
int fdtd_adj_backward(fdtd_adj_t* a, double jbar, double* grad_eps_r, int on_device);
int fdtd_adj_memory(const fdtd_adj_t* a, int64_t* bytes);
int fdtd_adj_destroy(fdtd_adj_t* a);

/* Test hook: the n-th device allocation of the library from now on (0 = the
 * next one) fails as an out-of-memory would, without calling CUDA; n < 0
 * disarms it.  For exercising the error and clean-up paths; process-wide. */
int fdtd_debug_fail_alloc(int64_t n);

/* Self-test of the bounded device waits (failure detection without a GPU
 * fault).  Every spin-wait in the kernels (the TMA kernels' mbarrier waits)
 * gives up after a time limit, records that in a device flag and returns, so
 * that the host reports FDTD_ERR_TIMEOUT and the context stays usable.  This
 * launches one block whose thread waits, through the same bounded wait, on an
 * mbarrier expecting one arrival: with arrive = 0 nobody arrives and the call
 * returns FDTD_ERR_TIMEOUT after about limit_ns; with arrive = 1 the thread
 * arrives first and the call returns FDTD_OK.  limit_ns in (0, 1e10];
 * synchronises stream (NULL = legacy default stream). */
int fdtd_selftest_bounded_wait(int64_t limit_ns, int arrive, void* stream);

/* FP64 FMA throughput of the current device, measured: a kernel of 8
 * blocks of 256 threads per SM, each thread running 8 independent chains of
 * `iters` FMAs, timed with CUDA events after one shorter warm-up launch.
 * *flops_per_s = 2 x FMAs / time.  The FP64 form of the line solve is bound
 * by this rate rather than by HBM, so it is the denominator of that form's
 * ALU roofline.  iters in [1, 1e6] (about 4.5 s on a GB300 at 1e6); synchronises stream (NULL = legacy
 * default stream). */
int fdtd_probe_fp64_fma(int64_t iters, double* flops_per_s, void* stream);

/* Static description of an error code. */
const char* fdtd_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_H_ */

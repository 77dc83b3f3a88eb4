/*
 * ugks.h -- C ABI of libugks: implicit unsteady unified gas-kinetic scheme
 * (UGKS) on moving and overset structured meshes, for one NVIDIA GB300
 * (sm_103a).  Method: arXiv 2604.09984, Sec. 2 (implicit UGKS with dual time
 * stepping, Eqs. BGK, BGKReduce, microscopicFlux, macroscopicFlux,
 * fullSolution, maxWalldes, dualTimeStepping_macro/micro, Steps 1-8) and
 * Sec. 3 (moving overset meshes: motion, assembly Sec. 3.1, interpolation
 * Sec. 3.2).
 *
 * Conventions shared by every call
 *  - Every function returns an int status: UGKS_OK (0) or a negative
 *    UGKS_ERR_* code; ugks_last_error() returns the message of the last
 *    failure on a context.  A failed call leaves the context usable unless it
 *    returned UGKS_ERR_CUDA (sticky device error).
 *  - Device memory is owned by the caller.  ugks_workspace_query() reports
 *    the bytes of one device workspace; the caller allocates it (any
 *    allocator, 256-byte aligned) and passes it to ugks_create(); the library
 *    never allocates or frees device memory and keeps only borrowed device
 *    pointers into that workspace plus host-side metadata.
 *  - Work is issued on the caller's CUDA stream (cudaStream_t passed as a
 *    void*; NULL = legacy default stream) and is asynchronous unless stated.
 *    Inside ugks_step part of each inner iteration runs on a stream the
 *    context creates for itself, forked from and joined back to the
 *    caller's stream with events, so completion of the caller's stream
 *    implies completion of all work.  Calls that return data in HOST buffers
 *    synchronise that stream.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Coordinates, fields and parameters cross the boundary in FP64.
 *
 * Units and notation: nondimensional with R = 1; particle velocity v, gas
 * velocity V, mesh/face velocity U, relative velocity w = v - U.  Distribution
 * functions are stored in the reduced pair (h, b) = (int f dxi, int xi^2 f
 * dxi) of Sec. 2.1, velocity-contiguous: f[cell][k][2], k = iy*nvx + ix.
 */
#ifndef UGKS_H
#define UGKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define UGKS_OK               0
#define UGKS_ERR_ARG         -1   /* invalid argument or size                 */
#define UGKS_ERR_CUDA        -2   /* a CUDA runtime call or launch failed     */
#define UGKS_ERR_GEOMETRY    -3   /* a cell volume <= 0 after a mesh move     */
#define UGKS_ERR_ORPHAN      -4   /* overset receptors without donor          */
#define UGKS_ERR_NONPHYSICAL -5   /* non-finite or non-positive rho or T      */
#define UGKS_ERR_WORKSPACE   -6   /* workspace missing, too small, misaligned */
#define UGKS_ERR_ORDER       -7   /* calls out of order (e.g. step w/o move)  */
#define UGKS_ERR_TIMEOUT     -8   /* a kernel's bounded wait for its data ran
                                     out; the step's results are invalid    */

/* arithmetic of the per-(cell, velocity) path */
#define UGKS_FP64 0   /* f, fluxes and sweeps in FP64                          */
#define UGKS_FP32 1   /* mixed precision: f, the per-velocity flux,
                         collision, sweep and interpolation arithmetic and the
                         lane sums of the velocity reductions in FP32 (sums
                         compensated, combined error-free); in FP64: the
                         velocity moments W, q and face sums once combined,
                         the macroscopic update (W', step-7 fix), the per-face
                         interface state (g0 primitives, micro and time slopes,
                         collision time, Shakhov heat-flux prefactor, time
                         integrals q1..q5, rounded once to FP32 for the
                         velocity loops), the per-cell Shakhov records and all
                         geometry (volumes, S n, S U.n, dt_s)                  */
#define UGKS_BF16F 2  /* experiment: as UGKS_FP32, but f itself stored as bf16
                         pairs (4 bytes a cell-velocity, rounded to nearest
                         on every store); errors of ~1e-3 relative, outside
                         the 1e-5 bound of the mixed path                      */

/* boundary kind of a block side (sides ordered i-low, i-high, j-low, j-high) */
#define UGKS_BC_NONE     0   /* interior; i-sides of a periodic block          */
#define UGKS_BC_WALL     1   /* diffuse isothermal wall moving with the mesh
                                (Sec. 2.1 wall condition, Eq. maxWalldes)      */
#define UGKS_BC_FARFIELD 2   /* ghost cell at the free-stream state (Sec. 2.1) */
#define UGKS_BC_OUTFLOW  3   /* ghost cell copying the interior state          */
#define UGKS_BC_OVERSET  4   /* outer edge of a component grid: its n_fringe
                                cell layers are overset receptors (Sec. 3.1)   */

/* cell status after overset assembly (Sec. 3.1) */
#define UGKS_FIELD    0   /* solved cell                                      */
#define UGKS_RECEPTOR 1   /* interpolated from donors (Sec. 3.2)              */
#define UGKS_HOLE     2   /* inactive                                         */

typedef struct ugks_ctx ugks_ctx;

/* Gas, velocity space and solver constants (Sec. 2.1, 2.2). */
typedef struct {
  int precision;            /* UGKS_FP64, UGKS_FP32 or UGKS_BF16F              */
  int nvx, nvy;             /* uniform tensor velocity grid, trapezoid weights */
  double vx_min, vx_max, vy_min, vy_max;
  int K;                    /* internal degrees of freedom (Keff = 1 + K)     */
  double Pr;                /* Prandtl number (Shakhov model)                 */
  double omega;             /* viscosity exponent, mu = mu_ref T^omega        */
  double mu_ref;            /* viscosity at T = 1                             */
  double cfl_s;             /* CFL of the flux-averaging step dt_s (0.5)      */
  double cfl_pseudo;        /* CFL of the pseudo time step dt' (100)          */
  double farfield[4];       /* free stream rho, Vx, Vy, T (far-field ghosts)  */
  int shard_iy0, shard_iy1; /* velocity sharding: this context holds the rows
                               shard_iy0 <= iy < shard_iy1 of the velocity
                               grid (k = iy*nvx + ix, whole rows); 0, 0 = all.
                               A sharded context needs ugks_shard_set_exchange */
} ugks_params;

/* One structured block: ni x nj quad cells, nodes (ni+1) x (nj+1).  Cell
 * (i, j) has counter-clockwise nodes (i,j),(i+1,j),(i+1,j+1),(i,j+1); global
 * cell id = (sum of earlier blocks' cells) + j*ni + i.  A periodic block
 * (O-grid, periodic channel) repeats node column 0 as column ni; the
 * difference of the two columns is the period vector (zero for an O-grid). */
typedef struct {
  int ni, nj;
  int periodic_i;           /* 1: i wraps (sides 0 and 1 must be BC_NONE)     */
  int bc[4];                /* UGKS_BC_* per side                             */
  double wall_T[4];         /* wall temperature of BC_WALL sides              */
  int priority;             /* overset: higher wins ties (body grids)         */
  int n_fringe;             /* receptor layers along BC_OVERSET sides         */
  int n_gap;                /* further layers not used to cut holes           */
  const double *x_ref;      /* HOST, (nj+1)*(ni+1)*2 doubles, node (i,j) at
                               2*(j*(ni+1)+i); copied during ugks_init_mesh    */
} ugks_block_desc;

/* Overset assembly counters (Sec. 3.1). */
typedef struct {
  int n_field, n_receptor, n_hole;
  int n_fresh;              /* cells uncovered by the motion (hole -> field),
                               initialised once from donors                   */
  int n_orphan;             /* receptors/fresh cells without donor            */
} ugks_connect_stats;

/* Metrics of one physical step (Sec. 2.2), sums over the solved cells of the
 * last inner iteration, each a fixed-order reduction (the same bits on every
 * run of a mesh):
 *   res_macro_sq  sum |R|^2, R = T_W - Omega^{n+1} W / dt - F / 2 the
 *                 right-hand side of the macro LU-SGS (Step 4, before W is
 *                 updated), 4 components per cell;
 *   res_micro_sq  sum |r|^2 of the micro residual (Step 5) over the cell's
 *                 velocities and both reduced distributions (on a velocity
 *                 shard: over this shard's velocities; add the shards' sums);
 *   fix_sq        sum |W^{s+1} - W'|^2, the Step-7 moment fix of the
 *                 macroscopic predictor (zero once micro and macro agree);
 *   total         sum Omega^{n+1} W over the field cells (mass, momentum,
 *                 energy), for the conservation defect between steps. */
typedef struct {
  double res_macro_sq, res_micro_sq, fix_sq;
  double total[4];
} ugks_step_metrics;

/* Device bytes of the workspace for these parameters and blocks.  Host-only,
 * no CUDA call.  Errors: UGKS_ERR_ARG for invalid sizes or BC combinations. */
int ugks_workspace_query(const ugks_params *p, int nblocks,
                         const ugks_block_desc *blocks, size_t *bytes);

/* Create a context on the current CUDA device.  `workspace` is a DEVICE
 * pointer (>= the queried bytes, 256-byte aligned) owned by the caller and
 * borrowed until ugks_destroy.  `stream` is a cudaStream_t (may be NULL).
 * The mesh is given by ugks_init_mesh.  Errors: UGKS_ERR_ARG,
 * UGKS_ERR_WORKSPACE. */
int ugks_create(const ugks_params *p, void *workspace, size_t bytes,
                void *stream, ugks_ctx **out);
int ugks_destroy(ugks_ctx *ctx);
const char *ugks_last_error(const ugks_ctx *ctx);

/* Upload the blocks (Sec. 2.1 physical discretisation) and the initial state:
 * `prim` is HOST (ncells x 4: rho, Vx, Vy, T per cell); f is set to the
 * reduced Maxwellian of each cell and q to its heat flux.  The mesh is placed
 * at t = 0 with the identity motion; with several blocks an overset assembly
 * at t = 0 is run.  Must match the blocks given to ugks_workspace_query.
 * Synchronises the stream.  Errors: UGKS_ERR_ARG, UGKS_ERR_GEOMETRY,
 * UGKS_ERR_ORPHAN, UGKS_ERR_CUDA. */
int ugks_init_mesh(ugks_ctx *ctx, int nblocks, const ugks_block_desc *blocks,
                   const double *prim);

/* Move the mesh to t_new (Sec. 3 Step 1, prescribed motion): HOST `affine`
 * holds 6 doubles per block (m00, m01, m10, m11, b0, b1) mapping the
 * reference nodes to x = (m00 x + m01 y) + b0, y = (m10 x + m11 y) + b1
 * (FP64, no contraction).  Computes the step's geometry: cell volumes at both
 * levels, mid-time face lengths / normals / centres, face velocities
 * U_f = mean node velocity and S U.n (so Omega^{n+1} - Omega^n =
 * dt sum S U.n), and the explicit flux-averaging step dt_s per cell.  Call
 * once before every ugks_step (identity for a static mesh); a second call
 * before the step replaces the pending move (the old level stays at t).
 * Errors: UGKS_ERR_ARG (t_new <= t), UGKS_ERR_GEOMETRY (some Omega <= 0,
 * detected on the device and reported by the next synchronising call). */
int ugks_move_mesh(ugks_ctx *ctx, double t_new, const double *affine);

/* Overset assembly at t^{n+1} (Sec. 3.1): wall distances, node and cell
 * classification with buffer layer, donor search and inverse-distance
 * weights (Sec. 3.2).  Bit-identical to an FP64 evaluation of the same
 * predicates without fused multiply-add.  The receptor and fresh-cell lists
 * the interpolation walks are compacted on the device (ascending cell
 * order).  `stats` is HOST (may be NULL); synchronises the stream once to
 * read the counters.  No-op for a single block.
 * Errors: UGKS_ERR_ORDER (no move since the last step), UGKS_ERR_ORPHAN,
 * UGKS_ERR_WORKSPACE (more receptors than the staging holds, nc/4 cells
 * but at least min(nc, 1024)). */
int ugks_overset_connect(ugks_ctx *ctx, ugks_connect_stats *stats);

/* One physical step t^n -> t^{n+1} of the implicit unsteady UGKS (Sec. 2.2
 * Steps 1-8): level-n flux and residual, then n_inner inner iterations of
 * {receptor interpolation, flux, macro LU-SGS, micro residual, micro LU-SGS,
 * step-7 moment fix}.  In place on f, W, q.  `dt` must equal t_new - t of
 * the preceding ugks_move_mesh.  Asynchronous.
 * The step's launches (both streams) are captured into a CUDA graph on the
 * first step with a given configuration and replayed by one graph launch on
 * later steps; a change of step size, inner count, tiles or wait limit, and
 * the first step after an assembly that uncovered cells (one more
 * interpolation), select or capture another graph.  Not graphed: while
 * profiling (ugks_profile_enable), on a velocity shard (its exchange runs on
 * the host), after ugks_set_graphs(ctx, 0) or with UGKS_NO_GRAPH=1 in the
 * environment at creation.  Graphed and direct steps issue the same kernels
 * with the same arguments.
 * Errors: UGKS_ERR_ORDER, UGKS_ERR_ARG, UGKS_ERR_CUDA (capture). */
int ugks_step(ugks_ctx *ctx, double dt, int n_inner);

/* Turn the CUDA-graph path of ugks_step on (default) or off.  Errors:
 * UGKS_ERR_ARG (null context). */
int ugks_set_graphs(ugks_ctx *ctx, int on);

/* Record ugks_step_metrics in the steps that follow (on != 0; off at
 * creation).  When on, the last inner iteration of a step runs four small
 * reduction kernels more (on graphs too: a graph of its own).  Errors:
 * UGKS_ERR_ARG. */
int ugks_set_metrics(ugks_ctx *ctx, int on);

/* Metrics of the last ugks_step (HOST output); synchronises the stream.
 * Errors: UGKS_ERR_ORDER (the last step ran with metrics off, or no step
 * yet), UGKS_ERR_ARG (null out). */
int ugks_get_metrics(ugks_ctx *ctx, ugks_step_metrics *out);

/* Graph captures (or updates) and graph replays of ugks_step since creation
 * (HOST outputs, each may be NULL).  Errors: UGKS_ERR_ARG. */
int ugks_graph_stats(const ugks_ctx *ctx, int64_t *captures, int64_t *replays);

/* Batched outer loop over n independent contexts ("instances": different
 * meshes, velocity grids and gases): for each instance i, ugks_move_mesh to
 * t_new[i] with the HOST map affine[i] (6 doubles per block of instance i),
 * the overset assembly, and ugks_step with dt = t_new[i] - t and n_inner
 * inner iterations.  Work is issued stage by stage across the instances
 * (all motions, all assemblies, all steps) and never waits on the device:
 * the assembly counters stay on the device and the interpolation reads them
 * there, so instances created on distinct streams run concurrently on the
 * GPU while the host returns at once.  Each instance computes what a
 * separate ugks_move_mesh / ugks_overset_connect / ugks_step sequence
 * computes (the face sums' atomic additions may land in another order).
 * Orphans, staging overflow and non-physical states are reported by the
 * next synchronising call on the instance (ugks_moments).  `failed` (HOST,
 * may be NULL) receives the index of the instance whose call failed, or -1.
 * Errors: UGKS_ERR_ARG, UGKS_ERR_ORDER, and those of ugks_move_mesh and
 * ugks_step. */
int ugks_advance_batch(ugks_ctx *const *ctx, int n, const double *t_new,
                       const double *const *affine, int n_inner, int *failed);

/* Torque of each block's wall force about the point center[b] (HOST,
 * nblocks x 2): sum over the block's wall faces of (x_f - center) x (S F_x,
 * S F_y) of the last flux evaluation, x_f the mid-time face centre; with the
 * force of ugks_moments it drives a rigid body's Newton-Euler update (Sec. 3
 * Step 1).  `torque` (nblocks doubles, host or device) receives the values.
 * Synchronises the stream.  Errors: UGKS_ERR_ORDER, UGKS_ERR_ARG. */
int ugks_wall_torque(ugks_ctx *ctx, const double *center, double *torque);

/* Tile autotuner, on the context's own state (`reps` timed passes after one
 * warm-up of each candidate, CUDA events on the stream), keeping the fastest:
 *  - the face kernels (velocity reduction and flux divergence, FP32 paths):
 *    their tile of 8x8 cells walks the velocities in chunks of `face_vk` in
 *    {8, 16, 32} with `face_nh` = 2 threads per face slot (each takes
 *    face_vk / face_nh velocities of a chunk); the FP64 path keeps (8, 2);
 *  - the micro LU-SGS sweeps, skewed wavefronts (a warp takes a band of 8
 *    rows, 4 lanes a row; 16 rows, 2 lanes a row when a block is taller than
 *    256 cells): velocities per lane `vpt` in {2, 4} (FP32 paths; 2 in FP64)
 *    and, per sweep, the prefetch ring depth in {2, 4, 6} steps (shallower
 *    where shared memory is short).
 * The candidates differ only in the grouping of the FP32 face sums over the
 * velocities (partial sums per thread and chunk, folded error-free), i.e. in
 * rounding; the sweeps take each velocity in the same lexicographic order.  f is saved before the trials and restored after them.  Needs
 * a preceding ugks_step (the kernels read records the step writes).  `items`
 * (the (cell, velocity) items of one sweep warp step, 32 x vpt), `vpt`,
 * `ring_fwd`, `ring_bwd`, `face_vk`, `face_nh` (HOST, each may be NULL)
 * receive the choice.  Synchronises the stream.  Errors: UGKS_ERR_ORDER,
 * UGKS_ERR_CUDA. */
int ugks_autotune(ugks_ctx *ctx, int reps, int *items, int *vpt, int *ring_fwd, int *ring_bwd, int *face_vk,
                  int *face_nh);

/* Copy the macroscopic fields to caller memory (host or device pointers,
 * cudaMemcpyDefault): W (ncells x 4: rho, rho Vx, rho Vy, rho E), q
 * (ncells x 2), status (ncells int32, UGKS_FIELD/RECEPTOR/HOLE) -- any may be
 * NULL -- and wall_loads (nblocks x 4 doubles: sum over the block's wall faces
 * of S times the wall macro flux (mass, x-momentum, y-momentum, energy) of
 * the last flux evaluation, i.e. the force and heat the gas exerts, Sec. 2.1
 * wall pressure/shear/heat).  Synchronises the stream.  Also reports a
 * pending device error flag: UGKS_ERR_NONPHYSICAL, UGKS_ERR_GEOMETRY, and
 * from an assembly issued by ugks_advance_batch UGKS_ERR_ORPHAN or
 * UGKS_ERR_WORKSPACE. */
int ugks_moments(ugks_ctx *ctx, double *W, double *q, int32_t *status,
                 double *wall_loads);

/* Sizes of the current problem. */
int ugks_sizes(const ugks_ctx *ctx, int *ncells, int *nfaces, int *nv,
               int *nv_stride);

/* Read / write the distribution f (ncells x nv x 2, FP64, host or device
 * pointer, velocity index k = iy*nvx + ix) and W, q (FP64).  get synchronises
 * the stream; set overwrites the state (any pointer may be NULL). */
int ugks_get_state(ugks_ctx *ctx, double *f, double *W, double *q);
int ugks_set_state(ugks_ctx *ctx, const double *f, const double *W, const double *q);

/* Checkpoint of what a context carries from one physical step to the next
 * besides f, W and q (ugks_get_state / ugks_set_state): the time t, the node
 * coordinates at t (nnodes x 2 FP64, nnodes = sum over blocks of
 * (ni + 1)(nj + 1) in block order, the layout of ugks_init_mesh) and the cell
 * status of the last assembly (ncells int32; the next assembly's previous
 * status, from which it finds uncovered cells).  Everything else a step uses
 * is recomputed by the next ugks_move_mesh / ugks_overset_connect, so a
 * context restored from (f, W, q, t, nodes, status) continues bit for bit as
 * the one the checkpoint was taken from.  Only between steps (no pending
 * move).  Until that next step, the geometry, connectivity and wall-load
 * accessors still describe this context's own last step.  `t`, `nodes`, `status` are HOST (each may be NULL on get);
 * ugks_get_checkpoint synchronises the stream.  Errors: UGKS_ERR_ORDER (a
 * move is pending), UGKS_ERR_ARG (null input on set). */
int ugks_get_checkpoint(ugks_ctx *ctx, double *t, double *nodes, int32_t *status);
int ugks_set_checkpoint(ugks_ctx *ctx, double t, const double *nodes, const int32_t *status);

/* Diagnostic of Steps 1/3: evaluate the time-averaged interface flux of the
 * current state with the current geometry (after ugks_move_mesh) and write
 * D = sum_faces S F_hat (ncells x nv x 2, outward positive, Eq.
 * microscopicFlux summed per cell) and F = sum_k V_k Psi_k D_k (ncells x 4,
 * Eq. macroscopicFlux) to caller memory (host or device, FP64).  Receptors are
 * interpolated first.  Synchronises the stream. */
int ugks_eval_flux(ugks_ctx *ctx, double *D, double *F);

/* Connectivity of the last assembly, HOST buffers: status (ncells int32),
 * donors (ncells x 5 int32, -1 unused; rows of non-receptors are -1) and
 * weights (ncells x 5 doubles).  Synchronises the stream. */
int ugks_get_connectivity(ugks_ctx *ctx, int32_t *status, int32_t *donors,
                          double *weights);

/* Geometry of the last move, HOST buffers (any may be NULL): vol_old,
 * vol_new (ncells), xc (ncells x 2, mid-time centres), dts (ncells),
 * Sn (nfaces x 2), SUn (nfaces).  Face order, block after block: the
 * i-faces row by row (j outer, i inner; a periodic block has ni per row, the
 * first joining cell ni-1 to cell 0), then the j-faces column by column (i
 * outer, j = 0..nj inner).  Interior faces point from the lower to the higher
 * logical index; boundary faces point out of the block. */
int ugks_get_geometry(ugks_ctx *ctx, double *vol_old, double *vol_new,
                      double *xc, double *dts, double *Sn, double *SUn);

/* Velocity-space sharding (the per-velocity work of a step -- flux
 * divergence, residual, both LU-SGS sweeps, interpolation -- is independent
 * per discrete velocity, Sec. 2.2; only velocity sums couple velocities).  A
 * context created with shard_iy0 < shard_iy1 holds those rows of the velocity
 * grid.  Twice per flux evaluation / inner iteration it needs the sums over
 * all shards of a buffer of partial velocity sums, and asks for them through
 * the caller's exchange function:
 *   which 0: the per-face sums of the velocity reduction (W0 and the f-parts
 *            of the macro flux), face_count doubles;
 *   which 1: the per-cell partial sums of the step-7 moment fix and of the
 *            heat flux, cell_count doubles.
 * fn(which, stream, user) is called on the host; the buffer's partial sums
 * are complete once `stream` (a cudaStream_t) has reached the call point.  It
 * must replace the buffer, in stream order, by the sum over all shards of the
 * same buffer -- the same bits on every shard (a fixed summation order) --
 * before it returns or through work it enqueues on `stream`, and return 0;
 * anything else fails the calling ugks_* function with UGKS_ERR_ARG.  All
 * other quantities (face states, equilibrium and wall fluxes, macroscopic
 * update, geometry) are computed identically on every shard.  Errors:
 * UGKS_ERR_ARG (context not sharded or fn NULL). */
typedef int (*ugks_exchange_fn)(int which, void *stream, void *user);
int ugks_shard_set_exchange(ugks_ctx *ctx, ugks_exchange_fn fn, void *user);

/* Where the two exchange buffers of a sharded context lie: byte offsets from
 * the start of the caller's workspace and lengths in doubles (FP64). */
int ugks_shard_buffers(const ugks_ctx *ctx, size_t *face_off, size_t *face_count, size_t *cell_off,
                       size_t *cell_count);

/* Number of kernel launches issued on the context's stream since creation
 * (counted on the host at each launch). */
int64_t ugks_launch_count(const ugks_ctx *ctx);

/* Bounded waits.  The only device-side waits of a step are those of the
 * wavefront sweeps: the macro LU-SGS CTA waits (mbarrier) for the bulk copy of
 * the next diagonal's records, the bands of a micro-sweep CTA wait for the
 * band before them (shared-memory progress counters, Sec. 2.2 sweep order).
 * Each wait polls at most `polls` times (0 restores the default, 2^21); a wait
 * that runs out sets a flag, the CTA stops its sweep at the end of the
 * current step, waits (default bound) for every copy it issued, and exits;
 * the step's results are then invalid and the next synchronising call
 * returns UGKS_ERR_TIMEOUT (and clears the flag, leaving the context usable:
 * set a valid state with ugks_set_state before stepping again).  Takes effect
 * for work issued after the call.  Errors: UGKS_ERR_ARG (polls < 0). */
int ugks_set_wait_limit(ugks_ctx *ctx, int polls);

/* Kernel groups timed by the profiler (CUDA events around every launch of the
 * group, on the stream it is launched on: the context's stream, or for the
 * macro sweep the library's internal side stream that overlaps it with the
 * flux kernel). */
#define UGKS_PROF_GEOMETRY    0   /* mesh motion, geometry, dt_s, slope geometry */
#define UGKS_PROF_CONNECT     1   /* overset assembly kernels                    */
#define UGKS_PROF_INTERP      2   /* receptor / fresh-cell interpolation          */
#define UGKS_PROF_CELL        3   /* ghost states, W gradients, per-cell records  */
#define UGKS_PROF_FACE_REDUCE 4   /* per-face velocity reduction (W0, flux parts) */
#define UGKS_PROF_FACE_COEF   5   /* per-face interface coefficients              */
#define UGKS_PROF_MACRO_SWEEP 6   /* macro LU-SGS                                 */
#define UGKS_PROF_MICRO_FWD   7   /* micro LU-SGS forward sweep                   */
#define UGKS_PROF_MICRO_BWD   8   /* micro backward sweep and update              */
#define UGKS_PROF_MOMENTS     9   /* step-7 moment fix and heat flux              */
#define UGKS_PROF_RHS        10   /* flux divergence (Step 3), tiled             */
#define UGKS_PROF_RESIDUAL   11   /* micro residual (Step 5)                      */
#define UGKS_NPROF           12

/* Start (on != 0) or stop per-group event timing.  While on, every launch is
 * bracketed by two cudaEventRecord calls (events are created on demand and
 * reused; no device memory).  Stopping drains the pending events. */
int ugks_profile_enable(ugks_ctx *ctx, int on);

/* Synchronise the stream and return, per group, the summed device time in ms
 * and the number of timed launches since the last reset (HOST arrays of
 * UGKS_NPROF entries, either may be NULL); reset != 0 clears the totals. */
int ugks_profile_read(ugks_ctx *ctx, double *ms, int64_t *launches, int reset);

/* FP64 throughput probe (measurement, no counterpart in the paper): the FP64
 * path of the scheme is bound by the FP64 pipe of the GPU, so its roofline is
 * the measured FP64 rate.  kind 0: nblocks x nthreads threads each run 8
 * independent fused-multiply-add chains for `iters` rounds (16 * iters flops
 * a thread); kind 1: 4 independent exp chains (4 * iters exponentials a
 * thread).  `out` is a DEVICE buffer of nblocks * nthreads doubles (the
 * results, so no work is dead).  Asynchronous on `stream`; the caller times
 * it with events on that stream.  Errors: UGKS_ERR_ARG, UGKS_ERR_CUDA. */
int ugks_probe_fp64(double *out, int kind, int nblocks, int nthreads, int iters, void *stream);

/* Allocation-free receptor interpolation.  No counterpart in the paper: it
 * exists for callers that cannot allocate device memory at all (a host
 * framework that owns every device allocation, or code that must not call
 * cudaMalloc while other work is being captured or replayed), not even the
 * workspace of ugks_create.  It performs the inverse-distance interpolation
 * of the receptor rows that ugks_step / ugks_eval_flux apply before each
 * flux evaluation, on caller buffers, staging the interpolated values in a
 * fixed scratch array of UGKS_STATIC_SCRATCH_DOUBLES doubles (4 MiB) that
 * the library holds as a static device variable on every GPU that loads it,
 * until the process exits.
 *
 * Arguments (all DEVICE pointers, FP64): f (ncells x nv x 2, the (h, b)
 * pairs of every cell, k = iy*nvx + ix), W (ncells x 4) and q (ncells x 2)
 * updated in place (W and q may be NULL); receptors: nrec cell ids whose rows
 * are overwritten; donors / weights: nrec x 5 stencils and weights, row r for
 * receptors[r], donor -1 unused (the layout of ugks_get_connectivity rows).
 * A row whose first donor is -1 is left unchanged (an orphan).  Donor ids
 * outside [0, ncells) other than -1 are skipped and the remaining weights of
 * that row are renormalised to their sum; a row with no valid donor left,
 * and a row whose receptor id lies outside [0, ncells), is left unchanged.
 * Every receptor reads its donors' values from before the call (Jacobi).
 * stream: a cudaStream_t (NULL = default).  Asynchronous; allocates nothing
 * and calls no allocating routine.
 *
 * Errors: UGKS_ERR_ARG when a pointer is NULL or
 * 2*nrec*nv + 7*nrec > UGKS_STATIC_SCRATCH_DOUBLES (nothing is launched);
 * UGKS_ERR_CUDA when the device lookup of the scratch or a launch fails.
 * The first call in each CUDA context looks up the scratch address with
 * cudaGetSymbolAddress (with that context's device current; a device reset
 * creates a new context and the next call looks the address up again); make
 * that first call before any stream capture.  All calls on a device share
 * the one scratch array, which keeps the last call's contents: calls that
 * overlap on the GPU (different streams, no ordering between them) race. */
#define UGKS_STATIC_SCRATCH_DOUBLES (1 << 19)
int ugks_idw_interpolate_static(double *f, double *W, double *q, int ncells, int nv,
                                const int32_t *receptors, int nrec,
                                const int32_t *donors, const double *weights,
                                void *stream);

#ifdef __cplusplus
}
#endif
#endif /* UGKS_H */

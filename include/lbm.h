/*
 * lbm.h -- C ABI of the GB300 lattice Boltzmann-BGK library (liblbm.so).
 *
 * The library runs the time step of the LBGK method of Colosqui, Karabacak, Ekinci & Yakhot,
 * "Lattice Boltzmann simulation of high-frequency flows: electromechanical resonators in gaseous
 * media" (2009), Sec. 5: advection (Eq. 17), moments (Eq. 16), Hermite equilibrium (Eq. 15),
 * regularized BGK collision (Eqs. 18-19), with bounce-back walls (Eq. 12) that move with
 * U_w = u0 sin(omega t) x (Sec. 6, "Fluid-solid interaction") or, in the body frame, a uniform
 * body force rho u0 omega cos(omega t) x on the fluid.  Each step also records the force on the body
 * by momentum exchange, in FP64; fitting it to sin/cos gives the dissipative and inertial parts of
 * the fluid force F_f of Eq. 1 and the normalized damping of Eq. 20.
 *
 * Units and conventions (all calls).
 *   - Lattice units: dx = dt = 1, lattice speed 1.  theta = c_s^2 = 1/1.19697977039307^2 for D2Q37
 *     (Appendix A, Table "D2Q37"), 1/3 for D2Q9 (textbook lattice, not in the paper).
 *   - tau is the LBGK relaxation time in steps (tau > 1/2); the physical nondimensional frequency
 *     of Sec. 6 is (tau - 1/2) * omega, because nu = theta (tau - 1/2) and tau_phys = nu / theta.
 *   - The wall velocity and body force of step n -> n+1 are taken at t = n + 1/2; the force of
 *     step n is stamped at the same time.
 *   - Grids are periodic in x and y.  Walls are solid nodes inside the box (labels, below).
 *   - Direction order: index 0 is the rest velocity; (1 + 2k, 2 + 2k) are +c and -c of pair k.
 *     lbm_lattice_velocities() returns the table.
 *   - Every call returns 0 on success or a negative LBM_E* code; lbm_last_error() then holds a
 *     message for the calling thread.  No call aborts the process.
 *   - All device memory of a simulation is allocated by lbm_create() and freed by lbm_destroy().
 *     Host buffers passed in are owned by the caller and are not kept after the call returns.
 *   - A simulation is used by one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_EINVAL (-1)      /* bad argument: tau <= 1/2, u0 >= omega, grid too small, ...     */
#define LBM_ENOMEM (-2)      /* device or host allocation failed                                 */
#define LBM_ECUDA (-3)       /* a CUDA call failed (message in lbm_last_error)                   */
#define LBM_ETIMEOUT (-4)    /* a bounded device wait gave up                                    */
#define LBM_ENONFINITE (-5)  /* the force became NaN or Inf: the run diverged                    */
#define LBM_ERANGE (-6)      /* index or size out of range                                       */

typedef struct lbm_sim lbm_sim; /* opaque; owned by the library */

enum { LBM_D2Q9 = 9, LBM_D2Q37 = 37 };
enum { LBM_GEOM_PLATE = 0, LBM_GEOM_BEAM = 1, LBM_GEOM_MASK = 2, LBM_GEOM_NONE = 3 };
enum { LBM_DRIVE_WALL = 0, LBM_DRIVE_BODYFORCE = 1 };
enum { LBM_COLL_BGK = 0, LBM_COLL_REGULARIZED = 1 };
enum { LBM_STORE_F64 = 0, LBM_STORE_F32 = 1, LBM_STORE_BF16 = 2, LBM_STORE_F16 = 3 };

/* Gas-wall interaction (lbm_geometry.wall_scheme).  Bounce-back (Eq. 12): a population sent into
 * a wall comes back reversed, plus 2 w_i rho0 c_i.U_w / theta for a moving wall (no slip).
 * Diffuse scattering (Eq. 11): the populations a wall returns to a node along its blocked links are
 * the wall's discrete Maxwellian (the equilibrium of the run's order at the wall velocity), with
 * the density that returns exactly the mass the node sent into that wall (fully accommodating
 * surface; the gas slips).  In free-molecular flow the diffuse force is half the bounce-back one. */
enum { LBM_SCHEME_BOUNCEBACK = 0, LBM_SCHEME_DIFFUSE = 1 };

/* Population storage layout (lbm_geometry.layout).  LBM_LAYOUT_AB: two buffers, each step pulls
 * from one into the other (Eq. 17).  LBM_LAYOUT_AA: one buffer updated in place; even steps pull
 * from the neighbours and push to them, odd steps read and write only the node itself (the "AA"
 * pattern).  Same results up to the rounding of the storage type; half the population memory.
 * AA runs the plain kernel only (lbm_set_variant 0) with bounce-back walls and is not available in
 * the persistent batch mode; lbm_get_state / lbm_set_state need an even number of steps done
 * (LBM_ERANGE otherwise).  lbm_step_noalloc always runs the two-buffer step on the caller's
 * buffers, whatever the simulation's layout. */
enum { LBM_LAYOUT_AB = 0, LBM_LAYOUT_AA = 1 };

/* Node labels of a geometry (LBM_GEOM_MASK input, lbm_get_labels output). */
enum { LBM_FLUID = 0, LBM_BODY = 1, LBM_WALL = 2 };

typedef struct {
    int kind;                  /* LBM_GEOM_*                                                       */
    int lx, ly;                /* BEAM: section lx nodes along the motion (x), ly across (y),
                                  centred in the box, AR = ly/lx (Sec. 3).  Others: ignored.        */
    int drive;                 /* LBM_DRIVE_WALL: label-1 nodes move with U_w = u0 sin(omega t) x;
                                  LBM_DRIVE_BODYFORCE: body frame, fluid force rho u0 omega
                                  cos(omega t) x, all walls static.                                 */
    double u0;                 /* drive amplitude, 0 <= u0 < omega (Sec. 6: U_0 < omega dx)        */
    double rho0;               /* rest density (> 0; 1 if 0 is passed)                            */
    const unsigned char* mask; /* MASK: ny*nx row-major labels (0 fluid, 1 body, 2 static wall),
                                  copied; solids must be at least the lattice reach (1 for D2Q9,
                                  3 for D2Q37) thick, or links tunnel through them                 */
    int eq_order;              /* 2 (Eq. 15) or 4 (Hermite continuation); D2Q9 requires 2         */
    int collision;             /* LBM_COLL_REGULARIZED (Eqs. 18-19) or LBM_COLL_BGK (Eq. 14)      */
    int storage;               /* LBM_STORE_*: population storage type; arithmetic is FP64 for F64
                                  and FP32 otherwise; the force is accumulated in FP64              */
    int wall_scheme;           /* LBM_SCHEME_BOUNCEBACK (0, default) or LBM_SCHEME_DIFFUSE          */
    int layout;                /* LBM_LAYOUT_AB (0, default) or LBM_LAYOUT_AA                       */
} lbm_geometry;

/*
 * Create a simulation on the current CUDA device: nx * ny nodes of lattice Q (LBM_D2Q9 or
 * LBM_D2Q37), relaxation time tau, drive angular frequency omega (rad/step), geometry `geom`.
 * PLATE: the bottom R rows are the plate (label 1), the top R rows a static wall (label 2), R the
 * lattice reach.  BEAM: an lx x ly body.  NONE: a periodic box with no solid.  The fluid starts at
 * rest, f_i = w_i rho0 (step 0).  Requires nx, ny >= 2R + 1.  *out receives the handle.
 * Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA.
 */
int lbm_create(int lattice, int nx, int ny, double tau, double omega, const lbm_geometry* geom, lbm_sim** out);

/* Enqueue n >= 0 time steps on the simulation's stream (asynchronous: returns before they run). */
int lbm_step(lbm_sim* sim, long n);

/* Wait for all enqueued steps; reports LBM_ENONFINITE if the force has become NaN/Inf. */
int lbm_synchronize(lbm_sim* sim);

/*
 * Copy the force history to host memory: out_xy[2k], out_xy[2k+1] = (Fx, Fy) on the body (label 1)
 * during step k, FP64, for k < min(cap_steps, steps done).  *n_steps receives the number of steps
 * done.  Synchronizes the stream first.
 */
int lbm_force_history(lbm_sim* sim, double* out_xy, size_t cap_steps, size_t* n_steps);

/*
 * Least-squares fit Fx(t_n) = A sin(omega t_n) + B cos(omega t_n) + C over the steps after the
 * first `skip_periods` periods (t_n = n + 1/2).  The body velocity is V(t) = s u0 sin(omega t) with
 * s = +1 for the wall drive and s = -1 in the body frame (where the fluid force equals -dV/dt), so
 * f_in = s A is the force part in phase with V (the dissipative part of F_f in Eq. 1) and
 * f_q = s B the part in phase with dV/dt (inertial); f_0 = C.  Any output pointer may be NULL.
 * Errors: LBM_ERANGE if fewer than one period remains after the skip.
 */
int lbm_fit(lbm_sim* sim, double skip_periods, double* f_in, double* f_q, double* f_0);

/* Normalized damping of Eq. 20 per unit length: -f_in / (u0 rho0 sqrt(theta/2) perimeter). */
int lbm_gamma_bar(lbm_sim* sim, double f_in, double perimeter, double* gamma_bar);

/* Free all memory of the simulation (waits for its work).  NULL is allowed. */
void lbm_destroy(lbm_sim* sim);

/* Message of the last failed call on this thread ("" if none). */
const char* lbm_last_error(void);

/* Run the simulation's work on `stream` (a cudaStream_t owned by the caller, who keeps it alive
 * until lbm_destroy or the next lbm_set_stream; 0 is the CUDA default stream).  Work already
 * enqueued is completed first.  Until this is called the simulation uses a private stream. */
int lbm_set_stream(lbm_sim* sim, void* stream);

/*
 * Deviations g_i = f_i - w_i rho0 of the current post-collision state, FP64, as count = Q*ny*nx
 * values in [Q][ny][nx] order (direction order of lbm_lattice_velocities).  Synchronizes.
 */
int lbm_get_state(lbm_sim* sim, double* out, size_t count);

/* Overwrite the current state with deviations g (same layout as lbm_get_state), rounded to the
 * storage type.  Values at solid nodes are ignored (solid nodes hold g = 0).
 * Storage convention: the device holds h_i = (f_i - w_i rho0) / (w_i s), s = u0 for 16-bit storage
 * and 1 otherwise; 16-bit runs with the body-force drive store h_i - H_i(n) instead, H_i(n) being
 * h_i of the equilibrium at rho0 of the uniform stream U(n) = sum_{k<n} u0 omega cos(omega (k+1/2))
 * (the flow the body force sets up far from the body), so that the stored values, and their
 * rounding errors, are small away from the body.  lbm_get_state and lbm_set_state convert. */
int lbm_set_state(lbm_sim* sim, const double* g, size_t count);

/* Node labels (ny*nx, row-major) the simulation runs with. */
int lbm_get_labels(lbm_sim* sim, unsigned char* out, size_t count);

typedef struct {
    int lattice, nx, ny, pitch;  /* pitch: elements per stored row                               */
    int storage, collision, eq_order, drive;
    double tau, omega, u0, rho0, theta;
    long steps_done;
    size_t n_fluid, n_boundary;  /* fluid nodes; fluid nodes with at least one blocked link     */
    size_t bytes_per_step;       /* algorithmic HBM bytes of one step: 2 Q sizeof(storage) n_fluid */
    size_t device_bytes;         /* device memory held by the simulation                          */
    int block_x, block_y;        /* tile shape of the step kernel                                  */
    size_t h2d_bytes, d2h_bytes; /* host<->device bytes copied by the library so far               */
    int variant;                 /* step kernel in use, see lbm_set_variant                        */
    int layout;                  /* LBM_LAYOUT_AB or LBM_LAYOUT_AA                                 */
    int force_1e4;               /* 1 if this storage type meets a force error of 1e-4 of the force
                                    amplitude (in-phase and quadrature, against FP64) in the library's
                                    precision study: FP64, FP32 and FP16; 0 for BF16, whose 8-bit
                                    significand gives about 1.5e-3 on the 256^2 beam               */
} lbm_info_t;

int lbm_info(lbm_sim* sim, lbm_info_t* out);

/* Use the plain step kernel (variant 0) with this tile (block_x a multiple of 32,
 * block_x * block_y <= 512).  Results do not depend on the tile, except for the order in which the
 * FP64 force partials of the tiles are summed. */
int lbm_set_tile(lbm_sim* sim, int block_x, int block_y);

/* Choose the step kernel.  0: plain kernel, one block per tile of lbm_set_tile's shape, wrapped
 * global loads.  1, 2: the plain kernel on 32 x 4 tiles compiled for at least 6 (1) or 7 (2)
 * resident blocks per SM (fewer registers, more warps to hide load latency; D2Q37, FP32/BF16/FP16
 * storage); 3, 4: 7 blocks per SM, each thread computing 2 or 4 nodes of its column (tiles of
 * 32 x 8 or 32 x 16 nodes).  lbm_create starts D2Q37 two-buffer bounce-back runs on variant 1 (FP32) or 2
 * (16-bit), the fastest single-instance kernels measured; lbm_set_tile selects variant 0.
 * Staged kernels (FP32/BF16/FP16 storage), whose interior tiles are copied to shared memory by
 * bulk tensor copies (TMA), one box per direction plane:
 * 10, 11, 12: one node per thread, one block per tile of 32 x 4, 64 x 2 or 64 x 4 nodes;
 * 13: as 11, with the outputs of interior tiles staged in shared memory and written by one bulk
 * tensor store per direction plane (D2Q37);
 * 18, 23, 24, 25, 26, 27: several nodes per thread, one row apart, on blocks of 64 x 1 (4 rows, at
 * least 12 blocks per SM), 64 x 1 (2 rows), 64 x 1 (4 rows, 10 blocks), 128 x 1 (2 rows), 64 x 1
 * (3 rows, 12 blocks), 64 x 1 (3 rows, 11 blocks) threads (D2Q37);
 * 20: two neighbouring nodes per thread with paired loads and stores, 64 x 4 tiles (D2Q9).
 * Every variant evaluates the same expressions in the same order; results agree to FP32 rounding
 * (the compiler may contract them into different fused multiply-adds in different kernels) and the
 * force also by the order in which tile partials are summed when the tile shape differs.
 * LBM_EINVAL if the variant is not built for the simulation's storage type. */
int lbm_set_variant(lbm_sim* sim, int variant);

/* One candidate of the autotuner: kernel variant (0 = plain kernel with tile block_x x block_y) and
 * its measured time per step. */
typedef struct {
    int variant, block_x, block_y;
    double us_per_step;
} lbm_tune_entry;

/* Time every step-kernel candidate built for the simulation's lattice/storage/collision (plain
 * kernel tiles and staged variants) for `steps` steps each, on a clone of the simulation (same
 * geometry, parameters and storage; the simulation itself is not advanced).  Fills up to cap
 * entries of out and sets *n to the number timed.  Needs device memory for the clone. */
int lbm_tune(lbm_sim* sim, int steps, lbm_tune_entry* out, int cap, int* n);

/* lbm_tune, then switch the simulation to the fastest candidate (reported in *best if not NULL). */
int lbm_autotune(lbm_sim* sim, int steps, lbm_tune_entry* best);

/* Velocity table of a lattice in the library's direction order: c_xy[2i], c_xy[2i+1], w[i], theta.
 * Any output may be NULL.  Returns Q, or LBM_EINVAL. */
int lbm_lattice_velocities(int lattice, int* c_xy, double* w, double* theta);

/* Node classes and blocked-link masks of a geometry on an nx x ny periodic grid, computed on the
 * host (no GPU, no simulation): the wall rule of Eq. 12 as lbm_create applies it.  Link i of a
 * fluid node is blocked when its pull source, or a lattice node strictly between source and node,
 * is solid; the first solid node met walking back from the node makes it a body link (label
 * LBM_BODY: bit i of body) or a static-wall link (bit i of wall).  cls: 0 bulk fluid, 1 solid, 2
 * fluid with a blocked link.  Outputs are ny*nx row-major; any may be null; count: the elements
 * each non-null output holds (at least nx*ny).  n_fluid, n_boundary (may be null): the counts
 * lbm_info reports.  Reads the geometry's kind, lx, ly and mask only.  LBM_EINVAL for a bad
 * lattice, grid, geometry kind or a short output. */
int lbm_geometry_links(int lattice, int nx, int ny, const lbm_geometry* geom, unsigned char* cls,
                       unsigned long long* body, unsigned long long* wall, size_t count, size_t* n_fluid,
                       size_t* n_boundary);

/*
 * Lattice parameters for a nondimensional frequency tau_omega = (tau - 1/2) omega (Sec. 6:
 * tau = mu/p = nu/theta): the period is P = max(p_min, ceil(2 pi delta_min / sqrt(2 theta
 * tau_omega))) steps, which puts delta_min nodes in the Stokes layer sqrt(2 nu/omega); then
 * omega = 2 pi / P and tau = 1/2 + tau_omega / omega.  Outputs may be NULL.
 */
int lbm_params_from_tau_omega(int lattice, double tau_omega, double delta_min, int p_min, double* tau,
                              double* omega, int* period);

/* ----------------------------------------------------------------------------------------------
 * Batches: many simulations of uneven sizes (a tau*omega and aspect-ratio sweep, or the requests
 * of a server) advanced together.  All instances of a batch share the lattice, storage type and
 * collision; each has its own grid, geometry, tau, omega, drive and length in steps (the tau*omega
 * and aspect-ratio sweep of Sec. 6).  In the persistent mode a run of K steps is one launch of a
 * persistent kernel, replayed through a CUDA graph (built once per grid size): its blocks take
 * (step, strip) items of every running instance from a queue in step order (a strip: one tile
 * column of a band of tile rows, lbm_batch_set_segment), and a strip waits only for the bands of
 * its own instance within the lattice reach of its band to have finished the previous step --
 * there is no grid-wide barrier, and steps of different instances (and of distant bands of one
 * instance) overlap.  Each wait is bounded (about 2 s by default); a wait that runs out sets
 * an error flag, the kernel returns, and lbm_batch_synchronize reports LBM_ETIMEOUT.  In both modes
 * every instance's arithmetic is that of lbm_step on the same instance with the same tile shape.
 * ---------------------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch; /* opaque; owned by the library */

/* How a batch runs its instances (lbm_batch_set_mode):
 *   LBM_BATCH_STREAMS     every instance step is a launch of the single-instance kernel (the
 *                         fastest variant for the storage type) on one of several parallel
 *                         streams, so that instances of different sizes overlap (the default);
 *   LBM_BATCH_PERSISTENT  one launch per run of the persistent kernel over all instances' tiles
 *                         for K steps (per-band step counters, no grid barrier), replayed through
 *                         a CUDA graph: staged 64 x 3 tiles (the shape of variant 27) with 16-bit
 *                         storage, plain 32 x 4 tiles otherwise (lbm_batch_set_variant). */
enum { LBM_BATCH_STREAMS = 0, LBM_BATCH_PERSISTENT = 1 };

/* One instance: the arguments of lbm_create plus the number of steps to run. */
typedef struct {
    int lattice, nx, ny;
    double tau, omega;
    lbm_geometry geom;
    long nsteps;
} lbm_instance_desc;

typedef struct {
    int lattice, storage, collision;
    int live, running;             /* instances held; instances with steps left                */
    size_t fluid_running;          /* fluid nodes of the running instances                     */
    size_t bytes_per_step;         /* algorithmic HBM bytes of one batch step of those          */
    long long batch_steps, launches;
    double lattice_updates;        /* fluid-node updates enqueued so far                        */
    size_t budget_bytes, used_bytes;
    int max_blocks;                /* resident blocks of the persistent kernel on the whole GPU */
    int uses_graph;                /* 1 if runs are replayed through a CUDA graph               */
    int block_x, block_y;
    int mode;                      /* LBM_BATCH_STREAMS or LBM_BATCH_PERSISTENT                 */
} lbm_batch_info_t;

/* New empty batch on the current device.  device_budget_bytes caps the device memory its instances
 * may hold (0: free memory at creation minus 1 GiB).  Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
int lbm_batch_create(int lattice, int storage, int collision, size_t device_budget_bytes, lbm_batch** out);

/* Device bytes an instance would hold in a batch (admission by footprint). */
int lbm_batch_footprint(const lbm_instance_desc* desc, size_t* bytes);

/* Add an instance; it starts at rest with the next run.  *slot receives its index.
 * LBM_ENOMEM if its footprint does not fit the budget left (nothing is allocated then). */
int lbm_batch_add(lbm_batch* batch, const lbm_instance_desc* desc, int* slot);

/* Enqueue `steps` batch steps (asynchronous): every instance with steps left advances by up to
 * `steps`; an instance stops after its own nsteps. */
int lbm_batch_run(lbm_batch* batch, long steps);

/* Wait for the enqueued runs.  LBM_ETIMEOUT if a wait of the persistent kernel gave up (the
 * states are then undefined). */
int lbm_batch_synchronize(lbm_batch* batch);

/* Steps enqueued for an instance and its length. */
int lbm_batch_status(lbm_batch* batch, int slot, long* steps_done, long* nsteps);

/* The simulation behind a slot (NULL if none), for lbm_force_history, lbm_fit, lbm_get_state,
 * lbm_set_state (before the first run) and lbm_info; owned by the batch. */
lbm_sim* lbm_batch_instance(lbm_batch* batch, int slot);

/* Free an instance's memory (waits for the batch's stream). */
int lbm_batch_remove(lbm_batch* batch, int slot);

/* Choose the mode (before the first lbm_batch_add); the persistent mode picks its kernel here. */
int lbm_batch_set_mode(lbm_batch* batch, int mode);

/* Step kernel of the instances added after this call, in the streams mode (lbm_set_variant
 * numbers; -1, the default: for D2Q37 the staged variant 27 with 16-bit storage and variant 2 with
 * FP32; for 16-bit D2Q9 the four-nodes-per-thread variant 30; else the plain kernel on 32 x 4
 * tiles).  An
 * instance whose layout or wall scheme the variant does not support falls back to the plain
 * kernel.  In the persistent mode (before the first lbm_batch_add) it picks the tile code the
 * persistent kernel runs: 27 staged 64 x 3 tiles, 28 staged 128 x 3 (D2Q37), 2 plain 32 x 4
 * (D2Q37 FP32/16-bit), 0 plain 32 x 4 (the others), -1 the default of the class (27 with 16-bit
 * storage, else 2 or 0); a number the class does not build is LBM_EINVAL there.  LBM_EINVAL for a
 * number below -1. */
int lbm_batch_set_variant(lbm_batch* batch, int variant);

/* Tile rows per work item of the persistent kernel (default 8): its items are strips, one tile
 * column of a band of this many tile rows; the strips of a band are taken one after another, so
 * they walk down their columns side by side and horizontally neighbouring tiles share their halo
 * reads in L2.  Longer strips spread the per-item cost (a queue atomic, the dependency check) over
 * more tiles; shorter ones give more items to balance.  Fixed once the batch has run in the
 * persistent mode (the band counters count strips).  LBM_EINVAL outside 1..1024 or after that. */
int lbm_batch_set_segment(lbm_batch* batch, int tiles);

/* Clock cycles a block of the persistent kernel waits for another tile's progress before giving
 * up (test hook: 0 gives up at once). */
int lbm_batch_set_barrier_limit(lbm_batch* batch, long long cycles);

int lbm_batch_info(lbm_batch* batch, lbm_batch_info_t* out);

/* Batch autotuning: the kernel a batch runs is chosen by timing the candidates on the instances
 * themselves, under batch conditions (concurrent streams or the persistent kernel over all of them),
 * since a kernel's speed alone and in a batch differ.  Each candidate runs a temporary batch of
 * clones of `descs` (as many as the batch's budget holds) in this batch's mode for 2 + steps batch
 * steps, the last `steps` timed.  Candidates: in the streams mode the step-kernel variants built for
 * the class (variant; segment 0); in the persistent mode the tile codes it runs for the class
 * (variants 27, 28, 2, 0) times strip lengths 4, 8, 12.  Needs device memory for the clones. */
typedef struct {
    int variant;               /* lbm_batch_set_variant number                                   */
    int segment;               /* persistent mode: tile rows per strip (lbm_batch_set_segment)   */
    double us_per_step;        /* time of one batch step of the clones                           */
} lbm_batch_tune_entry;

/* Time the candidates; fills up to cap entries of out, *n receives the number timed. */
int lbm_batch_tune(lbm_batch* batch, const lbm_instance_desc* descs, int n, int steps, lbm_batch_tune_entry* out,
                   int cap, int* n_out);

/* lbm_batch_tune, then set the fastest candidate on the batch (which must hold no instance yet);
 * *best receives it if not NULL. */
int lbm_batch_autotune(lbm_batch* batch, const lbm_instance_desc* descs, int n, int steps,
                       lbm_batch_tune_entry* best);

/* Run the batch on `stream` (caller-owned cudaStream_t; 0 is the default stream). */
int lbm_batch_set_stream(lbm_batch* batch, void* stream);

/* Free the batch and all its instances (waits for its work).  NULL is allowed. */
void lbm_batch_destroy(lbm_batch* batch);

/* ----------------------------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  Clients submit solves (an instance, its
 * length and how to fit it) from any thread; a worker thread admits them in arrival order as soon
 * as their device footprint fits the budget, runs all admitted instances of a lattice/storage/
 * collision class together in the batch kernel (K steps per round; requests that arrive during a
 * round join the next one), and retires each instance when it has run all its steps: FP64 fit of
 * its force history (lbm_fit), normalized damping (lbm_gamma_bar), device memory freed.  An
 * instance's result is the same whether it ran alone or among others (the batch kernel computes
 * each instance exactly as lbm_step does).  Times are seconds on the host's steady clock since
 * lbm_server_create.
 * ---------------------------------------------------------------------------------------------- */
typedef struct lbm_server lbm_server; /* opaque; owned by the library */

typedef struct {
    lbm_instance_desc desc;   /* the solve; plate, beam or open geometries (not masks)              */
    double skip_periods;      /* fit window: the steps after this many periods (lbm_fit)           */
    double perimeter;         /* wetted perimeter for gamma_bar (0: not computed)                  */
} lbm_request;

typedef struct {
    long long id;
    int status;               /* 0 waiting, 1 running, 2 done, negative: LBM_E* failure            */
    double submit_s, admit_s, done_s;
    double f_in, f_q, f_0;    /* lbm_fit of the force history                                      */
    double gamma_bar;
    long steps;
    size_t fluid_nodes;
} lbm_result;

typedef struct {
    long long submitted, completed, rounds;
    double lattice_updates;   /* fluid-node updates of the completed requests                      */
    double busy_s;            /* time with batch work in flight                                    */
    double elapsed_s;
    size_t budget_bytes, used_bytes, peak_used_bytes;
    int peak_running;         /* most instances resident at once                                   */
    int worker_error;         /* last error of the worker (0 if none)                              */
} lbm_server_stats_t;

/* Start a server on the current device.  device_budget_bytes caps the memory its instances hold
 * (0: free memory minus 2 GiB); steps_per_round is K. */
int lbm_server_create(size_t device_budget_bytes, int steps_per_round, lbm_server** out);

/* Queue a request (returns at once).  LBM_ENOMEM if it could never fit the budget. */
int lbm_server_submit(lbm_server* server, const lbm_request* req, long long* id);

/* Mode of the class batches the server creates from now on (lbm_batch_set_mode; default
 * LBM_BATCH_STREAMS).  Call it before the first lbm_server_submit so that every class uses it. */
int lbm_server_set_batch_mode(lbm_server* server, int mode);

/* Kernel of one (lattice, storage, collision) class of requests: the class batch the server creates
 * from now on gets lbm_batch_set_variant(variant) and, in the persistent mode,
 * lbm_batch_set_segment(segment) (0: the default) -- e.g. the choice lbm_batch_tune made on a sample
 * of the class's requests.  LBM_EINVAL for a variant below -1 or a negative segment. */
int lbm_server_set_class_kernel(lbm_server* server, int lattice, int storage, int collision, int variant, int segment);

/* Copy a request's result; returns 1 when it has finished (done or failed), 0 otherwise. */
int lbm_server_poll(lbm_server* server, long long id, lbm_result* out);

/* Wait up to timeout_s seconds for a request to finish; returns as lbm_server_poll. */
int lbm_server_wait(lbm_server* server, long long id, double timeout_s, lbm_result* out);

/* Force history of a completed request (as lbm_force_history); kept until released. */
int lbm_server_force_history(lbm_server* server, long long id, double* out_xy, size_t cap_steps, size_t* n_steps);

/* Forget a finished request. */
int lbm_server_release(lbm_server* server, long long id);

int lbm_server_stats(lbm_server* server, lbm_server_stats_t* out);

/* Stop the worker (running requests finish their current round and are marked failed), free
 * everything.  NULL is allowed. */
void lbm_server_destroy(lbm_server* server);

/*
 * One time step that allocates no device memory.  (The paper has no counterpart: this is a
 * service of the library.)
 *
 * For callers that cannot call cudaMalloc when they step the solver: code recording its work
 * into a CUDA graph (no allocation is allowed during stream capture), applications whose device
 * memory belongs to another allocator that has already reserved it, and loops with a fixed memory
 * budget where an allocation that may fail or stall is not acceptable.  lbm_step may allocate (it
 * grows the force history); this call never does, and makes no cudaMalloc, cudaFree or other
 * allocating call.
 *
 * It advances the populations in g_in by one step into g_out and writes the force on the body
 * during the step, (Fx, Fy) in FP64, to force_out[0..1].  All three are device buffers owned by
 * the caller: g_in and g_out hold Q * ny * pitch values of the simulation's storage type in the
 * simulation's layout (h_i = (f_i - w_i rho0) / (w_i s), [Q][ny][pitch], pitch and storage from
 * lbm_info; s = u0 for 16-bit storage, else 1) and must not overlap.  `sim` supplies the geometry,
 * parameters and tile shape only; its own state and force history are neither read nor changed.
 * n is the step index: the wall velocity or body force is taken at t = n + 1/2, as in lbm_step.
 * The work is enqueued on `stream` (a cudaStream_t; 0 is the default stream) and the call returns
 * before it runs.
 *
 * Scratch: the kernel's per-tile force partials and its reduction counter live in one static
 * device array of the library (LBM_NOALLOC_MAX_SLOTS * 16 + 256 bytes), held by every GPU that
 * loads the library until the process exits.  A geometry with more than LBM_NOALLOC_MAX_SLOTS
 * tiles holding body links is rejected with LBM_ERANGE (a larger tile, lbm_set_tile, needs fewer).
 * All calls in the process share that array: calls whose work overlaps on the GPU (two streams,
 * or two host threads) race and give wrong forces; serialize them.  The counter is cleared at
 * the start of every call, so a call that never completed does not affect the next one.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture (a lookup that fails is
 * not remembered: the next call tries again).
 * A diverged run is not reported by this call's return code (lbm_step's LBM_ENONFINITE comes from
 * a flag that lbm_synchronize reads; this call keeps no such state between calls): the force it
 * writes is then non-finite, so callers check force_out for NaN or Inf.
 * Errors: LBM_EINVAL (null or aliased buffers, n < 0), LBM_ERANGE, LBM_ECUDA.
 */
#define LBM_NOALLOC_MAX_SLOTS 8192
int lbm_step_noalloc(const lbm_sim* sim, long n, const void* g_in, void* g_out, double* force_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */

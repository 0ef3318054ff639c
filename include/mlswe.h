/*
 * mlswe.h -- C ABI of the GB300 multilayer shallow-water AMR library.
 *
 * Paper: A. Schwarzschild and K. Mandli, "An Implementation of Adaptive Mesh
 * Refinement for Shallow Water Equations", arXiv:1803.01450.
 *
 * The library advances an M-layer (M = 1 to 4) shallow-water model on a
 * hierarchy of refinement levels (Sec. 2, Eqs. (1)-(2): dx^{l+1} = dx^l / r^l)
 * for one or more independent ensemble members, in FP64 on one GPU (several
 * processes, one per GPU, can split a hierarchy's refined patches: see the patch
 * partition entry points near the end). Layer 1 is
 * the top layer (Sec. 2.1). The conserved fields of a cell are, per layer m,
 * (h_m, h_m u_m, h_m v_m); arrays of a level are stored field-major
 * [3M][ny][nx] (row-major, x fastest) in the order
 * (h_1, hu_1, hv_1, h_2, hu_2, hv_2).
 *
 * Storage: every level of every member is a dense array over the whole
 * domain at that level's resolution; patches are index boxes into it. Cells
 * outside all patches of a level hold ghost values only.
 *
 * Conventions (all entry points):
 *  - Every call returns an mlswe_status; nothing throws across the ABI. The
 *    text of the last error of a hierarchy is returned by mlswe_last_error.
 *  - Host arrays passed in are copied before the call returns; output
 *    pointers are owned by the caller. Device memory is owned by the library
 *    (obtained through the caller's allocator, or cudaMalloc when none is
 *    given) and released by mlswe_destroy.
 *  - All GPU work is issued on the stream given at creation. Calls with host
 *    outputs synchronise that stream before returning.
 *  - A hierarchy is used by one host thread at a time.
 *  - Box convention: int32 [i0, j0, i1, j1), half-open, in the cell indices
 *    of the level the box belongs to.
 */
#ifndef MLSWE_H
#define MLSWE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlswe_hier* mlswe_h;

typedef enum {
  MLSWE_OK = 0,
  MLSWE_EINVAL = 1,     /* bad argument (sizes, indices, null pointers, unsupported option) */
  MLSWE_ENOMEM = 2,     /* device or host allocation failed */
  MLSWE_ECUDA = 3,      /* a CUDA call failed; text in mlswe_last_error */
  MLSWE_ECFL = 4,       /* Courant number above cfl_max: mlswe_step_level undid the level step;
                           mlswe_advance spent its retake budget (see there) */
  MLSWE_ENEGDEPTH = 5,  /* a non-finite value was met in the wave-speed reduction */
  MLSWE_ENESTING = 6,   /* a patch layout violates nesting or overlaps */
  MLSWE_ETIMEOUT = 7,   /* reserved: a bounded device wait gave up */
  MLSWE_EHYPERB = 8,    /* reserved: edges that lost hyperbolicity are counted, not failed
                           (mlswe_hyperbolicity_losses) */
  MLSWE_EMISSING = 9    /* the CUDA library or device is not available */
} mlswe_status;

/* Device allocator callback. alloc returns a device pointer (NULL on failure)
 * for `bytes` bytes usable on `stream`; free releases it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} mlswe_allocator;

/* Model and AMR configuration.
 *  M            layers (1 to 4); rho[0..M-1] densities, increasing downwards
 *               (rho[0] < rho[1] < ...). M = 3 and 4 couple the layers through the
 *               general M-layer eigenproblem (the paper's Eqs. (4)-(5) hold for any
 *               M) and run one CTA per SM; the adjoint takes M <= 2, the
 *               unsplit step M <= 3.
 *  g            gravity; dry_tol: layer m is wet where h_m > dry_tol and every
 *               layer above is wet (top-down rule, Sec. 2.1).
 *  cfl_desired  target Courant number for the automatic time step;
 *  cfl_max      a coarse step of mlswe_advance above it is rejected and retaken; a level
 *               step of mlswe_step_level above it (with a Courant report) is undone.
 *  order        1 or 2 (second-order wave correction); limiter 0 none,
 *               1 minmod, 2 MC; eigen 0: eigenvalue guesses + 2 Newton steps,
 *               1: guesses only.
 *  max_levels   1..4; ratio[l] refinement ratio from level l to l+1 (2 or 4),
 *               used in x, y and time (Sec. 2: r_t = max(r_x, r_y)).
 *  flag_tol     refine where |grad eta_1| > flag_tol.
 *  regrid_interval  coarse steps between regrids inside mlswe_advance (0: never).
 *  n_buf        flag dilation in cells; cluster_eff: minimum box efficiency;
 *  min_side, max_side  patch side bounds in fine cells.
 *  dynamic_rt   0: time ratio r_t = ratio[l] on every level (the CFL-safe choice,
 *               Sec. 2); 1: each coarse step chooses r_t of every level as the fewest
 *               steps per parent step that keep the level's Courant number at
 *               cfl_desired, ceil(dt_parent * rate / cfl_desired) within [1, ratio],
 *               from the wave speeds of the previous step (Sec. 2: a smaller r_t
 *               where the refined region is shallow, as GeoClaw does).
 *  unsplit      0: dimensional splitting (x sweep, then y sweep on its result);
 *               1: the unsplit wave-propagation step of GeoClaw's solver
 *               family (Sec. 1) in corner-transport form: every edge solved on Q^n, the
 *               fluctuation each cell receives (correction flux included) split by a
 *               transverse Riemann solve at the edge state, its parts correcting the
 *               fluxes of the edges above and below (left and right) the receiving cell
 *               with weight dt/(2 dx); one update of every cell. It keeps x and y
 *               symmetric. It allocates 12 * 3M doubles per cell of every level for the
 *               per-edge arrays. The adjoint and mlswe_step_fixed_noalloc take unsplit = 0.
 */
typedef struct {
  int M;
  double rho[4];
  double g;
  double dry_tol;
  double cfl_desired;
  double cfl_max;
  int order;
  int limiter;
  int eigen;
  int max_levels;
  int ratio[4];
  double flag_tol;
  int regrid_interval;
  int n_buf;
  double cluster_eff;
  int min_side;
  int max_side;
  int dynamic_rt;
  int unsplit;
} mlswe_config;

/* Physical extent [x0,x1] x [y0,y1] and coarse (level 0) cell counts of a member. */
typedef struct {
  double x0, y0, x1, y1;
  int nx0, ny0;
} mlswe_domain;

/* Creates a hierarchy of n_members independent members. Level 0 of each
 * member is one patch covering its domain, with walls on all four sides.
 * alloc may be NULL (cudaMalloc is used). stream is a cudaStream_t; NULL makes
 * the library create (and destroy with the hierarchy) a non-blocking stream of
 * its own, since the legacy default stream cannot be captured into a CUDA graph.
 * Errors: EINVAL (config or domain), ENOMEM, ECUDA. */
mlswe_status mlswe_create_hierarchy(const mlswe_config* cfg, int n_members, const mlswe_domain* doms,
                                    const mlswe_allocator* alloc, void* cuda_stream, mlswe_h* out);

/* Releases all device and host memory of the hierarchy. */
mlswe_status mlswe_destroy(mlswe_h h);

/* Text of the last error (never NULL; "" when none). Valid until the next call on h. */
const char* mlswe_last_error(mlswe_h h);

/* Level-0 cell counts of level `level` of `member`: nx, ny (host outputs). */
mlswe_status mlswe_level_shape(mlswe_h h, int member, int level, int* nx, int* ny);

/* Bathymetry. B_finest: host [ny_f][nx_f] samples at the cell centres of the
 * finest level (nx_f = nx0 * prod(ratio[0..max_levels-2])). Every level's B is
 * the recursive r x r mean of the next finer one (the operator of Eq. (11)),
 * computed on the device. */
mlswe_status mlswe_set_bathymetry(mlswe_h h, int member, const double* B_finest);

/* Bathymetry of one level (host [ny][nx] output). */
mlswe_status mlswe_get_bathymetry(mlswe_h h, int member, int level, double* B_out);

/* State of one level: host [3M][ny][nx] on the level's full index space. */
mlswe_status mlswe_set_state(mlswe_h h, int member, int level, const double* q);
mlswe_status mlswe_get_state(mlswe_h h, int member, int level, double* q_out);

/* Rows [j0, j0 + n) of every field of the current state of one level, device to device:
 * get copies them into dst, set copies src into them; the buffer is device [3M][n][nx]
 * (caller-owned). Ordered on the hierarchy's stream, no synchronisation (the copy is done
 * when later work on that stream runs). For the halo rows of a grid split into slabs of
 * rows across GPUs (not in the paper; the paper's runs share memory, Sec. 3). EINVAL for
 * rows outside the level or a buffer that is not device memory. */
mlswe_status mlswe_get_rows_device(mlswe_h h, int member, int level, int j0, int n, double* dst);
mlswe_status mlswe_set_rows_device(mlswe_h h, int member, int level, int j0, int n, const double* src);

/* Asynchronous input for pipelined runs: q (host [3M][ny][nx], page-locked for the copy to
 * overlap) is copied to a device staging buffer on the library's own copy stream, and
 * from there into the level's state, in order with the work already enqueued on the
 * hierarchy's stream (so a step enqueued before reads the old state, one enqueued after
 * the new one). Returns before the copy ends: q must stay unchanged until the next
 * mlswe_synchronize or synchronising call. Two staging buffers alternate, so the copy of
 * the next input overlaps the step in flight. Errors: EINVAL (bad member, level or null
 * q), ENOMEM (staging allocation), ECUDA. */
mlswe_status mlswe_set_state_async(mlswe_h h, int member, int level, const double* q);

/* Patch layout of level >= 1: n boxes (host int32 [n][4], level-l indices).
 * Boxes must be disjoint, lie inside the domain, have sides that are
 * multiples of nothing in particular, and nest inside level l-1 patches with
 * a margin of two level-(l-1) cells (ENESTING otherwise). Setting the layout
 * does not touch the data of the level. */
mlswe_status mlswe_set_patches(mlswe_h h, int member, int level, int n, const int32_t* boxes);

/* Patch layout of a level: *n receives the count; boxes (may be NULL) must
 * hold 4 * (*n on entry, as capacity) int32. Level 0 returns its single box. */
mlswe_status mlswe_get_patches(mlswe_h h, int member, int level, int* n, int32_t* boxes);

/* Fixed time step of every member for the next mlswe_step_level of `level`:
 * dt host [n_members]. */
mlswe_status mlswe_set_dt(mlswe_h h, int level, const double* dt);

/* One dimensionally split finite-volume step of every patch of `level` of
 * every member with the time step set by mlswe_set_dt (or, if dt is not
 * NULL, with dt host [n_members]). Ghost cells of patches on level >= 1 must
 * have been filled (mlswe_fill_ghosts). cfl_out (host [n_members], may be
 * NULL) receives the Courant number of the step: dt * max(sx/dx, sy/dy); when
 * some member's exceeds cfl_max the step is undone for every member (the level's
 * state is the one before the call) and MLSWE_ECFL is returned, so the caller can
 * retry with a smaller dt. Without cfl_out nothing is checked. */
mlswe_status mlswe_step_level(mlswe_h h, int level, const double* dt, double* cfl_out);

/* Fills the ghost ring (2 cells) of every patch of `level` >= 1 that is not
 * covered by a sibling patch, by the refinement of Sec. 2.1 applied to the
 * level-(l-1) state interpolated linearly in time, at fraction alpha in
 * [0,1] between the last two level-(l-1) states. */
mlswe_status mlswe_fill_ghosts(mlswe_h h, int level, double alpha);

/* Refinement (Sec. 2.1, Eqs. (4), (5), (10), bottom-up over layers): fills
 * every cell of the level-(coarse_level+1) patches of `member` from the
 * current level-coarse_level state and the fine bathymetry. */
mlswe_status mlswe_interp_fine(mlswe_h h, int coarse_level, int member);

/* Coarsening (Sec. 2.2, Eq. (11)): every component of each level-(fine_level-1)
 * cell covered by a level-fine_level patch becomes the mean of its r x r fine cells. */
mlswe_status mlswe_average_coarse(mlswe_h h, int fine_level, int member);

/* Refinement flags of `level` from the current state (host uint8 [ny][nx]):
 * 1 where |grad eta_1|^2 > flag_tol^2 in a wet cell of the level. */
mlswe_status mlswe_get_flags(mlswe_h h, int member, int level, uint8_t* flags);

/* Rebuilds the patch layouts of levels base_level+1 .. max_levels-1 from flags
 * (dilated by n_buf, clustered into boxes), top down, and fills newly covered
 * fine cells by mlswe_interp_fine. */
mlswe_status mlswe_regrid(mlswe_h h, int base_level);

/* Advances every member by n_coarse_steps level-0 steps of the subcycled
 * Berger-Oliger scheme (r_t = ratio), with automatic time steps (cfl_desired),
 * averaging and mass reflux at coarse/fine interfaces, and a regrid every
 * regrid_interval coarse steps.
 * Courant control (Sec. 2 keeps every level's Courant number below one through
 * r_t): the Courant number of a coarse-step attempt is the largest over the levels
 * of dt_l * max(sx/dx_l, sy/dy_l). An attempt above cfl_max is rejected: every level
 * of that member returns to its state before the attempt (the refined levels' patch
 * cells are copied aside before each attempt, in one buffer per refined level and
 * member allocated at the first call) and its time does not advance; the next round
 * retakes the step with the time step the usual rule gives from the wave speeds the
 * rejected attempt measured (dt * cfl_desired / Courant number for the bounding
 * level). The call runs n_coarse_steps rounds (regrids at the rounds the interval
 * selects), then retake rounds without regrids, in which only members short of
 * n_coarse_steps kept steps take a step, until every member has them; after
 * n_coarse_steps + 8 retake rounds it returns MLSWE_ECFL (the members keep their
 * last kept state). Rejections are counted in mlswe_stats.cfl_exceeded. */
mlswe_status mlswe_advance(mlswe_h h, int n_coarse_steps);

/* Simulated time of every member (t_out, host [n_members]) and the level-0 time
 * step of its next coarse step (dt_out, host [n_members]); either may be NULL. */
mlswe_status mlswe_get_time(mlswe_h h, double* t_out, double* dt_out);

/* Execution form of mlswe_advance (not in the paper). use_graphs: capture one
 * coarse step per level-0 parity as a CUDA graph and replay it (kernels read
 * their work lists and time steps from device memory, so a regrid needs no
 * recapture). per_patch_launches: launch the sweeps once per patch instead of
 * once per level for all patches of all members (the unbatched form, kept for
 * comparison; disables graphs). */
mlswe_status mlswe_set_execution(mlswe_h h, int use_graphs, int per_patch_launches);

/* Tile autotuner (not in the paper): times the candidate sweep tiles on the
 * current patches of `level` (iters launches each, CUDA events, the state is not
 * advanced) and keeps the fastest per sweep direction, over 5 tile shapes and
 * 1 or 2 resident CTAs per SM. chosen (host int[6], may be NULL): x len, x lines,
 * x CTAs per SM, y len, y lines, y CTAs per SM. */
mlswe_status mlswe_autotune(mlswe_h h, int level, int iters, int* chosen);

/* Surface elevations eta_m (Eq. (4)) at n points (host [n][2], physical x, y)
 * from the finest level whose patch contains each point; eta_out host [n][M]. */
mlswe_status mlswe_read_gauges(mlswe_h h, int member, int n, const double* xy, double* eta_out);

/* mlswe_read_gauges without waiting: the gauge kernel and the copy into eta_out (host
 * [n][M], page-locked for an asynchronous copy) are enqueued on the hierarchy's stream;
 * the values are there after mlswe_synchronize. xy is read before the call returns. */
mlswe_status mlswe_read_gauges_async(mlswe_h h, int member, int n, const double* xy, double* eta_out);

/* Waits for all work of the hierarchy (its stream and the input copy stream). */
mlswe_status mlswe_synchronize(mlswe_h h);

/* Run counters (not in the paper; its own report counts cell updates and time,
 * Sec. 3). level_steps[l]: steps taken on level l (subcycles of mlswe_advance
 * and mlswe_step_level calls); cell_updates[l]: cells inside the patches of
 * level l times those steps, summed over members (multiply by M for
 * layer-cell updates); patches[l]: current patch count of level l over
 * members; regrids: regrids run; coarse_steps: coarse steps of mlswe_advance;
 * cfl_exceeded: member coarse-step attempts rejected because their Courant number
 * exceeded cfl_max (each was retaken); last_cfl: largest Courant number of the last
 * coarse-step attempt over the members. level_steps and cell_updates include the
 * steps of rejected attempts (work the GPU did); coarse_steps counts the rounds of
 * mlswe_advance that can regrid (not the retake rounds).
 * Levels beyond max_levels read 0. Synchronises the stream. */
typedef struct {
  long long coarse_steps;
  long long regrids;
  long long level_steps[4];
  long long cell_updates[4];
  int patches[4];
  long long cfl_exceeded;
  double last_cfl;
} mlswe_stats;

mlswe_status mlswe_get_stats(mlswe_h h, mlswe_stats* out);

/* Time-stepping state of the hierarchy, for checkpoint and resume (not in the
 * paper): member times, the wave speeds from which the next coarse step takes
 * its time step (or the pending speeds of a new state), whether that time step
 * is ready, and the coarse-step counter that schedules regrids, as
 * n_doubles = n_members * (1 + 3 * max_levels) + 3 doubles (host; speeds are
 * stored as their bit patterns). EINVAL for another n_doubles. A hierarchy
 * created with the same configuration and domains, given the same bathymetry,
 * then the patch layouts and states of every level (mlswe_set_patches,
 * mlswe_set_state) and last this clock, continues a run bit for bit. */
mlswe_status mlswe_get_clock(mlswe_h h, double* buf, int n_doubles);
mlswe_status mlswe_set_clock(mlswe_h h, const double* buf, int n_doubles);

/* Number of edges (counted once each, over the interior lines of every sweep
 * of every level step since the last reset) whose two-layer Roe state had
 * (u1 - u2)^2 >= (1 - r) g (hbar_1 + hbar_2), where the eigenvalue guesses
 * were used without the Newton steps (GeoClaw's treatment of a loss of
 * hyperbolicity, read for the solver the paper cites in Sec. 1). *count
 * (host) receives the count modulo 2^32; reset = 1 sets it back to zero.
 * Synchronises the stream. */
mlswe_status mlswe_hyperbolicity_losses(mlswe_h h, long long* count, int reset);

/* Launch configuration of the sweep kernels (not in the paper): tiles of at
 * most `len` cells along the sweep direction (each patch's extent is split into
 * equal parts) times at least `lines` lines (x sweep dir = 0: rows; y sweep
 * dir = 1: columns; a tile takes as many lines, up to 32, as fill 256 edges,
 * lines * (len + 3) <= 256), with len >= 4, and CTAs per SM of the persistent
 * grid (1 or 2). EINVAL for shapes out of range. Results do not depend on the
 * tiles. Default: 125 x 2 with 2 CTAs per SM in both directions. */
mlswe_status mlswe_set_tiles(mlswe_h h, int dir, int len, int lines, int ctas_per_sm);

/* Discrete adjoint of the fixed-grid step (not written out in the paper; the
 * forward step is the per-patch solver the paper's AMR drives, Sec. 1-2).
 * Gauge misfit J = sum_{n=1..n_steps} sum_g (eta_1(cell_g, Q^n) - obs[n-1][g])^2
 * with eta_1 = B + h_M + ... + h_1 (Eq. (4)). Requires a hierarchy with one
 * member, one level and order 1, a fixed time step (mlswe_set_dt) and a wet
 * state (every layer wet on both sides of every edge; EINVAL otherwise).
 * gauge_ij: host int32 [n_gauges][2] cell indices (i, j); obs: host
 * [n_steps][n_gauges]. The forward pass keeps a state every ckpt_every steps;
 * the backward pass recomputes each segment from it. Setup also times three
 * tile shapes of the transposed sweeps on the current state (CUDA events) and
 * keeps the fastest per direction (the timings are representative when it
 * follows mlswe_set_dt and mlswe_set_state; results never depend on the shape). */
mlswe_status mlswe_adjoint_setup(mlswe_h h, int n_steps, int ckpt_every, int n_gauges, const int32_t* gauge_ij,
                                 const double* obs);

/* Whether the adjoint keeps, for every step of the segment being recomputed, the
 * forward record of each coupled two-layer edge (eigenvalue guesses and Newton
 * iterates, the reciprocals of the Newton steps, of the Roe weights and of the
 * Vandermonde denominators, the wave strengths: 36 doubles per edge and sweep,
 * ckpt_every steps of them, about 2 * 36 * 8 * (nx + 1) * (ny + 1) * ckpt_every
 * bytes) so the transposed sweeps read it instead of rebuilding it. enable = 1
 * (the default) or 0; takes effect at the next mlswe_adjoint_setup, which keeps
 * the rebuilding path when the memory cannot be allocated. Results agree to
 * rounding either way. Not in the paper (a memory-for-arithmetic trade on a
 * device whose FP64 rate bounds the adjoint). */
mlswe_status mlswe_adjoint_keep_edge_data(mlswe_h h, int enable);

/* The controls of the gauge-misfit problem (Sec. 2.1, Eqs. (4)-(5) with the fluid at
 * rest): eta1_0, the initial top surface eta_1, and B, the bathymetry, both device
 * [ny][nx] (caller-owned, read before the call returns). The library writes B into the
 * level and builds the initial state on the device: for two layers with the interface
 * at rest at eta2, h_2 = eta2 - B and h_1 = eta1_0 - eta2; for one layer h_1 = eta1_0 - B
 * (eta2 unused); momenta 0. Needs one member and one level (EINVAL otherwise, and for
 * pointers that are not device memory). Synchronises the stream. */
mlswe_status mlswe_fixed_set_controls(mlswe_h h, const double* eta1_0, const double* B, double eta2);

/* mlswe_fixed_set_controls, then n_steps first-order steps from that state (advancing
 * it); returns J in *loss (host). Call mlswe_adjoint_setup once before (after a first
 * mlswe_fixed_set_controls, so that its tile timing sees a representative state). */
mlswe_status mlswe_fixed_forward(mlswe_h h, const double* eta1_0, const double* B, double eta2, double* loss);

/* Runs n_steps first-order steps from the current level-0 state, however it was set
 * (advancing it), and returns J in *loss (host). */
mlswe_status mlswe_fixed_forward_state(mlswe_h h, double* loss);

/* Gradient of J of the last forward pass with respect to the controls of
 * mlswe_fixed_forward: dL_deta1_0 and dL_dB, device [ny][nx] (caller-owned). B enters
 * the initial depth of the bottom layer, every step's flux jumps (Eq. (4) surfaces)
 * and every gauge's eta_1, so dL_dB = (dJ/dB at fixed Q^0) - dJ/dh_M(0); dL_deta1_0 =
 * dJ/dh_1(0). Computed on the device. EINVAL for pointers that are not device memory,
 * a missing forward pass, or an edge whose layers were not wet on both sides. */
mlswe_status mlswe_fixed_backward(mlswe_h h, double* dL_deta1_0, double* dL_dB);

/* Gradient of J of the last forward pass with respect to the initial state and, at fixed
 * initial state, the bathymetry: dL_dq0 device dense [3M][ny][nx], dL_dB device [ny][nx]
 * (caller-owned). The state-level form of mlswe_fixed_backward, for callers that set the
 * initial state themselves (mlswe_set_state + mlswe_fixed_forward_state). */
mlswe_status mlswe_fixed_backward_state(mlswe_h h, double* dL_dq0, double* dL_dB);

/* One dimensionally split step of a single grid with walls on all sides that
 * allocates no memory. The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory while they step the model
 * (for example a solver run inside a callback of a framework that owns the
 * device memory pool, or a service under a no-allocation-after-start-up rule).
 * The caller passes its own device buffers: q_in and q_out [3M][ny][nx], B
 * [ny][nx]; q_out may share no byte with q_in or B, and all three must be device (or
 * managed) memory (MLSWE_EINVAL otherwise, checked before any GPU work). The solver's working memory (state after the x sweep,
 * tile lists, descriptor, time step, wave-speed slots) lives in one static
 * device array of about 16 MB that every GPU loading the library holds until
 * the process exits; grids of M * nx * ny <= 2 * 512 * 512 layer cells (nx, ny >= 4;
 * 512 x 512 cells for one or two layers) fit, larger ones return MLSWE_EINVAL. M is
 * 1 to 4, densities strictly increasing downwards. The first call on a device looks up that
 * array's device address (a runtime query, not stream work). All calls
 * share the array: calls that overlap on the GPU race and must be serialised
 * by the caller. Uses the model settings of cfg (M, rho, g, dry_tol, order,
 * limiter, eigen); work is issued on cuda_stream. cfl_out (host, may be NULL)
 * receives the Courant number and then synchronises the stream. */
mlswe_status mlswe_step_fixed_noalloc(const mlswe_config* cfg, int nx, int ny, double dx, double dy, double dt,
                                      const double* q_in, const double* B, double* q_out, void* cuda_stream,
                                      double* cfl_out);

/* Launch instrumentation (not in the paper). Returns, and resets, the time in
 * ms and the launch count of each kernel class since the previous call, as
 * measured by CUDA events recorded around every launch on the hierarchy's
 * stream while enabled, and the total number of kernels launched (timed or
 * not). Classes: 0 x sweep, 1 y sweep, 2 ghost fill, 3 refinement, 4 coarsening
 * (and bathymetry means), 5 flags, 6 reflux, 7 other, 8 adjoint (the transposed
 * sweeps and the recomputed x sweeps of the backward pass). n: capacity of ms_out and
 * launches_out (either may be NULL). enable: timing on (1) or off (0) from now
 * on. Synchronises the stream. */
mlswe_status mlswe_timing(mlswe_h h, int enable, int n, double* ms_out, long long* launches_out,
                          long long* total_launches);

/* ---- Patch partition across ranks (not in the paper; its conclusion names parallel and
 * GPU work as the next step). One process per GPU holds the whole hierarchy; the work of
 * the refined levels is split by patches:
 *  - the patches of every level >= 1 are ordered by member, then by the Morton
 *    (Z-order) key of their centre (bits of the integer cell indices (i0 + i1) / 2 and
 *    (j0 + j1) / 2 interleaved, x in the even bits), then by patch index; with T the
 *    level's patch cells over all members and c_p the cells before patch p in that order,
 *    patch p goes to rank min(n - 1, floor((2 c_p + cells_p) n / (2 T))) (the rank whose
 *    share of the cells holds the patch's middle cell), so each rank's cells differ from
 *    T / n by at most the largest patch;
 *  - a rank sweeps and ghost-fills only its own patches of levels >= 1 (a patch's ghost
 *    ring is read by its own sweeps only; cells outside every patch may therefore differ
 *    between ranks), and coarsens only its own patches of the finest level; level 0, the
 *    other coarsenings, the reflux, the time step and the regrids run on every rank;
 *  - inside mlswe_advance the library calls the exchange hook at fixed points with a
 *    kind, and the hook must give every rank the other ranks' packed values of that kind
 *    (mlswe_partition_pack / mlswe_partition_unpack, through an all-gather), and, for
 *    kinds 0 to 2, the maximum over the ranks of the wave-speed slots
 *    (mlswe_wave_speed_slots):
 *      MLSWE_XCHG_FULL (0): every patch of the level: after each step of a refined
 *        level other than the finest, before every regrid and at the end of
 *        mlswe_advance (for the finest level);
 *      MLSWE_XCHG_HALO (1): after the finest level's substeps other than the last of a
 *        parent step, only the cells of each patch within two cells (corners included)
 *        of another rank's patch of the same member: nothing but the next substep reads
 *        the level then, and a substep of a patch reads other patches only that close;
 *      MLSWE_XCHG_LAST (2): after the last substep, the halo cells and every patch's
 *        boundary mass-flux accumulators (which the parent's reflux reads);
 *      MLSWE_XCHG_AVERAGED (3): after the finest level is coarsened onto its parent
 *        (`level` is the parent), the parent cells under every patch of the finest level
 *        (the only parent cells that coarsening wrote);
 *    so between the exchanges of the finest level the other ranks' patches of that level
 *    are stale on a rank, and every reader of them (the regrid, the end of the call) is
 *    preceded by a full exchange. Then after mlswe_advance the ranks' hierarchies equal
 *    the undivided hierarchy's.
 * The orders and the split are the same on every rank (host integer arithmetic on the
 * same layouts), so no owner table is sent. */

enum { MLSWE_XCHG_FULL = 0, MLSWE_XCHG_HALO = 1, MLSWE_XCHG_LAST = 2, MLSWE_XCHG_AVERAGED = 3 };

/* Exchange hook: called by mlswe_advance (and mlswe_regrid) on the calling thread at the
 * points above, with the kernels before it enqueued on the hierarchy's stream; work it
 * enqueues on that stream runs before the rest of the call. kind: an MLSWE_XCHG_ value, to
 * pass on to the sizes, pack and unpack calls. Returns 0, or non-zero to stop the call
 * with MLSWE_EINVAL. */
typedef int (*mlswe_exchange_hook)(void* ctx, int level, int kind);

/* Partition the refined levels' patches over world_size ranks (rank: this process's).
 * world_size 1 undoes it. The split step only (unsplit: MLSWE_EINVAL) and the batched
 * launch form (mlswe_set_execution per_patch_launches = 1 is refused while partitioned);
 * mlswe_advance launches directly (no graph capture) while a hook is set. hook may be
 * NULL for callers that step levels themselves (mlswe_step_level steps only this rank's
 * patches of a level >= 1; the caller exchanges). */
mlswe_status mlswe_set_partition(mlswe_h h, int rank, int world_size, mlswe_exchange_hook hook, void* ctx);

/* Owner rank of every patch of (member, level): owner_out host [n patches]. */
mlswe_status mlswe_partition_owners(mlswe_h h, int member, int level, int* owner_out);

/* Doubles in each rank's packed buffer of `level` and `kind` (host [world_size]). Every
 * buffer is a list of boxes in a fixed order, each with some of: the 3M state fields of its
 * cells (current buffer; field, then row, then column), the boundary mass-flux accumulators
 * of its rows' left and right edges and of its columns' bottom and top edges ([M][rows][2],
 * [M][columns][2]), the interface mass fluxes of every x edge and y edge of the box
 * including its sides ([M][rows][columns + 1], [M][rows + 1][columns]). FULL: every patch
 * the rank owns (in the order of the split above) with its state, accumulators and, on
 * levels with a finer level, interface fluxes. HALO: for every pair of a patch P the rank
 * owns and a patch Q of another rank (same member), the state of the box where Q grown by
 * two cells meets P. LAST: the HALO boxes, then every owned patch's accumulators. AVERAGED
 * (level = the finest level's parent): for every finest-level patch the rank owns, the
 * state of the parent cells under it. */
mlswe_status mlswe_partition_sizes(mlswe_h h, int level, int kind, long long* doubles_per_rank);

/* This rank's packed buffer of `level` and `kind` into dst (device, mlswe_partition_sizes
 * doubles), enqueued on the hierarchy's stream. */
mlswe_status mlswe_partition_pack(mlswe_h h, int level, int kind, double* dst);

/* Writes the values rank `from` packed for `level` and `kind` from its packed buffer src
 * (device), enqueued on the hierarchy's stream. */
mlswe_status mlswe_partition_unpack(mlswe_h h, int level, int kind, int from, const double* src);

/* Device address and length of the wave-speed slots (n doubles: the largest wave speed of
 * every member, level and sweep direction in the current coarse step, non-negative). An
 * exchange hook replaces them by their maximum over the ranks. */
mlswe_status mlswe_wave_speed_slots(mlswe_h h, double** dev, int* n);

#ifdef __cplusplus
}
#endif

#endif /* MLSWE_H */

/*
 * ls.h -- C ABI of the B300 narrow-band level-set library (libls.so).
 *
 * The library advances a level-set function phi on a 3-D grid with the
 * explicit first-order upwind scheme of arXiv 1612.04040, section 1:
 *
 *   Eq. 3  phi^{n+1}_{ijk} = phi^n_{ijk} - dt [max(F,0) G+ + min(F,0) G-]
 *   Eq. 4  G+ = sqrt( sum over x,y,z of max(D-,0)^2 + min(D+,0)^2 )
 *   Eq. 5  G- = sqrt( sum over x,y,z of max(D+,0)^2 + min(D-,0)^2 )
 *
 * restricted to a narrow band (section 1.1): the tube T = {|phi| < gamma}
 * (Eq. 6), gamma = halfwidth * h, is tested per 8x8x8 tile, and the active
 * tiles are the tube tiles dilated by one tile (covering the region N of
 * Eq. 11).  Points of inactive tiles are frozen.  The band is rebuilt every
 * `rebuild_every` steps; in CFL mode dt = CFL * h / max|F| over the active
 * points (CFL * h if that max is 0).  D-x = (phi_i - phi_{i-1})/h and
 * D+x = (phi_{i+1} - phi_i)/h; at a domain face the missing one-sided
 * difference equals the existing one (LS_BC_EXTRAPOLATE, default) or is 0
 * (LS_BC_NEUMANN).
 *
 * Conventions for every call:
 *  - Return value: an ls_status code (0 = LS_OK, negative = error).  No call
 *    aborts, throws or exits.
 *  - Arrays crossing the ABI are dense row-major phi[z][y][x] (x fastest,
 *    index = (z*ny + y)*nx + x, the indexing of the paper's GPU listing in
 *    section 3), in the context's precision: float for LS_FP32, double for
 *    LS_FP64.  `*_on_device` = 1 means a CUDA device pointer of the current
 *    device, 0 a host pointer.  Inputs are copied; the caller keeps
 *    ownership of every buffer it passes.  The library owns all device state
 *    of a context and frees it in ls_destroy.
 *  - Work is queued on the context's stream (ls_set_stream; default: the
 *    legacy default stream).  Calls that return values to the host
 *    (ls_get_*, ls_band_rebuild with a non-NULL count, ls_step with a
 *    non-NULL last_dt, the non-finite checks of ls_set_phi / ls_set_speed)
 *    synchronise that stream.
 *  - Device-side failures are recorded in a sticky status word read by
 *    ls_get_status; device waits are bounded and end in LS_ETIMEOUT, never
 *    in a trap or a hang.
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef LS_H
#define LS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ls_ctx ls_ctx; /* opaque; created and freed by the library */

typedef enum {
    LS_OK = 0,
    LS_EINVAL = -1,     /* bad argument (size, pointer, enum, alignment)   */
    LS_ENOMEM = -2,     /* device or host allocation failed                */
    LS_ECUDA = -3,      /* a CUDA call failed (see ls_last_cuda_error)     */
    LS_ETIMEOUT = -4,   /* a bounded device wait ran out                   */
    LS_ENONFINITE = -5, /* NaN or Inf in phi or F                          */
    LS_ESTATE = -6,     /* call not valid in the context's current state   */
    LS_EIO = -7         /* an output file could not be written              */
} ls_status;

enum { LS_FP32 = 0, LS_FP64 = 1 };               /* storage + arithmetic precision */
enum { LS_DT_FIXED = 0, LS_DT_CFL = 1, LS_DT_KEEP = 2 };  /* meaning of dt_or_cfl  */
enum { LS_PLAIN = 0, LS_LEARNED = 1 };           /* step flavour                   */
enum { LS_SCHEME_PLAIN = 0, LS_SCHEME_LOCAL = 1 }; /* advance scheme (ls_set_scheme) */
enum { LS_BC_EXTRAPOLATE = 0, LS_BC_NEUMANN = 1 };

/* ---------------------------------------------------------------------
 * Single grid
 * ------------------------------------------------------------------- */

/* Create a context for an nx*ny*nz grid with spacing h (section 1, Eq. 3).
 * nx, ny, nz: multiples of 8, >= 8, nx*ny*nz <= 2^31; h > 0 and finite;
 * precision LS_FP32 or LS_FP64.  Allocates two phi buffers (ping-pong), the
 * speed field and the tile tables on the current CUDA device (FP32: also 512
 * bytes per tile for copies of the x-faces of frozen tiles next to the band,
 * one eighth of a phi buffer).
 * Errors: LS_EINVAL (sizes, h, precision, out == NULL), LS_ENOMEM, LS_ECUDA. */
int ls_create(int nx, int ny, int nz, double h, int precision, ls_ctx **out);

/* Free every device and host resource of ctx (NULL is accepted). */
int ls_destroy(ls_ctx *ctx);

/* Queue all later work of ctx on cuda_stream (a cudaStream_t, e.g. PyTorch's
 * current stream; NULL = legacy default stream). */
int ls_set_stream(ls_ctx *ctx, void *cuda_stream);

/* Initial level-set function phi^0 (Eq. 1; Step 0 of section 1.1).  Copies
 * nx*ny*nz values from src (row-major, context precision).  Marks the band
 * stale: the next ls_step rebuilds it from the whole grid.
 * Errors: LS_EINVAL (NULL src), LS_ENONFINITE (NaN/Inf; phi unchanged is not
 * guaranteed, the band stays stale), LS_ECUDA. */
int ls_set_phi(ls_ctx *ctx, const void *src, int src_on_device);

/* Step 0 on the device (section 1.1; Eq. 1: phi(x,0) = +-d, negative
 * inside), evaluated in FP64 at the cell centres ((i+1/2)h, (j+1/2)h,
 * (k+1/2)h) and stored in the context's precision.  params: host array of
 * nparams doubles, copied before the call returns.
 *   LS_SHAPE_SPHERES  [n, (cx, cy, cz, r) x n]: min_i |x - c_i| - r_i
 *   LS_SHAPE_TORUS    [cx, cy, cz, ax, ay, az, R, r], unit axis a:
 *                     sqrt((rho - R)^2 + s^2) - r, s = (x-c).a,
 *                     rho = distance from the axis line
 *   LS_SHAPE_SH       [cx, cy, cz, base, amp, lmax, a_lm...]
 *                     ((lmax+1)^2 - 1 coefficients, l = 1..lmax, m = -l..l,
 *                     1 <= lmax <= 16): |x - c| - (base + amp sum a_lm Y_lm)
 *                     with the real orthonormal spherical harmonics
 *                     Y_lm = N_lm P_l^|m|(cos theta) T_m(phi),
 *                     N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!),
 *                     T_m = sqrt2 cos(m phi) / 1 / sqrt2 sin(|m| phi) for
 *                     m > 0 / m = 0 / m < 0, P without the Condon-Shortley
 *                     phase (a radial level-set function)
 * Marks the band stale.  Errors: LS_EINVAL (kind or parameter count). */
enum { LS_SHAPE_SPHERES = 0, LS_SHAPE_TORUS = 1, LS_SHAPE_SH = 2 };
int ls_init_phi(ls_ctx *ctx, int shape, const double *params, int nparams);

/* Speed fields on the device (FP64 evaluation, stored in the context's
 * precision, per-tile max|F| computed as by ls_set_speed):
 *   LS_SPEED_SINUSOID  1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z)
 *   LS_SPEED_COSCOS    cos(4 pi x) cos(4 pi y)
 *   LS_SPEED_FOURIER   [n, (a, kx, ky, kz, theta) x n]:
 *                      sum a cos(2 pi k.x + theta) / sum |a|  (|F| <= 1)
 * params may be NULL for the first two. */
enum { LS_SPEED_SINUSOID = 0, LS_SPEED_COSCOS = 1, LS_SPEED_FOURIER = 2 };
int ls_init_speed(ls_ctx *ctx, int kind, const double *params, int nparams);

/* Speed field F (Eq. 2/3), same layout and precision as phi.  Also computes
 * the per-tile max|F| used by the CFL rule.  Errors as ls_set_phi. */
int ls_set_speed(ls_ctx *ctx, const void *src, int src_on_device);

/* Constant speed F everywhere (replaces a speed field).  LS_ENONFINITE if F
 * is not finite. */
int ls_set_speed_const(ls_ctx *ctx, double F);

/* Domain-face rule for the one-sided differences (LS_BC_*). */
int ls_set_bc(ls_ctx *ctx, int bc);

/* Build the band now (section 1.1, Step 1): gamma = halfwidth_in_h * h in
 * FP64; a tile is in the tube when min |phi| over its points < gamma (Eq. 6,
 * strict), the active set is the tube tiles plus their 26 neighbours, and the
 * active tile ids are compacted in ascending order.  Scans the whole grid.
 * Stores halfwidth for the rebuilds inside ls_step.  If n_active_tiles is not
 * NULL the stream is synchronised and the active-tile count written there.
 * Errors: LS_EINVAL (halfwidth <= 0 or not finite), LS_ESTATE (phi not set),
 * LS_ECUDA. */
int ls_band_rebuild(ls_ctx *ctx, double halfwidth_in_h, long long *n_active_tiles);

/* Advance nsteps steps of Eq. 3 (section 1.1, Step 2) on the active tiles.
 * dt_mode LS_DT_FIXED: dt = dt_or_cfl.  LS_DT_CFL: dt = dt_or_cfl * h / M,
 * M = max|F| over the points of the active tiles at the latest rebuild (over
 * the whole grid in full-domain mode), dt = dt_or_cfl * h when M = 0; dt is
 * computed in FP64 on the device.  rebuild_every > 0: the band is rebuilt
 * before a step whenever rebuild_every steps ran since the last rebuild
 * (counted across calls); 0: never inside this call.  A stale band (after
 * ls_set_phi / ls_set_speed*) is rebuilt from the whole grid before the first
 * step.  If last_dt is not NULL the stream is synchronised and the dt of the
 * last step written there.
 * LS_DT_KEEP (single grid, band, plain steps): the dt already on the
 * device (from the last rebuild, or from ls_set_dt_from_bound) is used and
 * dt_or_cfl is ignored; the caller makes every rebuild (ls_band_refresh),
 * so a call in which one would fall due returns LS_ESTATE; the tube test is
 * still fused into the step before it.  Calls in this mode do not
 * synchronise (unless last_dt is given), so a sequence of them can be
 * captured in a CUDA graph by the caller.
 * Errors: LS_EINVAL (nsteps < 0, rebuild_every < 0, dt_or_cfl <= 0 or not
 * finite, bad dt_mode), LS_ESTATE (phi or speed not set; no halfwidth given
 * yet and not in full-domain mode; LS_DT_KEEP outside its conditions),
 * LS_ECUDA. */
int ls_step(ls_ctx *ctx, int nsteps, double dt_or_cfl, int dt_mode,
            int rebuild_every, double *last_dt);

/* Advance scheme of ls_step.
 *
 * LS_SCHEME_PLAIN (default): Eq. 3 with speed F on the active tiles.
 *
 * LS_SCHEME_LOCAL: the paper's local level-set algorithm (section 1.1,
 * Steps 1-3), one ls_step step being
 *   1. N = the points whose point or one of its six face neighbours has
 *      |phi^n| < gamma (Eq. 11; T of Eq. 6 plus its one-cell ring);
 *   2. the cut-off advance phi-bar = Eq. 3 with the speed c(|phi^n|) F,
 *      c of Eq. 7 with beta = beta_in_h * h and gamma = halfwidth * h (so
 *      points with |phi| >= gamma keep their value: Eq. 8 on T);
 *   3. reinit_iters pseudo-time iterations of Eq. 12 on N from d = phi-bar:
 *      d <- d - dtau S (g - 1), g = the upwind |grad d| of Eq. 4 where d > 0
 *      and of Eq. 5 where d < 0, S = d / sqrt(d^2 + g^2 h^2) (Eq. 13),
 *      dtau = dtau_in_h * h; points outside N keep their value;
 *   4. the clamp of Eq. 10 on N: phi^{n+1} = min(max(d, -gamma), gamma).
 * The advance runs on the active tiles (band, rebuilds, CFL and frozen
 * tiles as in the plain scheme) and flags the tiles holding a point of N;
 * the reinitialisation passes visit only those (the other tiles cannot
 * change in the step).  The result equals the pointwise algorithm while the
 * active tiles contain N, which ls_band_breaches checks.
 * reinit_iters = -1 selects ceil(halfwidth / dtau_in_h) iterations (enough
 * for the pseudo-time front to cross the band once; "steady state").
 * Single FP32 / FP64 contexts; not with the learned step mode.  Takes effect
 * at the next ls_step; beta_in_h must be below the band's halfwidth then
 * (LS_ESTATE otherwise).
 * Errors: LS_EINVAL (unknown scheme, beta_in_h or dtau_in_h <= 0 or not
 * finite, reinit_iters < -1, batched context), LS_ESTATE (learned mode on),
 * LS_ENOMEM, LS_ECUDA. */
int ls_set_scheme(ls_ctx *ctx, int scheme, double beta_in_h, int reinit_iters, double dtau_in_h);

/* Number of (point of T, inactive face-neighbour tile) pairs met by the
 * local scheme's advance passes since ls_set_scheme: 0 means every point of
 * N lay inside the active tiles, so the tiled passes computed exactly the
 * pointwise algorithm.  Synchronises the stream. */
int ls_band_breaches(ls_ctx *ctx, unsigned long long *n);

/* Band dilation of the rebuild: the core tiles plus their 26 (default) or
 * only 6 face neighbours (a smaller band: fronts that move diagonally reach
 * its edge sooner).  Marks the band stale.  Errors: LS_EINVAL. */
int ls_set_dilation(ls_ctx *ctx, int neighbours);

/* How ls_step's periodic band rebuild (section 1.1: the tube T of Eq. 6
 * dilated by one tile, which covers N of Eq. 11) is computed when the step
 * before it ran the fused tube test on every active tile:
 *   LS_REBUILD_FULL         the dilation and the compaction each walk every
 *                           tile of the context (two launches);
 *   LS_REBUILD_INCREMENTAL  the dilation is marked from the core entries of
 *                           the previous active list (a core tile is always
 *                           active, so no other tile can be core), and only
 *                           the compaction reads every tile's flags, 16 per
 *                           thread (four launches);
 *   LS_REBUILD_AUTO         (default) incremental for contexts of at least
 *                           LS_REBUILD_AUTO_TILES tiles, else full (measured:
 *                           at 2^18 tiles the full walk is the faster, at
 *                           1.1 M and 2^21 tiles the incremental).
 * Both give the same list, flags, M, dt and values.  ls_band_rebuild, the
 * first rebuild after any change of state, full-domain mode and slab
 * contexts with ghost rows always walk every tile.  Clears the cached step
 * graphs.  Errors: LS_EINVAL (NULL context, unknown mode). */
enum { LS_REBUILD_AUTO = 0, LS_REBUILD_FULL = 1, LS_REBUILD_INCREMENTAL = 2 };
#define LS_REBUILD_AUTO_TILES (1 << 19)
int ls_set_rebuild_mode(ls_ctx *ctx, int mode);

/* ---------------------------------------------------------------------
 * Slab split along z (section 2: the grid is decomposed by one axis, each
 * part with a ghost layer from each neighbour; the tube's rows are shared
 * out by the greedy rule of Eq. 14).  A context then holds one slab of
 * whole tile rows plus, on each side that has a neighbour, one ghost tile
 * row holding that neighbour's copy.  The host moves the data between
 * slabs (its transport: a device copy, NCCL, ...); these calls only pack,
 * unpack, rebuild and report.
 * ------------------------------------------------------------------- */

/* Mark the bottom (lo = 1) and / or top (hi = 1) tile row of a single-grid
 * context as ghost rows: they are never active, their tube test is made on
 * the values last imported into them, and only they accept
 * ls_set_tile_rows.  Marks the band stale.  Errors: LS_EINVAL (batch
 * context, flags not 0 / 1, fewer than lo + hi + 1 tile rows). */
int ls_set_ghost_rows(ls_ctx *ctx, int lo, int hi);

/* The band rebuild that ls_step would make before its next step (Step 1 of
 * section 1.1): from the tube test fused into the last step when that step
 * made one, else by a scan of every tile; ghost rows are tested on their
 * current values.  Returns M = max |F| over the points of the new active
 * tiles (0 if none) and the active-tile count (both nullable).  Resets the
 * rebuild counter, so ls_step's own rebuild_every counts from here.
 * Synchronises the stream.  Errors: LS_EINVAL, LS_ESTATE (phi, speed or
 * halfwidth not set, full-domain mode). */
int ls_band_refresh(ls_ctx *ctx, double *M, long long *n_active);

/* With M and n_active both NULL, ls_band_refresh does not synchronise (it
 * can then be captured in a CUDA graph).  The bound M of the current band:
 * ls_band_speed_bound copies it to dst (device: asynchronous on the
 * context's stream; host: synchronises); ls_set_dt_from_bound sets, on the
 * device, M := *M_device and dt = cfl h / M (cfl h when M = 0) in FP64 with
 * the rebuild's expression, for the steps that follow in LS_DT_KEEP mode
 * (the slab split's common dt from an all-reduced M).  Errors: LS_EINVAL
 * (NULL, batch context, cfl not finite and positive), LS_ESTATE (no band). */
int ls_band_speed_bound(ls_ctx *ctx, double *dst, int dst_on_device);
int ls_set_dt_from_bound(ls_ctx *ctx, const double *M_device, double cfl);

/* Active tiles per tile row z (counts[tz], nrows = nz / 8) of the current
 * band: the row weights of Eq. 14.  Synchronises.  Errors: LS_EINVAL,
 * LS_ESTATE (no band). */
int ls_band_row_counts(ls_ctx *ctx, long long *counts, int nrows);

/* Copy tile rows [row0, row0 + nrows) of the current phi out to dst, or one
 * ghost row (nrows = 1) in from src.  plane = -1: whole rows, 512 values
 * per tile in the bricked order (tile by tile in row order, each x fastest,
 * then y, then z); plane = 0..7: only that z-plane of every tile, 64 values
 * per tile (x fastest, then y).  Values in the context precision.  Device
 * buffers (16-byte aligned) are asynchronous on the context's stream; host
 * buffers synchronise.  ls_set_tile_rows writes the buffer the next step
 * reads and leaves the band as it is.  Errors: LS_EINVAL (range, plane, not
 * a ghost row for ls_set_tile_rows), LS_ESTATE (phi not set). */
int ls_get_tile_rows(ls_ctx *ctx, int row0, int nrows, int plane, void *dst, int dst_on_device);
int ls_set_tile_rows(ls_ctx *ctx, int row0, int nrows, int plane, const void *src,
                     int src_on_device);

/* Copy tile row src_row of the context src (its current phi) straight into
 * ghost row `row` of ctx (plane as above): slabs of one grid held on the
 * same device in one process.  Asynchronous on ctx's stream; the caller
 * orders it after src's work (one stream for both, or an event).  Errors:
 * LS_EINVAL (batch context, precision or tile rows differ, range, not a
 * ghost row of ctx), LS_ESTATE (phi not set). */
int ls_copy_ghost_row(const ls_ctx *src, int src_row, ls_ctx *ctx, int row, int plane);

/* Full-domain mode, FP32 single grids, plain scheme: on, every step streams
 * tile columns along z (each tile's z halos are the neighbouring tiles of
 * its column, staged once); off (default): the active-list kernel over all
 * tiles, which measured faster.  The results are the same bits.  Errors:
 * LS_EINVAL. */
int ls_set_dense_kernel(ls_ctx *ctx, int on);

/* Full-domain mode on/off: every tile is active and no rebuild happens
 * (the O(n^3) variant the narrow band of section 1.1 replaces). */
int ls_set_full_domain(ls_ctx *ctx, int on);

/* Copy the current phi out (row-major, context precision) to dst.
 * Synchronises the stream.  Errors: LS_EINVAL, LS_ESTATE (phi not set). */
int ls_get_phi(ls_ctx *ctx, void *dst, int dst_on_device);

/* Copy the speed field F out (row-major, context precision) to dst, as
 * ls_get_phi.  Errors: LS_EINVAL (NULL, batch context, misaligned device
 * dst), LS_ESTATE (no speed field: none set, or a constant speed). */
int ls_get_speed(ls_ctx *ctx, void *dst, int dst_on_device);

/* Stream-ordered host input/output, for a sequence of problems on one
 * single-grid context (Eq. 1 inputs in, Eq. 3 results out; the transfers
 * overlap the computation as the output of section 2 does): the next
 * problem's inputs travel to the device and the previous result travels
 * back while the current one computes (one copy stream per direction; the
 * transfers overlap the stencil only when the host buffers are
 * page-locked).
 *
 * ls_stage_inputs: start copying phi (row-major, nx*ny*nz values of the
 *   context precision) and, if speed_host is not NULL, the speed field into
 *   device staging buffers; returns at once.  The host buffers must stay
 *   unchanged until ls_load_staged has returned.  LS_ESTATE if inputs are
 *   already staged and not loaded.
 * ls_load_staged: on the context's stream, after those copies, make the
 *   staged arrays the context's phi (and speed field), as ls_set_phi /
 *   ls_set_speed with device sources do (the band is rebuilt at the next
 *   step; LS_ENONFINITE on NaN/Inf; synchronises the context's stream).
 *   LS_ESTATE if nothing is staged.
 * ls_get_phi_async: after the work enqueued so far on the context's
 *   stream, copy the current phi to host_dst (row-major); returns at once.
 *   host_dst is written when ls_wait_host returns.
 * ls_wait_host: wait for every staged copy and read-back to finish.
 * Errors: LS_EINVAL (NULL arguments, batched contexts), LS_ESTATE, LS_ECUDA. */
int ls_stage_inputs(ls_ctx *ctx, const void *phi_host, const void *speed_host);
int ls_load_staged(ls_ctx *ctx);
int ls_get_phi_async(ls_ctx *ctx, void *host_dst);
int ls_wait_host(ls_ctx *ctx);

/* Checkpoint: copy the current phi of every instance into a context-owned
 * device buffer (allocated on the first call).  Errors: LS_ESTATE (phi not
 * set), LS_ENOMEM. */
int ls_snapshot(ls_ctx *ctx);

/* Resume from the last ls_snapshot: phi is restored in both ping-pong
 * buffers and the band becomes stale, exactly as after ls_set_phi with the
 * saved values.  Errors: LS_ESTATE (no snapshot). */
int ls_restore(ls_ctx *ctx);

/* Copy the ascending active tile ids (tile id = (tz*(ny/8) + ty)*(nx/8) + tx)
 * to host array dst of capacity cap; *n receives the count (may exceed cap,
 * then only cap ids are written).  Synchronises the stream.
 * Errors: LS_EINVAL (n == NULL, cap < 0, dst == NULL with cap > 0),
 * LS_ESTATE (no band). */
int ls_get_active_tiles(ls_ctx *ctx, int *dst, long long cap, long long *n);

/* Total grid-point updates done by ls_step since creation (sum over steps of
 * 512 x active tiles).  Synchronises the stream. */
int ls_get_updates(ls_ctx *ctx, unsigned long long *n);

/* Record every later ls_step call as a CUDA graph (on = 1) and replay it
 * when a call starts from the same schedule state with the same arguments;
 * the graph is rebuilt after any change of phi, speed, band, face rule,
 * stream or launch configuration.  Graphs are not used while profiling is
 * enabled.  With the legacy default stream the context uses a private
 * blocking stream for the replays. */
int ls_set_graphs(ls_ctx *ctx, int on);

/* Autotuner: time every launch configuration of the FP32 stencil (points
 * per thread 4 (128-thread CTAs), 8 (64-thread CTAs) or 16 (one warp per
 * tile) x cp.async ring depth 2/3/4/6 x persistent grid 50/75/100 % of full
 * occupancy) on the current
 * active set, `reps` launches each, and keep the fastest for later steps.
 * Every configuration computes the same bits.  The probes write only the
 * buffer the next step overwrites, so the state is unchanged.  Outputs
 * (nullable): the chosen configuration.  Needs a valid band (LS_ESTATE
 * otherwise).  FP64 contexts have a single configuration and return it. */
int ls_autotune(ls_ctx *ctx, int reps, int *stages, int *grid_pct, int *points_per_thread);

/* Steps per stencil pass (FP32 single grids, plain scheme): 1, or 2 -- two
 * upwind steps per pass over the active tiles (temporal blocking: the
 * intermediate step is also computed on the one-cell face layers around
 * each tile, so a pass reads phi and F and writes phi once for two steps);
 * a pair of steps is taken whenever both fall inside one rebuild period,
 * the other steps run one per pass.  The results are the same bits either
 * way.  ls_autotune includes this choice.  Errors: LS_EINVAL. */
int ls_set_steps_per_pass(ls_ctx *ctx, int steps);
int ls_get_steps_per_pass(ls_ctx *ctx, int *steps);

/* Set the FP32 stencil launch configuration directly (stages 2, 3, 4 or 6, grid
 * 1..100 % of full occupancy, points per thread 4, 8 or 16; default 3, 100, 4). */
int ls_set_step_config(ls_ctx *ctx, int stages, int grid_pct, int points_per_thread);

/* Profiling counters of a context. */
typedef struct {
    unsigned long long kernel_launches;  /* library kernels launched by this context */
    unsigned long long stencil_launches; /* of which upwind-step (Eq. 3) launches    */
    double stencil_ms;                   /* summed device time of the step launches
                                            made while profiling was enabled         */
    unsigned long long stencil_timed;    /* number of launches stencil_ms covers     */
    double reinit_ms;                    /* of stencil_ms: reinitialisation passes of
                                            the local scheme (Eq. 12)                */
    unsigned long long reinit_timed;     /* number of launches reinit_ms covers      */
    unsigned long long reinit_updates;   /* point-iterations of the reinitialisation
                                            passes since the local scheme was first
                                            set (they visit only tiles holding a
                                            point of N)                             */
    unsigned long long two_step_points;  /* points passed by two-step passes (each
                                            counted once, updated twice) since the
                                            context was created                     */
    unsigned long long stencil_updates;  /* point updates of the launches stencil_ms
                                            covers (reinitialisation point-iterations
                                            included)                               */
} ls_profile;

/* Enable (on >= 1) or disable (0) CUDA-event timing of the upwind-step
 * launches: one event pair, recorded on the context's stream, brackets a run
 * of back-to-back stencil launches of one kind (the plain step or the local
 * scheme's advance; the reinitialisation passes), so stencil_ms is their
 * summed device time including the gaps between them, stencil_timed the
 * number of launches it covers and stencil_updates their point updates.  Any
 * other kernel ends a run.  on = N times one run in N (the first of every N
 * since the call): an event record between two launches costs the next
 * launch its overlap with the previous one, so sampling disturbs the timed
 * work less.  Errors: LS_EINVAL (on < 0). */
int ls_profile_enable(ls_ctx *ctx, int on);

/* Read the counters (synchronises the stream).  Errors: LS_EINVAL. */
int ls_get_profile(ls_ctx *ctx, ls_profile *out);

/* Zero the counters. */
int ls_reset_profile(ls_ctx *ctx);

/* Sticky device status word: LS_OK, or the first device-side error. */
int ls_get_status(ls_ctx *ctx);

/* Self-test of the bounded device waits used by the tensor-core kernels and
 * by the one-warp stencil's bulk-copy staging: a kernel waits on two
 * barriers that nothing completes, one with each wait, and sets bit 1
 * (timeout) in the device word *status when both gave up after `polls`
 * polls; the context and the device stay usable.  For failure-detection
 * tests. */
int ls_selftest_bounded_wait(unsigned *status, long long polls, void *cuda_stream);

/* Measured FP64 peak of the current device in TFLOP/s (a fused multiply-add
 * counted as 2): independent FMA chains on every SM for `iters` iterations,
 * timed with CUDA events on `cuda_stream` (NULL: the default stream).  The
 * FP64 stencil's roofline is taken against it. */
int ls_probe_dfma(long long iters, double *tflops, void *cuda_stream);

/* Static message for a status code. */
const char *ls_strerror(int status);

/* Last CUDA error code seen by any call (0 = none), for diagnostics. */
int ls_last_cuda_error(void);

/* ---------------------------------------------------------------------
 * Batched contexts: n independent grids advanced together
 * ------------------------------------------------------------------- */

/* Create one context for n independent grids (instance i: nx[i]*ny[i]*nz[i]
 * points, spacing h[i]; same rules as ls_create per instance, 1 <= n <=
 * 65535, total points <= 2^31, precision LS_FP32 only).  All instances share
 * one set of buffers and one global active-tile queue: ls_band_rebuild,
 * ls_step, ls_set_bc, ls_set_full_domain, ls_set_graphs, ls_autotune and the
 * profiling calls act on every instance at once (one stencil launch per step
 * for the whole batch); dt is per instance (CFL mode: CFL*h_i/M_i).  The
 * speeds of all instances must be of one kind (all constant or all fields)
 * when ls_step runs (LS_ESTATE otherwise).  ls_set_phi / ls_set_speed /
 * ls_get_phi need n == 1; use the ls_inst_* calls.  ls_get_active_tiles
 * returns global ids (instance i owns the ids after those of instances
 * 0..i-1). */
int ls_batch_create(int n, const int *nx, const int *ny, const int *nz, const double *h,
                    int precision, ls_ctx **out);

/* Number of instances of a context (1 for ls_create). */
int ls_batch_size(ls_ctx *ctx, int *n);

/* Per-instance versions of ls_set_phi, ls_set_speed, ls_set_speed_const and
 * ls_get_phi (same layout, ownership and errors; i out of range ->
 * LS_EINVAL). */
int ls_inst_set_phi(ls_ctx *ctx, int i, const void *src, int src_on_device);
int ls_inst_set_speed(ls_ctx *ctx, int i, const void *src, int src_on_device);
int ls_inst_set_speed_const(ls_ctx *ctx, int i, double F);
int ls_inst_get_phi(ls_ctx *ctx, int i, void *dst, int dst_on_device);

/* Active tiles of instance i, as local tile ids (ascending); like
 * ls_get_active_tiles. */
int ls_inst_get_active_tiles(ls_ctx *ctx, int i, int *dst, long long cap, long long *n);

/* Per-instance Step 0 fields (as ls_init_phi / ls_init_speed). */
int ls_inst_init_phi(ls_ctx *ctx, int i, int shape, const double *params, int nparams);
int ls_inst_init_speed(ls_ctx *ctx, int i, int kind, const double *params, int nparams);

/* dt of instance i's last step (synchronises the stream). */
int ls_inst_last_dt(ls_ctx *ctx, int i, double *dt);

/* ---------------------------------------------------------------------
 * Overlapped output (section 2: results are written while the computation
 * goes on, by a worker that does nothing else)
 *
 * With an output attached, every `every`-th step of ls_step (counted over
 * the context's lifetime) copies phi into a free device snapshot slot on the
 * context's stream; a copy stream moves it to pinned host memory and a host
 * writer thread writes <prefix><step, 8 digits>.vts (VTK XML StructuredGrid
 * with the point coordinates (i + 1/2) h, as the paper's files) or .vti
 * (ImageData, origin h/2, spacing h), raw appended little-endian data in the
 * context's precision, point data "phi", x fastest.  When all `slots`
 * snapshots are still being written, ls_step waits for one (counted in
 * wait_seconds).  Steps with an output attached run eagerly (no graph
 * replay).  Single-instance contexts only.
 * ------------------------------------------------------------------- */
enum { LS_OUTPUT_VTS = 0, LS_OUTPUT_VTI = 1 };

typedef struct {
    unsigned long long files;   /* files written                                  */
    unsigned long long bytes;   /* bytes written                                  */
    double write_seconds;       /* writer thread time (waiting for the copy, writing) */
    double wait_seconds;        /* time ls_step waited for a free snapshot slot   */
    int status;                 /* first error (LS_EIO, LS_ECUDA) or LS_OK        */
} ls_output_report;

/* Attach the output (1 <= slots <= 8 snapshot buffers of the grid's size on
 * the device and in pinned host memory).  Errors: LS_EINVAL (bad argument or
 * batched context), LS_ESTATE (an output is attached already), LS_ENOMEM. */
int ls_output_open(ls_ctx *ctx, const char *prefix, int every, int format, int slots);

/* Counters so far (the writer may still be busy). */
int ls_output_stats(ls_ctx *ctx, ls_output_report *report);

/* Wait for every queued snapshot to be written, detach the output and
 * release its buffers; report (nullable) gets the final counters.  Returns
 * the first write error (LS_EIO) or LS_OK. */
int ls_output_close(ls_ctx *ctx, ls_output_report *report);

/* Write one row-major host array (context-free; the same file layout as the
 * output above).  Errors: LS_EINVAL, LS_EIO. */
int ls_write_vtk(const char *path, const void *phi, int nx, int ny, int nz, double h,
                 int precision, int format);

/* ---------------------------------------------------------------------
 * Learned coarse-grid corrector (no counterpart in the paper)
 *
 * A small 3-D CNN (4 convolutions 3x3x3: 3 -> 16 -> 16 -> 16 -> 1 channels,
 * ReLU between; BF16 weights and activations on the tensor cores, FP32
 * accumulation, FP32 master parameters) corrects the plain step on a coarse
 * grid: phi~ = plain step of phi^n (Eq. 3), features = [clamp(phi^n/h, +-8),
 * F, (phi~ - phi^n)/h], phi^{n+1} = phi~ + h * CNN(features) on the points of
 * the active tiles.  A residual check rejects a step's correction (keeping
 * phi~, the plain method as fallback) when a corrected value is not finite
 * or |h * CNN| exceeds dt * max|F|.  Training pairs are (phi^n, phi_ref,
 * F) on the coarse grid, phi_ref = the restricted fine-grid plain solution
 * one coarse step later.  The corrected step computes the network only on
 * the blocks of 8 x 16 x 4 points within one tile of an active tile (its
 * four 3x3x3 layers reach 4 cells, so the outputs on the active tiles are
 * those of the whole grid).  Single FP32 contexts with nx and nz multiples
 * of 8 and ny of 16; LS_EINVAL otherwise.
 * ------------------------------------------------------------------- */

/* Number of FP32 parameters of the network (layer l = 0..3: W_l
 * [27][ci][co] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1), then b_l [co]). */
int ls_learned_num_params(long long *n);

/* Seeded Kaiming-uniform weights, zero biases (the last layer scaled by 0.01
 * so the corrector starts near zero); resets the optimiser. */
int ls_learned_init(ls_ctx *ctx, unsigned long long seed);

/* Copy the parameters from / to host memory (n = ls_learned_num_params). */
int ls_learned_set_params(ls_ctx *ctx, const float *src, long long n);
int ls_learned_get_params(ls_ctx *ctx, float *dst, long long n);

/* Store one training pair on the device: coarse row-major FP32 phi^n, the
 * reference phi one coarse step later, and the speed field F. */
int ls_learned_add_pair(ls_ctx *ctx, const float *phi_n, const float *phi_ref, const float *F,
                        int on_device);
int ls_learned_num_pairs(ls_ctx *ctx, long long *n);

/* Load the parameters from a BF16 image (n = ls_learned_num_params values
 * in the parameter layout above, 2 * n bytes, host memory); resets the
 * optimiser.  ls_learned_save writes the current parameters as BF16 (round
 * to nearest even).  Errors: LS_EINVAL (NULL, wrong byte count, unsupported
 * context), LS_ESTATE (save before any parameters exist). */
int ls_learned_load(ls_ctx *ctx, const void *bf16_weights, size_t bytes);
int ls_learned_save(ls_ctx *ctx, void *bf16_weights, size_t bytes);

/* Copy stored pair i out (row-major FP32, host or device memory). */
int ls_learned_get_pair(ls_ctx *ctx, long long i, float *phi_n, float *phi_ref, float *F,
                        int on_device);

/* iters Adam steps (learning rate lr), each on one stored pair drawn with a
 * seeded generator: plain coarse step with fixed dt, forward, MSE of the
 * network output against (phi_ref - phi~)/h over the points with
 * |phi^n| < halfwidth*h, backward, update.  Uses the context's phi and
 * speed as scratch (phi must be set again afterwards).  *final_loss
 * (nullable) = the last iteration's loss. */
int ls_learned_train_stored(ls_ctx *ctx, int iters, double lr, double dt, double halfwidth_in_h,
                            unsigned long long seed, double *final_loss);

/* Training driven by a pair specification: "key=value" items separated by
 * ',' or ';' (pairs_spec may be NULL or empty):
 *   source=stored  train on the stored pairs (default); needs dt
 *   source=fine    first generate pairs on the device and store them: per
 *                  problem a seeded sphere union (2..5 spheres in the middle
 *                  60 % of the box) and an 8-mode Fourier speed (|k|_inf <= 2,
 *                  |F| <= 1), a plain narrow-band run on the 4x finer grid
 *                  (band 4 * halfwidth fine cells, dt_f = cfl * h_f), every 4
 *                  fine steps restricted to this grid as one pair
 *   dt=<double>         coarse step (default for source=fine: cfl * h)
 *   halfwidth=<double>  loss tube and coarse band in cells (default 6)
 *   seed=<integer>      order of the pairs drawn (default 0)
 *   problems=<n>, pairs=<n>, gen_seed=<integer>, cfl=<double>
 *                       generation (defaults 8, 24 per problem, 1, 0.5)
 * then as ls_learned_train_stored.  Needs initialised parameters.  Errors:
 * LS_EINVAL (unknown key, malformed value, missing dt for stored pairs),
 * LS_ESTATE, LS_ENOMEM, LS_ECUDA. */
int ls_learned_train(ls_ctx *ctx, const char *pairs_spec, int iters, double lr,
                     double *final_loss);

/* LS_PLAIN (default) or LS_LEARNED for the steps of ls_step; LS_LEARNED
 * needs initialised parameters (LS_ESTATE). */
int ls_set_step_mode(ls_ctx *ctx, int mode);

/* Number of steps whose correction the residual check rejected. */
int ls_learned_fallbacks(ls_ctx *ctx, unsigned long long *n);

/* Layer primitives on caller-owned device buffers (no allocation):
 * ls_conv3_bf16: x = BF16 [p][16] channels-last (nx a multiple of 8, ny of
 * 16, nz of 4), W = FP32 [27][ci][co] (ci, co <= 16), work = device scratch
 * of LS_CONV3_WORK_BYTES, status = device word that records LS_ETIMEOUT-type
 * failures (bit 1).  mode 0: out = BF16 [p][16] relu(conv(x) + b);
 * mode 1: out = FP32 [p] conv(x)[0] + b[0]; mode 2 (input gradient): out =
 * BF16 [p][16] conv^T(x) * [mask > 0], x = gradient of the layer output,
 * W = the forward weights, mask = BF16 [p][16].
 * ls_conv3_wgrad: dW [27][ci][co] += sum_p x[p + off(tap)] dy[p],
 * db[co] += sum_p dy[p] (db may be NULL), on the tensor cores with FP32
 * accumulation; x and dy BF16 [p][16] (16-byte aligned), nx a multiple of
 * 64; the caller zeroes dW and db; status as for ls_conv3_bf16.
 * ls_restrict4: coarse[I] = mean of the fine points 4I+1, 4I+2 per axis. */
#define LS_CONV3_WORK_BYTES 13824
int ls_conv3_bf16(const void *x, int nx, int ny, int nz, const float *W, int ci, int co,
                  const float *bias, int mode, const void *mask, void *out, void *work,
                  unsigned *status, void *cuda_stream);
int ls_conv3_wgrad(const void *x, const void *dy, int nx, int ny, int nz, int ci, int co,
                   float *dW, float *db, unsigned *status, void *cuda_stream);
int ls_restrict4(const float *fine, int nfx, int nfy, int nfz, float *coarse, void *cuda_stream);

/* The corrector's element-wise steps on caller-owned device buffers (no
 * allocation; asynchronous on cuda_stream).  Not in the paper.
 * ls_learned_features: X = BF16 [n][16] channels-last (16-byte aligned),
 *   channels [clamp(phi / h, -8, 8), F, (phit - phi) / h, 0 ... 0] from FP32
 *   [n] arrays phi (phi^n), phit (the plain step of phi^n, Eq. 3) and F
 *   (NULL: the constant Fc).  LS_EINVAL on NULL inputs, n < 1, h not
 *   finite and positive, Fc not finite, X misaligned.
 * ls_learned_loss_grad: over the tube |phi| < gamma (Eq. 6, compared in
 *   FP64), target t = (phiref - phit) / h; *count = tube size (int),
 *   *loss = sum (z - t)^2 / max(count, 1) (double, summed in FP64),
 *   dz = BF16 [n][16] with channel 0 = 2 (z - t) / max(count, 1) on the
 *   tube and 0 elsewhere, channels 1..15 = 0.  count and loss are device
 *   pointers the call zeroes first.  LS_EINVAL on NULL pointers, n < 1, h
 *   or gamma not finite and positive, dz misaligned.
 * ls_adam_step: one Adam step t >= 1 on FP32 [n] parameters w with
 *   gradient g and moments m, v (updated in place): beta1 0.9, beta2
 *   0.999, eps 1e-8, bias-corrected.  LS_EINVAL on NULL pointers, n < 1,
 *   t < 1, lr not finite and positive. */
int ls_learned_features(const float *phi, const float *phit, const float *F, double Fc, double h,
                        long long n, void *X, void *cuda_stream);
int ls_learned_loss_grad(const float *z, const float *phi, const float *phit, const float *phiref,
                         long long n, double h, double gamma, void *dz, int *count, double *loss,
                         void *cuda_stream);
int ls_adam_step(float *w, const float *g, float *m, float *v, int n, double lr, int t,
                 void *cuda_stream);

/* ---------------------------------------------------------------------
 * Allocation-free band tile list
 * ------------------------------------------------------------------- */

/* Largest tile count (nx/8 * ny/8 * nz/8) ls_band_tiles_noalloc accepts:
 * 2^21 tiles, i.e. a 1024^3 grid. */
#define LS_NOALLOC_MAX_TILES (1 << 21)

/* The paper has no counterpart to this call.  It is for callers that cannot
 * allocate device memory: code running while someone else captures a CUDA
 * graph, allocation-free real-time sections, or hosts whose own memory pool
 * owns the device.  It computes the same active-tile list as
 * ls_band_rebuild + ls_get_active_tiles (tube test min |phi| < halfwidth*h
 * per 8^3 tile in FP64, 26-neighbour dilation, ascending ids), straight from
 * a caller-owned row-major phi, without a context and without any
 * allocation: its scratch (about 4.2 MB of tile flags and block counts) is
 * one fixed __device__ array that every device that loads the library holds
 * until the process exits.
 *   phi        device pointer, nx*ny*nz values of the precision's type,
 *              row-major [z][y][x]; read only.
 *   tiles_out  device pointer to tiles_cap ints (tiles_cap >= number of
 *              tiles); receives the ascending active tile ids.
 *   count_out  device pointer to one int; receives the active-tile count.
 *   cuda_stream  stream the work is queued on (NULL = legacy default).
 * The call is asynchronous: results are valid once the stream has reached
 * the queued work.
 * First call per device: it looks up the scratch array's device address
 * (cudaGetSymbolAddress) and caches it.  Under CUDA's lazy module loading
 * (the default) that lookup loads the library's module on the device and
 * reserves the array there, so the first call does allocate; make it
 * outside any stream capture and outside any allocation-free section (one
 * throwaway call warms a device up).  Later calls on that device allocate
 * nothing.
 * All calls share the one scratch array: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Every scratch byte a call reads it has written first, so nothing
 * needs clearing between calls.
 * Errors: LS_EINVAL (NULL pointer, sizes not multiples of 8 or < 8, h or
 * halfwidth not finite and positive, bad precision, more than
 * LS_NOALLOC_MAX_TILES tiles, tiles_cap too small), all decided on the host
 * before any CUDA call; LS_ECUDA (device query or launch failure).  The
 * call takes each launch's status from the launch itself: it neither reads
 * nor clears the CUDA runtime's pending-error state left by earlier work
 * (a failed launch of its own is also recorded there, as for any runtime
 * call).  Never calls cudaMalloc, cudaFree or any allocating routine. */
int ls_band_tiles_noalloc(const void *phi, int nx, int ny, int nz, double h, int precision,
                          double halfwidth_in_h, int *tiles_out, long long tiles_cap,
                          int *count_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LS_H */

/*
 * hydro.h -- C ABI of libhydro: the directionally split second-order Godunov
 * scheme of the HYDRO mini-application (§1), advanced on one GB300 GPU.
 *
 * The library owns a context holding one or more independent 2D grids of
 * conserved variables U = (rho, rho*u, rho*v, E) (the "2D grid buffer for
 * conservative variables" of Fig. 5).  A time step of every grid is the one
 * §1 and Fig. 5 describe: a 1D Godunov sweep along x over every row, then
 * one along y over every column (the order alternates from step to step),
 * each sweep computing primitive variables, solving a Riemann problem at
 * every cell interface and applying the interface fluxes.  The update of a
 * cell in a sweep reads the cells i-2..i+2 of its line (Figs. 1-2).
 *
 * Conventions shared by every entry point
 *   - Host-side state arrays are FP64, SoA planes [4][ny][nx] in the order
 *     (rho, rho*u, rho*v, E), x fastest, interior cells only (no ghosts).
 *   - Pointers marked "host or device" are device pointers when the call's
 *     on_device argument is non-zero (e.g. a CUDA tensor's data pointer in
 *     the same CUDA context), host pointers otherwise.  Host buffers may be
 *     pageable; page-locked buffers copy faster.
 *   - The caller owns every buffer it passes; the library copies in and out
 *     and keeps no pointer to a caller buffer after a call returns.
 *   - Every call returns a hydro_status; no exception or signal crosses the
 *     ABI.  On failure hydro_last_error(ctx) gives a one-line message.
 *   - A context is used by one host thread at a time.
 *   - Work is enqueued on the context's CUDA stream; calls that return data
 *     to the host synchronise that stream.
 */
#ifndef HYDRO_H
#define HYDRO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hydro_ctx hydro_ctx; /* opaque; owns all device memory */

typedef enum {
    HYDRO_OK = 0,
    HYDRO_EINVAL = 1,    /* bad argument: null pointer, size, index, bc, ... */
    HYDRO_ENOMEM = 2,    /* device or host allocation failed */
    HYDRO_ECUDA = 3,     /* a CUDA runtime call failed (no device, launch error) */
    HYDRO_ENEGATIVE = 4, /* a non-positive or NaN density or energy appeared */
    HYDRO_ETIMEOUT = 5   /* a bounded device-side wait (TMA copy) gave up */
} hydro_status;

/* Boundary conditions of one side (§1/Fig. 5 "apply boundary conditions";
 * 2 ghost cells per side, the stencil width of Figs. 1-2):
 *   REFLECT      mirror image, momentum normal to the wall negated
 *   TRANSMISSIVE mirror image without sign change (zero gradient)
 *   PERIODIC     wrap-around; both sides of an axis must be periodic */
enum { HYDRO_BC_REFLECT = 0, HYDRO_BC_TRANSMISSIVE = 1, HYDRO_BC_PERIODIC = 2 };

enum { HYDRO_PREC_FP32 = 32, HYDRO_PREC_FP64 = 64 };

/* Scheme variants (§1 leaves the details of the scheme to its ref. [5]; the
 * HYDRO code it studies offers these options).  The defaults (0) are the
 * method as this library reads §1: the exact Riemann solver and minmod.
 *   riemann_solver  HYDRO_RIEMANN_EXACT: Newton on the exact pressure
 *                   function (shock and rarefaction branches);
 *                   HYDRO_RIEMANN_TWO_SHOCK: Newton on the two-shock
 *                   approximation (the shock relation for both waves,
 *                   whatever the sign of p - p_K); the state at x/t = 0 is
 *                   sampled from the same wave pattern in both.
 *   slope_type      HYDRO_SLOPE_MINMOD, HYDRO_SLOPE_MC (monotonized central:
 *                   the smallest of 2a, 2b, (a+b)/2 when a, b share a sign),
 *                   HYDRO_SLOPE_NONE (no reconstruction: first-order Godunov).
 *   trace_type      HYDRO_TRACE_MUSCL_HANCOCK: both faces take the whole
 *                   half-step predictor; HYDRO_TRACE_CHARACTERISTIC: the slopes
 *                   are split into the acoustic, entropy and shear waves and
 *                   each face takes only the waves moving toward it. */
enum { HYDRO_RIEMANN_EXACT = 0, HYDRO_RIEMANN_TWO_SHOCK = 1 };
enum { HYDRO_SLOPE_MINMOD = 0, HYDRO_SLOPE_MC = 1, HYDRO_SLOPE_NONE = 2 };
enum { HYDRO_TRACE_MUSCL_HANCOCK = 0, HYDRO_TRACE_CHARACTERISTIC = 1 };

/* One grid: nx * ny interior cells (each in [2, 2^24], and ny times nx
 * rounded up to a multiple of 32 below 2^31), square cells of side h > 0,
 * boundary conditions bc[] = {x low, x high, y low, y high}. */
typedef struct {
    int nx, ny;
    double h;
    int bc[4];
} hydro_grid;

/* Scheme and run parameters.
 *   precision      HYDRO_PREC_FP64: state and arithmetic in FP64.
 *                  HYDRO_PREC_FP32: state and arithmetic in FP32; a Riemann
 *                  problem near vacuum is solved again in FP64; dt and the
 *                  conservation sums are FP64.
 *   gamma          ratio of specific heats (> 1)
 *   cfl            Courant number C of dt = C h / max(max(|u|,|v|) + c)
 *   niter_riemann  maximum Newton iterations of the Riemann solver (the
 *                  iteration stops earlier once it has converged)
 *   rho_floor      density floor (> 0)
 *   c_floor        sound-speed floor: p >= rho c_floor^2 / gamma (> 0)
 *   ngrids, grids  the grids this context advances together (>= 1)
 *   cuda_stream    a cudaStream_t to enqueue on, or NULL for a stream the
 *                  context creates and owns
 *   riemann_solver, slope_type, trace_type  scheme variants (above; 0 = the
 *                  defaults) */
typedef struct {
    int precision;
    double gamma, cfl;
    int niter_riemann;
    double rho_floor, c_floor;
    int ngrids;
    const hydro_grid *grids;
    void *cuda_stream;
    int riemann_solver;
    int slope_type;
    int trace_type;
} hydro_params;

/* Launch shape of the sweep kernels (0 = library default / automatic).
 *   tile_len      y sweep: rows per tile of 32 columns (a multiple of 4)
 *   ctas_per_sm   resident CTAs per SM of the persistent sweep launches
 *                 (at most the occupancy limit)
 *   graph_steps   steps captured per CUDA graph (even, 0 = no graph)
 *   span_len      x sweep: results of a row per warp task (a multiple of 60).
 *                 FP32: a warp walks a row in overlapping 64-cell segments
 *                 that yield 60 results each.  FP64: a warp walks 32 rows
 *                 at once, a lane per row, over span_len cells.
 *   fused         0: a step is two sweep launches, one per direction (the
 *                 state crosses HBM once per sweep).  1: a step is one
 *                 launch of the fused step kernel, which sweeps both
 *                 directions of a tile of 60 columns x 32 rows held in
 *                 shared memory (its input box with 2 halo cells on each
 *                 side crosses HBM once per step; the halo rows or columns
 *                 are swept by both tiles that hold them).  Same results
 *                 bit for bit; tile_len and span_len do not apply.
 * tile_len = 0 (default) and span_len = 0 take the tile length with the
 * best makespan of a list-scheduling model of the tile queue on the
 * resident warps (uniform cost per cell).  In FP64 contexts they also make
 * the tiles of their direction adaptive (tile_len: y, span_len: x): every
 * sweep records an estimate of the work (Newton iterations, powers, copies
 * of uniform cells) spent on each tile, spread over its cost blocks (a row
 * of a 32-column group in y, 4 columns of a 32-row group in x), and before
 * the next sweep in that direction the library splits each model tile into
 * pieces whose recorded work stays below the mean work of a model tile
 * (pieces reaching half that work and half the largest piece of the
 * previous sweep are queued first, spread over the SMs), so regions where
 * the Riemann solver works harder get shorter tiles.  The tiling follows
 * the state, not the timing.  Results are bit-identical for every
 * admissible setting (a cell's update does not depend on the schedule). */
typedef struct {
    int tile_len;
    int ctas_per_sm;
    int graph_steps;
    int span_len;
    int fused;
} hydro_tuning;

/* Counters kept on the device since hydro_init (hydro_stats()).
 *   steps          completed steps
 *   riemann_fp64   FP32 contexts: interface solves redone in FP64 near vacuum
 *   status_flags   bit 0: non-positive/NaN density, bit 1: non-positive/NaN
 *                  energy, bit 2: a bounded wait timed out, bit 3: internal
 *                  error, a tile outside its grid was skipped (sticky until
 *                  hydro_set_state)
 *   kernel_launches  kernels the step calls launched (host count; a step of
 *                  an FP64 context launches 6 with adaptive x and y tiles, of
 *                  an FP32 context 5; a fused step 3)
 *   wait_site, wait_tile  the first bounded wait that gave up since the last
 *                  hydro_set_state: kernel (0 none, 1 x sweep, 2 y sweep,
 *                  3 fused step, 4 its FP32 second pass) and work-list tile */
typedef struct {
    long long steps;
    long long riemann_fp64;
    unsigned int status_flags;
    long long kernel_launches;
    int wait_site, wait_tile;
} hydro_stats;

/* Create a context (the "2D grid buffer for conservative variables" of
 * Fig. 5 and the scheme parameters of §1): validates params, allocates two
 * state buffers (the step ping-pongs between them) for all grids plus the
 * per-grid dt/time records, and builds the tile work-lists.  The state is zero until hydro_set_state.
 * Returns HYDRO_EINVAL for invalid params, HYDRO_ECUDA when no usable GPU is
 * present, HYDRO_ENOMEM when allocation fails; *out is NULL on failure. */
hydro_status hydro_init(const hydro_params *params, hydro_ctx **out);

/* Release the context and all its device memory.  NULL is a no-op. */
void hydro_destroy(hydro_ctx *ctx);

/* Choose the launch shape (see hydro_tuning).  The paper's counterpart is
 * the choice of domain sizes and task granularity of its CPU versions
 * (§3-§6); here it only changes the schedule, never a result.  HYDRO_EINVAL
 * for values out of range.  Applies to later hydro_step calls. */
hydro_status hydro_set_tuning(hydro_ctx *ctx, const hydro_tuning *tuning);

/* Failure detection (the paper has no counterpart; its MPI/OpenMP runs have
 * no bounded waits).  Every wait of a sweep warp for a TMA copy into shared
 * memory gives up after `polls` polls of its mbarrier; the warp then records
 * the timeout, waits for its own copies still in flight (at most the default
 * number of polls each) and leaves the kernel, and the hydro_step call that
 * launched it returns HYDRO_ETIMEOUT.  The state is then undefined until the
 * next hydro_set_state; the context stays usable.  polls < 0 restores the
 * default (2^22, far above any real copy's latency).  A small value exists
 * to exercise this path: polls = 0 makes every sweep give up at its first
 * wait.  HYDRO_EINVAL for polls >= 2^32.  Synchronises the context's stream;
 * applies to later hydro_step calls. */
hydro_status hydro_set_wait_limit(hydro_ctx *ctx, long long polls);

/* Load the state of grid `grid` from U (host or device, [4][ny][nx] FP64).
 * Resets the grid's time to 0 and the context's step counter (which sets the
 * sweep order) to 0, clears the status flags, and computes the CFL wave
 * speed of the new state.  FP32 contexts round U to FP32. */
hydro_status hydro_set_state(hydro_ctx *ctx, int grid, const double *U, int on_device);

/* Copy the current state of grid `grid` into U_out (host or device,
 * [4][ny][nx] FP64).  Synchronises the context's stream. */
hydro_status hydro_get_state(hydro_ctx *ctx, int grid, double *U_out, int on_device);

/* Rows [row0, row0 + nrows) of grid `grid`: write them from U (host or
 * device, FP64 [4][nrows][nx], x fastest), or read them into U_out.  Used
 * to exchange the ghost rows of a grid split into slabs across processes
 * (the subdomain interface buffers of §5, Fig. 10; the Coarse-Grain
 * decomposition of §3): hydro_set_rows then recomputes the grid's CFL wave
 * speed over all its cells (so hydro_cfl_dt and the next step's dt see the
 * new rows), and changes neither the step counter nor the time.  FP32
 * contexts round U to FP32.  HYDRO_EINVAL for rows outside the grid.
 * Synchronise the context's stream. */
hydro_status hydro_set_rows(hydro_ctx *ctx, int grid, int row0, int nrows, const double *U, int on_device);
hydro_status hydro_get_rows(hydro_ctx *ctx, int grid, int row0, int nrows, double *U_out, int on_device);

/* Advance every grid by nsteps steps (§1, Fig. 5).  Step k (counted from the
 * last hydro_set_state) sweeps x then y when k is even and y then x when k
 * is odd; both sweeps use the step's dt.  dt is each grid's CFL step of the
 * state at the start of the step, unless dt_override (host, nsteps * ngrids
 * values, step-major: dt_override[s * ngrids + g]) is given.  Returns
 * HYDRO_ENEGATIVE when a non-positive or NaN density or energy appeared (the
 * state is then the one after the last step; the context stays usable).
 * Synchronises the context's stream once at the end to read the status. */
hydro_status hydro_step(hydro_ctx *ctx, int nsteps, const double *dt_override);

/* hydro_step that also returns the dt each grid used at each step in
 * dt_used (host, nsteps * ngrids values, step-major) when non-NULL. */
hydro_status hydro_step_dt(hydro_ctx *ctx, int nsteps, const double *dt_override,
                           double *dt_used);

/* hydro_step without graph capture that also times every kernel launch
 * with CUDA events on the context's stream: kernel_ms (host, 3 * nsteps
 * values) receives, per step, the durations of the dt prologue, the first
 * sweep and the second sweep in milliseconds.  Same results as hydro_step. */
hydro_status hydro_step_profiled(hydro_ctx *ctx, int nsteps, double *kernel_ms);

/* CFL time step dt = C h / max over cells of (max(|u|,|v|) + c) of the
 * current state of grid `grid` (FP64). */
hydro_status hydro_cfl_dt(hydro_ctx *ctx, int grid, double *dt_out);

/* Simulated time of grid `grid` (sum of the dt it was advanced by). */
hydro_status hydro_get_time(hydro_ctx *ctx, int grid, double *t_out);

/* Step counter since the last hydro_set_state (its parity sets the sweep
 * order of the next step).  hydro_set_step restores it when a run resumes
 * from a checkpoint (hydro_get_state + hydro_get_step + hydro_get_time);
 * step >= 0. */
hydro_status hydro_get_step(hydro_ctx *ctx, long long *step_out);
hydro_status hydro_set_step(hydro_ctx *ctx, long long step);

/* Set the simulated time of grid `grid` (checkpoint restore). */
hydro_status hydro_set_time(hydro_ctx *ctx, int grid, double t);

/* Domain totals h^2 * sum over cells of each conserved variable of grid
 * `grid`, in FP64 and in a fixed summation order (bit-reproducible). */
hydro_status hydro_conservation(hydro_ctx *ctx, int grid, double sums[4]);

/* Domain totals h^2 * sum over cells of each conserved variable of a state
 * the caller holds on the device, computed without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run (work recorded into a stream
 * capture or CUDA graph, where cudaMalloc/cudaFree are not allowed; loops
 * with hard latency limits, since cudaMalloc/cudaFree can synchronise the
 * device; plugins whose host framework owns all GPU memory) and so cannot
 * create a hydro_ctx.
 *   U          device, FP64 [4][ny][nx] (rho, rho*u, rho*v, E), x fastest
 *   nx, ny     >= 1; ny <= 32768 (larger ny returns HYDRO_EINVAL)
 *   h          cell size (> 0)
 *   sums       device, 4 doubles, written with the totals
 *   cuda_stream  stream to enqueue on (NULL: the legacy default stream)
 * Asynchronous on the stream; same summation order, hence the same bits, as
 * hydro_conservation on an FP64 context holding the same state.  It calls no
 * cudaMalloc, cudaFree or allocating library routine: the per-row partial
 * sums live in a fixed 1 MiB device array that every GPU loading the library
 * keeps until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress, with the device current);
 * make that first call before any stream capture.  Every call shares the
 * array (each call overwrites the rows it uses), so calls that overlap on
 * the GPU -- on different streams, or from several threads -- race.
 * Returns HYDRO_EINVAL for null pointers or bad sizes, HYDRO_ECUDA if the
 * device or the launch fails.  hydro_last_error does not report on it. */
hydro_status hydro_conservation_noalloc(const double *U, int nx, int ny, double h, double *sums,
                                        void *cuda_stream);

/* Device counters (see hydro_stats): the run's bookkeeping, which the
 * paper's timings of whole runs (§7) leave to the host. */
hydro_status hydro_get_stats(hydro_ctx *ctx, hydro_stats *out);

/* Message of the last failure on this context ("" if none); valid until the
 * next call on ctx.  With ctx == NULL: the last hydro_init failure.  (Error
 * reporting of the ABI; the paper has no counterpart.) */
const char *hydro_last_error(const hydro_ctx *ctx);

/* Library version, "major.minor.patch" (the paper has no counterpart). */
const char *hydro_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HYDRO_H */

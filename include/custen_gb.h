/*
 * custen_gb.h -- C ABI of the GB300-native cuSten hot path (arXiv:1902.09931).
 *
 * The library applies finite-difference stencils to 2D grids and ragged batches of 1D lines
 * (Sec. 2-4) and advances the periodic Cahn-Hilliard ADI scheme of Sec. 5.1.  Its verbs follow
 * the paper's Create / Compute / Swap / Destroy API (Sec. 3), with the x / y / xy direction,
 * the periodic / non-periodic boundary and the weights-or-function choice passed as values
 * instead of being spelled into sixteen function names.
 *
 * Memory and streams.  Every field buffer is allocated and owned by the caller in device
 * memory (PyTorch tensors, cudaMalloc, ...), must be contiguous, 16-byte aligned for the fast
 * path (any alignment of the element type is accepted), and must stay alive until the plan
 * that references it is destroyed.  Layout of a 2D field: row-major, x fastest, element (j, i)
 * at index j * nx + i (the contiguous y-tiles of Sec. 2).  All compute calls are asynchronous
 * with respect to the host and ordered on the CUDA stream passed in (NULL = legacy default
 * stream), except where a call says it synchronises.  A plan may be used from one host thread
 * at a time; different plans are independent.  Unlike the paper there is no HOST/DEVICE flag
 * and no y-tile count: fields stay resident in device memory (Sec. 2's Unified-Memory
 * streaming is not needed when the whole grid fits in HBM).  cs_compute_host() is the
 * host-buffer form of Compute for callers whose data lives in host memory, and
 * cs_plan_create_2d_host() streams grids of any size through bounded device memory.
 *
 * Errors.  Every call returns CS_OK (0) or a negative cs_status.  Nothing aborts or exits.
 * cs_last_error() returns a description of the last failure on the calling host thread.
 * Invalid arguments leave every buffer untouched.  CS_ECUDA reports a CUDA runtime error
 * (launch failure, invalid device pointer); the plan stays valid unless the error is sticky.
 */
#ifndef CUSTEN_GB_H
#define CUSTEN_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cs_plan* cs_plan_t; /* opaque; created and freed by the library */

typedef enum {
  CS_OK = 0,
  CS_EINVAL = -1,       /* invalid argument (sizes, extents, enum values, null pointers) */
  CS_EALIAS = -2,       /* input and output overlap: Sec. 2 requires distinct buffers */
  CS_ENOMEM = -3,       /* library-owned workspace could not be allocated */
  CS_ECUDA = -4,        /* a CUDA runtime call failed */
  CS_EUNSUPPORTED = -5, /* valid request that this build does not implement */
  CS_ETIMEOUT = -6      /* a bounded device-side wait ran out (cs_plan_check, cs_compute_host) */
} cs_status;

/* Direction of a 2D stencil (Sec. 3: X, Y, XY).  XY stencils read corner halos. */
typedef enum { CS_DIR_X = 0, CS_DIR_Y = 1, CS_DIR_XY = 2 } cs_dir;

/* Boundary treatment (Sec. 3: p / np).  Periodic wraps indices modulo the grid size.
 * Non-periodic leaves every output cell whose stencil would leave the grid untouched
 * (cells with i < left, i >= nx - right, j < top, j >= ny - bottom; Sec. 3 and Sec. 4.1). */
typedef enum { CS_BC_NONPERIODIC = 0, CS_BC_PERIODIC = 1 } cs_bc;

/* Storage (and stencil arithmetic) type of the fields.  CS_F32 stencils compute in FP32;
 * Cahn-Hilliard line solves and reductions always run in FP64. */
typedef enum { CS_F64 = 0, CS_F32 = 1 } cs_dtype;

/* The "Fun" variant (Sec. 4.2, Sec. 5.2).  The paper takes a user device-function pointer
 * double f(double* data, double* coe, int loc); this library compiles a fixed set of
 * functions into its kernels instead (so they inline into the tiled sweep) and takes their
 * coefficients `coe` at create time.  Each function fixes its own footprint.
 *   CS_FN_CENTRAL_D2X      Sec. 4.2 example: (u[i-1] - 2u[i] + u[i+1]) * coe[0], X, 1 left/right
 *   CS_FN_CH_NONLIN_LAP    Sec. 5.2: 5-point Laplacian of N = u^3 - u, coe[0] = 1/h^2, XY, r = 1
 *   CS_FN_CUBIC_MINUS_LAP  u^3 - u - (5-point Laplacian of u), coe[0] = 1/h^2, XY, r = 1 */
typedef enum {
  CS_FN_NONE = 0,
  CS_FN_CENTRAL_D2X = 1,
  CS_FN_CH_NONLIN_LAP = 2,
  CS_FN_CUBIC_MINUS_LAP = 3
} cs_fn;

/* Stencil description (Sec. 3, Sec. 4.1).  Enumerations are carried as int32_t.
 *   nx, ny     grid size (ny = 1 allowed); ignored (nx) by cs_plan_create_1d_batch
 *   dir        cs_dir; X requires top = bottom = 0, Y requires left = right = 0
 *   bc         cs_bc
 *   dtype      cs_dtype of the in / out buffers
 *   left, right, top, bottom
 *              stencil points on each side of (i, j) (numStenLeft / numStenRight and the y
 *              analogues of Sec. 4.1); any non-negative values up to CS_MAX_EXTENT, asymmetric
 *              allowed; periodic grids smaller than the stencil wrap more than once.
 *   weights    host array of (left+right+1)*(top+bottom+1) values for fn == CS_FN_NONE,
 *              numbered from the top-left of the stencil box, left to right in i, then row by
 *              row in j (Sec. 5.2); the first row is j - top.  Copied at create time.
 *              A zero weight is not part of the stencil: its tap is not evaluated, so an inf
 *              or nan there does not reach the output.
 *   fn, coe, num_coe
 *              user-function variant; coe (host, num_coe values) is copied at create time.
 *              When fn != CS_FN_NONE, weights must be NULL and the extents must equal the
 *              function's footprint. */
#define CS_MAX_EXTENT 16
typedef struct {
  int64_t nx, ny;
  int32_t dir, bc, dtype;
  int32_t left, right, top, bottom;
  const double* weights;
  int32_t fn;
  int32_t num_coe;
  const double* coe;
} cs_stencil_desc;

/* Create (Sec. 3): validates the description, copies weights / coefficients, picks the kernel
 * variant and tile shape, and binds the caller's device buffers d_in (read) and d_out
 * (written).  d_in and d_out must not overlap (CS_EALIAS): blocks read overlapping halos, so
 * outputs cannot be written in place (Sec. 2).  One compute covers the grid in one launch:
 * ny <= 2,097,120 rows (cs_compute returns CS_EUNSUPPORTED beyond; cs_plan_create_2d_host
 * streams taller grids in bands). */
int cs_plan_create_2d(cs_plan_t* plan, const cs_stencil_desc* desc, const void* d_in, void* d_out);

/* Create for a ragged batch of 1D lines (Abstract; Sec. 5.4's batched 1D problems): line m
 * occupies elements [offsets[m], offsets[m+1]) of the packed buffers.  desc->dir must be
 * CS_DIR_X (top = bottom = 0); a periodic stencil wraps at each line's own length.
 *   d_offsets  device array of num_lines + 1 int64 values, non-decreasing, offsets[0] = 0,
 *              offsets[num_lines] = total_len, every line shorter than 2^31 elements.  Read at create time (the library builds its
 *              load-balancing table from it) and by every compute; must stay alive.
 *   total_len  number of packed elements. */
int cs_plan_create_1d_batch(cs_plan_t* plan, const cs_stencil_desc* desc, int64_t num_lines,
                            const int64_t* d_offsets, int64_t total_len, const void* d_in,
                            void* d_out);

/* Compute (Sec. 3): applies the stencil, d_in -> d_out, stream-ordered and asynchronous.  A
 * non-periodic FP64 2D plan on the digit path runs the border ring of its tiles on a stream the
 * plan owns, forked from cuda_stream and joined back into it by two events, so work issued on
 * cuda_stream afterwards still follows the whole sweep. */
int cs_compute(cs_plan_t plan, void* cuda_stream);

/* Grouped Compute: applies `count` 2D stencil plans -- independent grids of any sizes -- in one
 * persistent kernel launch per 64 plans: the launch has as many CTAs as the GPU holds at once,
 * and each walks the tiles of all grids in turn.  The plans must share dtype, stencil shape
 * (left/right/top/bottom and the non-zero tap pattern, i.e. the same specialised kernel) and
 * tile shape; CS_EINVAL otherwise, CS_EUNSUPPORTED for plans on the generic kernel.  Each tile
 * is evaluated as cs_compute's cp.async tiles of the same height evaluate it, so results are
 * those of the plans computed alone with that tile choice, bit for bit: FP32 storage in FP32, FP64
 * storage on the exact digit path when every plan allows it (integer weight ratios, or the cubic
 * user function; CS_FP64_AUTO), else in native FP64.  Allocates nothing and never synchronises,
 * so the call can be captured into a CUDA graph (the graph keeps the plans' buffers of capture
 * time).  Used by the serving loop to batch small sweeps.  Stream-ordered and asynchronous. */
int cs_compute_group(const cs_plan_t* plans, int32_t count, void* cuda_stream);

/* Periodic XY WENO advection (Sec. 4.2, "Advection"): the XY periodic stencil variant whose
 * inputs are a field C and velocities u, v, and whose per-point solver is the fifth-order WENO
 * scheme for Hamilton-Jacobi equations of the reference the paper cites (Osher & Fedkiw, Sec. 3.4).
 * Compute writes the advection term
 *     out = u * C_x + v * C_y
 * with each derivative upwinded: the left-biased WENO5 approximation (points i-3 .. i+2) where
 * the velocity component is > 0, the right-biased one (i-2 .. i+3) elsewhere; eps = 1e-6 *
 * max(v_k^2) + 1e-99 over the five differences (the floor is left out with FP32 storage).  A
 * time stepper advances C_t = -out.  All four fields are n_y x n_x, row-major (x fastest),
 * periodic in both directions, of the description's dtype; arithmetic in that dtype.
 *   hx, hy    grid spacings, in [1e-60, 1e60] (CS_EINVAL otherwise).
 *   d_out     must not overlap d_c, d_u or d_v (CS_EALIAS); the three inputs are only read.
 * cs_compute runs one kernel (CS_EUNSUPPORTED when ny > 2,097,120 rows, the launch's limit);
 * graph replay applies; cs_swap, cs_set_buffers and cs_compute_host do not (CS_EINVAL);
 * cs_autotune leaves the plan unchanged. */
typedef struct {
  int64_t nx, ny;
  int32_t dtype;    /* CS_F64 or CS_F32 */
  int32_t reserved;
  double hx, hy;
} cs_weno_desc;
int cs_plan_create_weno_adv(cs_plan_t* plan, const cs_weno_desc* desc, const void* d_c,
                            const void* d_u, const void* d_v, void* d_out);

/* Create for a 2D grid that lives in host memory (Sec. 2's y-tile streaming of grids larger
 * than device memory).  The plan owns a ring of 3 band slots in device memory, each holding
 * input and output for a band of rows plus halo rows; cs_compute_host then streams the grid
 * through them -- copy in, sweep, copy out on three streams, overlapped -- so device memory
 * stays bounded by device_bytes whatever the grid's size.
 *   desc          as for cs_plan_create_2d; ny >= 128 (CS_EINVAL otherwise).
 *   device_bytes  device memory the slots may use (0 = 512 MiB).  Band height = the largest
 *                 multiple of 64 rows that fits (at most the grid, rounded up to 64); CS_EINVAL
 *                 when not even 64 rows fit, CS_ENOMEM when the allocation fails.
 * Results equal a device-buffer plan's sweep (same description, tile choice and FP64 mode) bit
 * for bit; for a non-periodic plan, host output cells of the boundary rows and columns are left
 * untouched.  cs_compute, cs_swap, cs_set_buffers and graph replay do not apply (CS_EINVAL /
 * CS_EUNSUPPORTED); cs_autotune leaves the plan unchanged; tile choice and FP64 mode may be set. */
int cs_plan_create_2d_host(cs_plan_t* plan, const cs_stencil_desc* desc, int64_t device_bytes);

/* Band height in rows and device bytes held by a host-resident plan (either output may be
 * NULL); CS_EINVAL for any other plan. */
int cs_plan_host_info(cs_plan_t plan, int64_t* band_rows, int64_t* device_bytes);

/* Compute with host buffers (Sec. 3's HOST flag): copies h_in (host, the full input field)
 * into the plan's device input, computes, and copies the device output back into h_out.
 * Either pointer may be NULL to skip that copy.  A 2D plan of 16 MB or more with both pointers
 * set is processed in row bands whose copy-in, sweep and copy-out overlap on streams the plan
 * owns (the results equal a device sweep bit for bit); the device input then holds the copied
 * field and the device output the result, as with one copy.  Pinned host memory is needed for
 * the overlap; pageable memory works but is slower.  Synchronises the stream before returning
 * when h_out is non-NULL.  For a host-resident plan (cs_plan_create_2d_host) both pointers are
 * required (full host fields, not overlapping, CS_EALIAS otherwise) and the grid streams through
 * the plan's band slots; pinned host memory gives the overlap. */
int cs_compute_host(cs_plan_t plan, const void* h_in, void* h_out, void* cuda_stream);

/* Swap (Sec. 3): exchanges the bound input and output buffers so the next Compute reads what
 * the last one wrote. */
int cs_swap(cs_plan_t plan);

/* Arithmetic used for CS_F64 stencils (GB300 issues FP64 at 1/64 of the FP32 rate).
 * CS_FP64_AUTO (default), for the specialised stencils:
 *   - weights w_k = c * n_k with integers n_k, sum |n_k| <= 64 (every stencil of the paper):
 *     exact digit evaluation -- each value cut into two 24-bit integer digits on a grid
 *     set by the largest value of its tile (tile = 64 x TY outputs plus halo; bits below 2^-48
 *     of the grid's top dropped), digit sums exact in int32, their combination rounded to 2^-44
 *     of the grid's top and scaled with one FP64 FMA (c rounded to 51 bits, so that its
 *     constants are exact); error at most (2^-47 + 2^-44 / sum|n_k| + 2^-50) of
 *     sum|w| * (largest |value| in the tile and its halo);
 *   - other weights: double-float arithmetic (values as unevaluated float pairs, error-free
 *     products and sums on the FP32 pipes); error below ~2^-46 of sum|w| * max|in|;
 *   tiles holding inf / nan or values outside the methods' exponent ranges, and weights
 *   outside [2^-60, 2^50), are evaluated in native FP64.
 * CS_FP64_NATIVE always uses FP64 instructions (each output accurate on its own
 * neighbourhood's scale).  CS_F32 plans ignore this. */
typedef enum { CS_FP64_AUTO = 0, CS_FP64_NATIVE = 1 } cs_fp64_mode;
int cs_plan_set_fp64_mode(cs_plan_t plan, int32_t mode);

/* Tile / pipeline shape of a 2D stencil plan (normally picked by cs_autotune):
 *   0  tiles of 32 rows staged with cp.async, one tile per CTA
 *   1  tiles of 64 rows staged with cp.async, one tile per CTA
 *   2  TMA-pipelined persistent sweep: tiles of 64 rows, each CTA walks its tiles through a
 *      two-stage shared-memory ring filled by tensor-memory-access copies (default; used when
 *      nx is a multiple of 16 bytes / element size and d_in is 16-byte aligned, else 1).
 * Choices 1 and 2 give the same results bit for bit (the same tiles).  Choice 0 does too for
 * FP32 storage; on the FP64 integer-digit path its digit grid is set by 32-row tiles, so results
 * can differ from choices 1 and 2 within that path's error bound.  CS_EINVAL for another value. */
int cs_plan_set_tile_choice(cs_plan_t plan, int32_t choice);
int cs_plan_get_tile_choice(cs_plan_t plan, int32_t* choice);

/* Completion check of a plan's work (no counterpart in the paper: it reports the bounded waits
 * of this library's TMA pipeline).  Waits for cuda_stream, then returns CS_ETIMEOUT if, since
 * the previous check, a TMA-pipelined sweep of this 2D plan (tile choice 2) had an mbarrier wait
 * run out: the CTAs concerned returned early and part of that sweep's output was not written.
 * The count lives in a 4-byte device word the plan owns, so plans (and the streams they run on)
 * do not mask one another.  cs_compute_host runs this check itself.  Returns CS_OK otherwise,
 * for every plan kind. */
int cs_plan_check(cs_plan_t plan, void* cuda_stream);

/* Test hook for cs_plan_check (no counterpart in the paper): from CTA-local tile index `tile`
 * on, the TMA sweep of this 2D device plan issues no copies, so each CTA's wait for such a tile
 * runs out (after a short bounded wait, with no copy in flight) and the sweep returns early;
 * tile < 0 (the default) turns it off.  CS_EINVAL for other plans. */
int cs_plan_debug_stall(cs_plan_t plan, int32_t tile);

/* Rebinds the device buffers of a stencil plan without re-planning (same sizes and dtype). */
int cs_set_buffers(cs_plan_t plan, const void* d_in, void* d_out);

/* Captures the plan's compute into a CUDA graph on first use and replays it afterwards
 * (enable = 1), or launches kernels directly (enable = 0, the default).  The graph is rebuilt
 * automatically after cs_swap / cs_set_buffers. */
int cs_plan_use_graph(cs_plan_t plan, int enable);

/* Times the candidate tile / launch shapes of the plan's kernel on its own buffers (it
 * overwrites d_out), each launch from a cold L2 (the first call allocates a 256 MB buffer that
 * the library reads to evict the cache, kept until exit), keeps the fastest, and records it in
 * the process-wide tuning table.  For a Cahn-Hilliard plan it times one ADI step for every
 * valid number of chunks per line (the line-solve partition) from the plan's current state and
 * restores the fields afterwards.  The
 * table is keyed by (kernel, dtype, shape class, SM count) and can be saved to / loaded from a
 * JSON file with cs_tune_save / cs_tune_load.  Synchronises the stream. */
int cs_autotune(cs_plan_t plan, void* cuda_stream);
int cs_tune_save(const char* path);
int cs_tune_load(const char* path);

/* Destroy (Sec. 3): frees the plan and the workspace the library allocated.  Never frees the
 * caller's buffers.  Destroying NULL is a no-op. */
int cs_destroy(cs_plan_t plan);

/* ---- Cahn-Hilliard ADI (Sec. 5.1) on (0, 2 pi)^2, periodic or with no-flux boundaries --------
 * One step:  Cbar = 2 C^n - C^{n-1};
 *            RHS = -(2/3)(C^n - C^{n-1}) - (2/3) D gamma dt lap4(Cbar) + (2/3) D dt lap2(C^3 - C)^n;
 *            L_x w = RHS;  L_y v = w;  C^{n+1} = Cbar + v;  L = I + (2/3) D gamma dt d^4
 * with second-order central differences (Eq. 5), h = 2 pi / n, and cyclic pentadiagonal line
 * solves (Sec. 5.1).  The printed right-hand side omits D gamma on the lap4 term; the library
 * uses the coefficient of L_x, the reading under which steady states of the scheme are steady
 * states of the equation.
 *   n        grid points per side (n x n), a multiple of 64 in [64, 65536]
 *   storage  CS_F64, or CS_F32 (fields stored in FP32, stencils in FP32, solves in FP64)
 *   D, gamma mobility and interface parameter (Sec. 5.3: 1.0 and 0.01)
 *   dt       time step (Sec. 5.3: 0.1 h)
 *   boundary CS_CH_PERIODIC (0, the paper's case) or CS_CH_NOFLUX: the same scheme on a
 *            bounded domain, the np stencils plus a boundary treatment (Sec. 4's pattern) --
 *            cell-centred points x_i = (i + 1/2) h, every stencil reading ghost cells by even
 *            reflection (C_{-1-k} = C_k, C_{n+k} = C_{n-1-k}: dC/dn = 0 and d(lap C)/dn = 0,
 *            so no mass crosses the boundary), and non-cyclic line solves with
 *            L = I + a D4, D4 the reflected fourth difference (rows (2,-3,1), (-3,6,-4,1),
 *            then (1,-4,6,-4,1), mirrored at the far end).  Mass and energy are as for periodic
 *            fields, the forward difference across the boundary being zero. */
typedef enum { CS_CH_PERIODIC = 0, CS_CH_NOFLUX = 1 } cs_ch_boundary;
typedef struct {
  int64_t n;
  int32_t storage;
  int32_t boundary; /* cs_ch_boundary */
  double D, gamma, dt;
} cs_ch_desc;

/* Binds three caller-owned n x n device fields.  On entry d_c_prev holds C^{n-1} and d_c_cur
 * holds C^n; for the first step of a run pass the initial condition in both (Sec. 5.1 sets
 * C^{-1} = C^0).  d_c_next is workspace that receives C^{n+1}.  The plan rotates the three
 * buffers after every step; cs_ch_fields reports where C^{n-1} and C^n currently live. */
int cs_ch_create(cs_plan_t* plan, const cs_ch_desc* desc, void* d_c_prev, void* d_c_cur,
                 void* d_c_next);

/* Advances nsteps ADI steps on the stream.  When h_mass / h_energy are non-NULL they receive,
 * for each step s, the mass h^2 sum C and the free energy of Eq. (1) (forward differences,
 * rectangle rule) of the field after step s, computed in FP64 on the device; the call then
 * synchronises the stream.  With both NULL the call is asynchronous. */
int cs_ch_step(cs_plan_t plan, int64_t nsteps, double* h_mass, double* h_energy, void* cuda_stream);

/* Mass and free energy of the current field C^n (synchronises the stream). */
int cs_ch_invariants(cs_plan_t plan, double* mass, double* energy, void* cuda_stream);

/* Coarsening measures of the current field C^n (Sec. 5.1, "Numerical Results"), both in FP64:
 *   *s  = 1 / (1 - <C^2>), <.> the domain average by Simpson's rule applied per direction on the
 *         periodic grid (the point 2 pi coincides with the point 0, so every even-index point has
 *         weight 2 and every odd-index point weight 4, total 3 n per direction);
 *   *k1 = sum |C^(k)|^2 / sum |k|^-1 |C^(k)|^2 over the n x n discrete wavenumbers of the 2D DFT
 *         (signed, |k| <= n / 2), with k = (0, 0) left out of both sums.
 * Either output may be NULL.  Requires a periodic plan, n a power of two and n <= 8192 (CS_EUNSUPPORTED
 * otherwise); uses the plan's n x n scratch, so it may be called only between steps on the
 * plan's stream.  The first call allocates 4 n + 4 doubles of device memory (CS_ENOMEM on
 * failure), held until cs_destroy.  Synchronises the stream. */
int cs_ch_coarsening(cs_plan_t plan, double* s, double* k1, void* cuda_stream);

/* Current device pointers of C^{n-1} and C^n (either output may be NULL), and the number of
 * steps taken since create. */
int cs_ch_fields(cs_plan_t plan, void** d_c_prev, void** d_c_cur, int64_t* steps_taken);

/* Rebinds a Cahn-Hilliard plan to three other caller-owned n x n fields (same meaning as in
 * cs_ch_create; the step count restarts at 0).  Lets a caller keep a plan -- and its device
 * workspace -- for many runs of the same grid size without allocating again. */
int cs_ch_set_fields(cs_plan_t plan, void* d_c_prev, void* d_c_cur, void* d_c_next);

/* Line-solve partition of a Cahn-Hilliard plan: every periodic line of n points is split into
 * *chunks pieces of *chunk_len points (see cs_ch_create); either output may be NULL. */
int cs_ch_config(cs_plan_t plan, int32_t* chunks, int32_t* chunk_len);

/* ---- a Cahn-Hilliard grid decomposed into row bands (one process per GPU) -------------------
 * The paper's route to several GPUs (Sec. 6.2) splits the grid into bands of rows with halo
 * exchanges between neighbours.  For the ADI step (Sec. 5.1) a rank holding rows [r0, r0 + rows)
 * of the n x n field runs, per step:
 *   1. exchange 2 halo rows of C^n and C^{n-1} with its neighbours (periodic: the last band's
 *      neighbour below is the first band; no-flux: the first band's rows above and the last
 *      band's rows below are its own rows mirrored, ghost row -1 = row 0, -2 = row 1);
 *   2. cs_ch_band_rhs: the right-hand side of its rows (and, optionally, its mass and energy sums);
 *   3. cs_ch_band_solve: the x line solves, one per row;
 *   4. a transpose among the ranks (all-to-all), so each rank holds a band of columns as rows;
 *   5. cs_ch_band_solve: the y line solves;
 *   6. the transpose back;
 *   7. cs_ch_band_update: C^{n+1} = 2 C^n - C^{n-1} + v on its rows.
 * Steps 1, 4 and 6 are the caller's communication (paper_1902_09931_gb300.distributed does them
 * with torch.distributed); the arithmetic is the full-grid step's own kernels, so the decomposed
 * step gives the values cs_ch_step gives.
 * Without transposes, when every band is a whole number of the y lines' chunks (the spike
 * method's partition, cs_ch_partition): steps 4-6 become
 *   4'. cs_ch_band_ycols_local: the chunk-local solves of the band's chunks of every column, and
 *       their end values (4 per column and chunk);
 *   5'. an all-gather of the end values of every band, in chunk order (4 * chunks * n values, the
 *       only data the ranks exchange for the y lines);
 *   6'. cs_ch_band_ycols_correct: the spike correction of the band's chunks, giving v.
 *
 * cs_ch_band_create: desc as for cs_ch_create (boundary CS_CH_PERIODIC or CS_CH_NOFLUX; the
 *   partition is the one cs_ch_create picks for the same description); rows = the band's row
 *   count, a multiple of 32 in [32, n].  The plan owns the line solver's tables and an FP64
 *   scratch of rows x n, plus 4 * chunks * rows values.
 * Padded fields: (rows + 4) x n values of the storage type, row-major; rows 0-1 hold the two rows
 *   above the band, rows 2 .. rows+1 the band, rows rows+2 .. rows+3 the two rows below.
 * cs_ch_band_rhs(d_prev, d_cur): padded C^{n-1}, C^n (halos filled) -> d_rhs (rows x n FP64; may be
 *   NULL when only sums are wanted); d_sums (device, 2 FP64, nullable): h^2 sum C and h^2 sum of
 *   the free-energy density over the band's rows (Eq. 1, forward differences), for an allreduce.
 * cs_ch_band_solve(d_in, d_out): (I + a D4) x = b along each of the rows rows of n values (FP64,
 *   row-major; periodic lines, or with no-flux the reflected fourth difference); d_out may equal
 *   d_in.
 * cs_ch_band_update(d_prev, d_cur, d_v, d_next): the band rows of the padded d_next get
 *   2 C^n - C^{n-1} + v (v: rows x n FP64), rounded to the storage type; its halo rows are not
 *   written.  The three padded fields must not overlap.
 * All are stream-ordered and asynchronous. */
int cs_ch_band_create(cs_plan_t* plan, const cs_ch_desc* desc, int64_t rows);
int cs_ch_band_rhs(cs_plan_t plan, const void* d_prev, const void* d_cur, double* d_rhs, double* d_sums,
                   void* cuda_stream);
int cs_ch_band_solve(cs_plan_t plan, const double* d_in, double* d_out, void* cuda_stream);
int cs_ch_band_update(cs_plan_t plan, const void* d_prev, const void* d_cur, const double* d_v, void* d_next,
                      void* cuda_stream);

/* The line partition of the ADI step (Sec. 5.1: the line solves, each line cut into *chunks chunks
 * of *chunk_len points for the partitioned solve) that cs_ch_create and cs_ch_band_create pick for
 * desc (the autotuner's recorded choice for it, else the default); either output may be NULL.
 * CS_EINVAL for an invalid description.  Host only. */
int cs_ch_partition(const cs_ch_desc* desc, int32_t* chunks, int32_t* chunk_len);

/* The y line solves of a band holding chunks chunk0 .. chunk0 + rows / chunk_len - 1 of every
 * column (rows a whole number of chunks; CS_EINVAL otherwise), in two phases:
 * cs_ch_band_ycols_local(d_in, d_ends): d_in the band's rows x n FP64 values of w (the x solves'
 *   result); solves each chunk of each column locally into the plan's scratch and writes the
 *   chunks' end values to d_ends (device, 4 * (rows / chunk_len) * n FP64, chunk-major).
 * cs_ch_band_ycols_correct(d_ends_all, d_v): d_ends_all the end values of all chunks of the line,
 *   in chunk order (every band's d_ends, gathered); writes v (rows x n FP64) for the band's rows,
 *   which cs_ch_band_update turns into C^{n+1}.  Uses the scratch phase 1 filled: no
 *   cs_ch_band_solve between the two.
 * Stream-ordered and asynchronous. */
int cs_ch_band_ycols_local(cs_plan_t plan, int64_t chunk0, const double* d_in, double* d_ends, void* cuda_stream);
int cs_ch_band_ycols_correct(cs_plan_t plan, int64_t chunk0, const double* d_ends_all, double* d_v,
                             void* cuda_stream);

/* Self-check of the line solver (no counterpart in the paper; host code only, no GPU needed):
 * builds the partitioned-solve tables cs_ch_create would build for lines of n points split into
 * `chunks` chunks with coefficient a = (2/3) D gamma dt / h^4 and the given boundary
 * (cs_ch_boundary), replays the two device phases on the host in the kernels' order of operations
 * for a fixed pseudo-random right-hand side b in [-1, 1), and writes the backward error
 * ||L x - b||_inf / ((1 + 16 a) ||x||_inf) of the result against the line operator L = I + a D4
 * itself.  CS_EINVAL for an invalid partition (n / chunks >= 16, a multiple of 8, chunks <= 64),
 * a < 0 or a non-finite a. */
int cs_ch_solver_check(int64_t n, int32_t chunks, double a, int32_t boundary, double* residual);

/* Allocation-free batched 1D sweep.  The paper has no counterpart: this entry point exists for
 * callers that cannot let a library allocate device memory -- code running under a fixed
 * device-memory budget or inside an arena owned by another runtime, latency-critical loops that
 * cannot afford an allocation or its implicit synchronisation, and plain C callers that only
 * hand over buffers they already own.  It computes exactly what cs_plan_create_1d_batch +
 * cs_compute compute (same arguments, same layout), without a plan and without calling
 * cudaMalloc / cudaFree or any allocating routine.
 *   Its scratch (the line-lookup table, one int32 per 64 packed elements) lives in a fixed
 *   file-scope device array created when the library is loaded; every GPU that loads the
 *   library holds it (4 MiB + 256 B) until the process exits.  total_len is limited to
 *   2^26 = 67,108,864 elements; larger requests return CS_EINVAL (use a plan instead).
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *   that device current.
 *   Every call shares the array and overwrites it: calls that overlap on the GPU (different
 *   streams, or host threads) race and must be serialised by the caller.
 *   The offsets are validated on the device first: every call synchronises the stream once,
 *   to read the result of that check back to the host; invalid offsets return CS_EINVAL and
 *   leave d_out untouched.  Because of that read-back no call can be captured into a CUDA
 *   graph: under stream capture the call returns CS_ECUDA and the capture is invalidated. */
int cs_batch1d_compute_noalloc(const cs_stencil_desc* desc, int64_t num_lines,
                               const int64_t* d_offsets, int64_t total_len, const void* d_in,
                               void* d_out, void* cuda_stream);

/* ---- diagnostics --------------------------------------------------------------------------- */

/* Description of the last error on the calling host thread ("" if none). */
const char* cs_last_error(void);

/* Number of kernels this library has launched in the process (graph replays count each
 * kernel node).  Used to report launch counts in benchmarks. */
int64_t cs_launch_count(void);

/* Library version, e.g. "custen_gb 0.1.0 sm_103a". */
const char* cs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CUSTEN_GB_H */

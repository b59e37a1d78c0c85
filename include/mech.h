/*
 * mech.h -- C ABI of libmech, a GB300 (sm_103a) implementation of the
 * per-time-step cell-mechanics update of an agent-based multicellular
 * simulation: the "update velocity" region that the paper analyses in
 * Sec. 5.4 (a loop over all cells that updates each cell's velocity from its
 * neighbouring cells, found through the mechanics voxel grid; Listing 4 and
 * the non-empty-voxel variant that follows it), plus the position update.
 *
 * One step (mech_step) does, for every cell i:
 *   1. Binning.  i_d = clamp(floor((x_d - lo_d) * (1/h)), 0, n_d - 1) on a uniform
 *      voxel grid of side h over the domain [lo, hi] (n_d = ceil((hi_d -
 *      lo_d) / h); the index is one IEEE subtraction and one multiplication
 *      by the once-rounded reciprocal 1/h, no contraction, in the precision
 *      of the positions); cells outside the domain are counted in the edge
 *      voxel;
 *      the cells are then permuted into voxel order by a counting sort
 *      (histogram, exclusive scan, scatter) whose order inside a voxel is
 *      ascending caller index.  This is the GPU form of the paper's lesson
 *      that cells should be stored and computed in the order of the 3-D mesh
 *      and that empty voxels should cost nothing (Sec. 5.4).
 *   2. Velocity.  Over every cell j != i in the 27 voxels around i's voxel,
 *      with d = |x_i - x_j| > 0 and S = R_i + R_j:
 *        c_r = sqrt(ccr_i ccr_j) (1 - d/S)^2          if d < S,   else 0
 *        c_a = sqrt(cca_i cca_j) (1 - d/(A S))^2      if d < A S, else 0
 *        v_i = sum_j (c_r - c_a) (x_i - x_j) / d.
 *   3. Two-step Adams-Bashforth: x_i += dt (1.5 v_i - 0.5 v_i,prev), then
 *      v_i,prev = v_i.  Before the first step v_prev = 0.
 * The paper names these regions but prints none of the formulas; the force
 * law and the integrator above are the problem this library solves.
 *
 * Optional velocity variants (mech_set_affinity, mech_set_walls): a per-type
 * adhesion affinity that scales c_a, and repulsive domain walls.
 *
 * Beyond the step: cells removed and added between steps (mech_remove_cells,
 * mech_add_cells, mech_add_cells_batch), and a substrate diffusion solver
 * with gradients for the microenvironment regions of Sec. 5.1-5.2
 * (mech_diffusion_*), both described with their calls below.
 *
 * Units: um and min.  All per-cell arrays are in the CALLER's cell order
 * (index 0..n-1, concatenated over replicates for a batch); positions and
 * velocities are interleaved xyz, 3*n doubles.  The library copies every
 * input array before returning; the caller owns every output buffer.  The
 * internal voxel order is never exposed.
 *
 * Every call returns MECH_OK (0) or a negative MECH_E_* code; the message of
 * the last failure on the calling thread is in mech_last_error().  Calls on
 * one handle are not thread-safe; distinct handles are independent.
 * Device work is queued on the handle's CUDA stream (mech_set_stream); the
 * read calls synchronise that stream.  Host pointers may be pageable or
 * pinned; pinned buffers copy faster.
 */
#ifndef MECH_H
#define MECH_H

#include <stdint.h>

#if defined(__GNUC__)
#define MECH_API __attribute__((visibility("default")))
#else
#define MECH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define MECH_OK 0
#define MECH_E_ARG (-1)              /* invalid argument (null pointer, bad size, bad mode) */
#define MECH_E_NONFINITE (-2)        /* NaN or Inf in an input array or parameter */
#define MECH_E_VOXEL_TOO_SMALL (-3)  /* voxel_size < 2 A max R: the 27-voxel stencil would miss pairs */
#define MECH_E_OOM (-4)              /* device allocation failed, or the grid does not fit */
#define MECH_E_CUDA (-5)             /* a CUDA runtime call failed */
#define MECH_E_TIMEOUT (-6)          /* a bounded device wait gave up */
#define MECH_E_DEVICE_FLAG (-7)      /* a kernel raised its error flag (non-finite state, bad index) */
#define MECH_E_STATE (-8)            /* call out of order (e.g. mech_step before mech_set_params) */

/* Precision modes (mech_set_precision). */
#define MECH_FP64 0           /* positions, velocities and pair arithmetic in FP64 */
#define MECH_MIXED_FP64POS 1  /* pair arithmetic and sums in FP32, positions and AB2 accumulation in FP64 */
#define MECH_MIXED_KAHAN 2    /* pair arithmetic in FP32, positions in FP32 with a Kahan compensation term */

typedef struct mech mech_t;

/* Message of the last failing call on this thread ("" if none). */
MECH_API const char* mech_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
MECH_API int mech_version(void);

/*
 * Create a handle for one population of n >= 0 cells on the current CUDA
 * device.  xyz: 3n doubles; R (radius, > 0), ccr, cca (>= 0): n doubles each;
 * type: n int32 cell types in [0, 16) (used only by the per-type adhesion
 * affinity, mech_set_affinity; NULL = all type 0).  The arrays are
 * copied.  Precision defaults to MECH_MIXED_FP64POS; parameters must be set
 * with mech_set_params before the first step.  The domain defaults to a cube
 * centred at the origin whose half side is 1.5 times the largest |coordinate|
 * (at least half a voxel).  *h is set to NULL on failure.
 */
MECH_API int mech_create(mech_t** h, int64_t n, const double* xyz, const double* R, const double* ccr,
                const double* cca, const int32_t* type);

/*
 * Create a handle for n_rep >= 1 independent replicates (counts[r] >= 0 cells
 * each) advanced together: every kernel launch covers all replicates, each on
 * its own voxel grid.  The per-cell arrays hold the replicates one after
 * another (replicate 0 first), sum(counts) cells in total.
 */
MECH_API int mech_create_batch(mech_t** h, int32_t n_rep, const int64_t* counts, const double* xyz,
                      const double* R, const double* ccr, const double* cca, const int32_t* type);

/*
 * A >= 1: adhesion range factor; voxel_size: mechanics voxel side (um), must
 * be >= 2 A max_i R_i (else MECH_E_VOXEL_TOO_SMALL); dt > 0: time step (min).
 * Applies to every replicate.  Resets nothing else.
 */
MECH_API int mech_set_params(mech_t* h, double A, double voxel_size, double dt);

/*
 * Domain of replicate rep (rep = -1: every replicate): lo[3] < hi[3].  The
 * grid has n_d = ceil((hi_d - lo_d) / voxel) voxels per axis; cells outside
 * it stay where they are and are binned into the edge voxel (there are no
 * walls).  Fails with MECH_E_OOM if the grids of all replicates exceed
 * 2^31 voxels or device memory.
 */
MECH_API int mech_set_domain(mech_t* h, int32_t rep, const double lo[3], const double hi[3]);

/* MECH_FP64, MECH_MIXED_FP64POS or MECH_MIXED_KAHAN.  Converts the current
 * state (positions and previous velocities) to the new representation. */
MECH_API int mech_set_precision(mech_t* h, int mode);

/*
 * Voxel side used internally for binning (the autotuner's knob).  0 restores
 * voxel_size.  Must be >= 2 A max R (1 + 1e-6).  The set of interacting pairs
 * does not depend on it; the FP32 summation order does.
 */
MECH_API int mech_set_internal_voxel(mech_t* h, double voxel);

/* Kernel shape: threads per block of the force kernel (32..256, multiple of
 * 32; 0 = default).  Autotuner knob; results do not depend on it. */
MECH_API int mech_set_launch(mech_t* h, int32_t force_block);

/*
 * Voxel tiles (autotuner knob): dense regions are processed one tile of
 * tile_x * tile_y * tile_z voxels at a time, with the tile's halo staged in
 * shared memory; a tile holding at least dense_min cells is dense.  Supported
 * tiles: 4x4x4 (the default, dense_min 12), 4x4x8 and 8x4x4; (0, 0, 0) sends
 * every cell through the thread-per-cell kernel.  The FP32 summation order does not
 * depend on this setting.
 */
MECH_API int mech_set_tiling(mech_t* h, int32_t tile_x, int32_t tile_y, int32_t tile_z, int32_t dense_min);

/*
 * Kernel for the cells of dense tiles (autotuner knob; no counterpart in the
 * paper, whose update-velocity loop is one thread per cell or per voxel of an
 * OpenMP team, Sec. 5.4):
 *   MECH_DENSE_BLOCK_PER_TILE (default): one thread per target cell, the
 *     tile's halo staged in shared memory by TMA bulk copies; interior tiles
 *     only (tiles touching a grid face go to the thread-per-cell kernel);
 *   MECH_DENSE_WARP_PER_VOXEL: 32 threads per voxel - the lanes hold the
 *     voxel's candidates and its target cells are taken in turn; works on any
 *     dense tile.
 * Both give velocities within FP32 rounding of each other (their summation
 * orders differ); each is bitwise reproducible run to run.
 */
#define MECH_DENSE_WARP_PER_VOXEL 0
#define MECH_DENSE_BLOCK_PER_TILE 1
MECH_API int mech_set_dense_kernel(mech_t* h, int32_t kernel);

/*
 * Per-type adhesion affinity (a velocity variant; the paper names PhysiCell,
 * Sec. 3.2, whose cell types adhere selectively, but states no law; the
 * statement is this library's): aff is an ntypes x ntypes row-major matrix,
 * symmetric, finite entries >= 0, ntypes in [1, 16] and above every cell's
 * type.  The adhesion coefficient of a pair becomes
 *   c_a = (aff[t_i][t_j] sqrt(cca_i cca_j)) (1 - d/(A S))^2.
 * ntypes = 0 or aff = NULL switches the affinity off (the base law; a matrix
 * of ones gives the same velocities).  The library copies the matrix.
 * Errors: MECH_E_ARG (size, sign, asymmetry, a cell type outside the table),
 * MECH_E_NONFINITE.
 */
MECH_API int mech_set_affinity(mech_t* h, int32_t ntypes, const double* aff);

/*
 * Domain walls (a velocity variant; statement as for the affinity): bit f of
 * face_mask enables face f of every replicate's domain box (mech_set_domain),
 * in the order -x, +x, -y, +y, -z, +z.  A cell whose centre lies at inward
 * distance d_w from an enabled face, d_w < R_i, is pushed along the inward
 * normal by c_wall t^2, t = 1 - d_w / R_i for d_w > 0 and t = 1 at or beyond
 * the face; the terms are added after the pair terms, face by face in the
 * order above.  face_mask = 0 switches the walls off.  c_wall in um/min,
 * finite and >= 0.  Errors: MECH_E_ARG, MECH_E_NONFINITE.
 */
MECH_API int mech_set_walls(mech_t* h, int32_t face_mask, double c_wall);

/* Stream (a cudaStream_t) for all device work of this handle; NULL = the
 * handle's own stream.  The caller keeps the stream alive. */
MECH_API int mech_set_stream(mech_t* h, void* stream);

/*
 * Use a CUDA graph holding `steps_per_graph` consecutive steps (an even
 * number >= 2; 0 disables graphs).  mech_step then replays the graph and
 * launches the remainder directly.  The graph is (re)captured on first use
 * after any change of parameters, domain, precision or launch shape; capture
 * happens on the handle's stream.
 */
MECH_API int mech_set_graph(mech_t* h, int32_t steps_per_graph);

/* Advance n_steps >= 0 steps.  Asynchronous on the handle's stream. */
MECH_API int mech_step(mech_t* h, int64_t n_steps);

/* Velocities v_n of the current positions (steps 1-2 only, no integration);
 * writes 3n doubles in caller order.  Synchronous. */
MECH_API int mech_compute_velocities(mech_t* h, double* out3n);

/*
 * Per-phase timing with CUDA events on the handle's stream: while enabled,
 * every directly launched step (graphs are bypassed) records events around
 * its phases.  mech_read_profile waits for the stream and returns the summed
 * device milliseconds of each phase since the previous read: phase_ms[0] scan
 * (histogram prefix sum), [1] scatter, [2] in-voxel ordering and FP32 record
 * build, [3] tile classification, [4] velocity + AB2 of the cells in dense
 * tiles, [5] velocity + AB2 of all other cells (all cells in MECH_FP64 mode),
 * and the number of steps recorded (at most 4096 between reads).
 */
MECH_API int mech_set_profiling(mech_t* h, int32_t enable);
MECH_API int mech_read_profile(mech_t* h, double* phase_ms, int64_t* steps);

/* Wait for the handle's stream; report a raised device error flag as
 * MECH_E_DEVICE_FLAG. */
MECH_API int mech_sync(mech_t* h);

/* Current positions (3n doubles, caller order).  In MECH_MIXED_KAHAN mode the
 * value is x_hi - c evaluated in FP64.  Synchronous. */
MECH_API int mech_read_positions(mech_t* h, double* out3n);

/* Velocities of the last step (v_n, computed from the positions at the start
 * of that step), 3n doubles in caller order; zeros before the first step. */
MECH_API int mech_read_velocities(mech_t* h, double* out3n);

/* Replace all positions (3n doubles, caller order); previous velocities are
 * kept.  Asynchronous: the host buffer must stay valid until the next
 * synchronising call on the handle. */
MECH_API int mech_write_positions(mech_t* h, const double* xyz3n);

/*
 * Exact state for checkpoint/resume: xyz (3n; in MECH_MIXED_KAHAN mode the
 * FP32 x_hi values), vprev (3n), comp (3n, the Kahan compensation c, zeros in
 * the other modes; may be NULL), step (may be NULL).  mech_load_state takes
 * the same arrays; a run resumed from a saved state is bitwise identical to
 * the uninterrupted run with the same precision, parameters and internal voxel.
 */
MECH_API int mech_read_state(mech_t* h, double* xyz, double* vprev, double* comp, int64_t* step);
MECH_API int mech_load_state(mech_t* h, const double* xyz, const double* vprev, const double* comp, int64_t step);

/*
 * Dynamic population (the cell count changes between steps, as cells divide
 * and die).  These calls are ordered after the work already enqueued on the
 * handle's stream and return when done; the next step bins the new
 * population (keys are recomputed from the positions), and the handle's step
 * count is unchanged.  Every replicate of a batch stays one contiguous range
 * of caller indices, in replicate order.
 *
 * mech_remove_cells: alive holds n bytes in caller order (all replicates);
 * the cells with alive[i] == 0 are removed.  The survivors keep their
 * relative order and are renumbered 0 .. n'-1 (caller index i becomes the
 * number of survivors before it) with their whole state: position (and Kahan
 * compensation), previous velocity, radius and coefficients.  The device work
 * is two prefix sums and, for a single population, the survivors moved into
 * the dead cells' slots (a batch: an order-preserving compaction), plus a
 * compaction of the caller-order parameters; nothing changes when every cell
 * is alive.
 *
 * mech_add_cells (single population): appends m cells with caller indices
 * n .. n+m-1, positions xyz (3m doubles), radii, coefficients and types as
 * in mech_create; their previous velocity is zero (their AB2 starts as at
 * creation).  mech_add_cells_batch: counts[r] new cells for replicate r
 * (n_rep counts; the arrays hold them in replicate order); replicate r's new
 * cells follow its existing ones and the later replicates' caller indices
 * move up by the cells added before them.  When the total exceeds the device
 * capacity, every per-cell buffer grows to max(n + m, 1.5 n) cells (one copy
 * of the state).  A radius for which the handle's voxel (or internal voxel)
 * is too small fails with MECH_E_VOXEL_TOO_SMALL and non-finite or invalid
 * cells with MECH_E_NONFINITE / MECH_E_ARG, before anything changes.
 *
 * mech_add_cells on a batch handle fails with MECH_E_ARG; all three fail
 * with MECH_E_STATE on a handle a device error left inconsistent.
 */
MECH_API int mech_remove_cells(mech_t* h, const uint8_t* alive);
MECH_API int mech_add_cells(mech_t* h, int64_t m, const double* xyz, const double* R, const double* ccr,
                            const double* cca, const int32_t* type);
MECH_API int mech_add_cells_batch(mech_t* h, const int64_t* counts, const double* xyz, const double* R,
                                  const double* ccr, const double* cca, const int32_t* type);

/*
 * Binning of the current positions, for inspection (steps 1 of the update,
 * without advancing): key (n, caller order), count (V), start (V + 1) and
 * order (n: caller index of the cell at each sorted position), V = total
 * voxels of all replicates (mech_info).  Any output may be NULL.  Synchronous.
 */
MECH_API int mech_debug_bins(mech_t* h, uint32_t* key, uint32_t* count, uint32_t* start, int64_t* order);

/*
 * Neighbour statistics of the current positions (Sec. 5.4: each cell's
 * velocity is gathered from the cells of its 27 neighbouring mechanics
 * voxels; a neighbour contributes when 0 < d < A (R_i + R_j)):
 *   candidates: ordered pairs (i, j != i) with j in one of the 27 voxels
 *               around i's voxel on the internal grid the step uses
 *               (mech_set_internal_voxel), i.e. the neighbour tests one step
 *               performs;
 *   pairs:      unordered interacting pairs {i, j}, 0 < d < A (R_i + R_j),
 *               decided in FP64 from the current positions (x_hi - c in
 *               MECH_MIXED_KAHAN mode) with the same operations as the
 *               definition (no contraction, IEEE square root).
 * Either output may be NULL.  Synchronous; does not advance the state.
 */
MECH_API int mech_pair_stats(mech_t* h, int64_t* candidates, int64_t* pairs);

/*
 * Binning without allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they call it --
 * code whose device memory is already entirely reserved by another allocator
 * (a framework's caching pool that owns the GPU), or a latency-critical loop
 * that cannot afford cudaMalloc's implicit device synchronisation.  It runs
 * the binning of step 1 for one grid, with the voxel index taken in FP64 as in
 * MECH_FP64 mode and the cells of a voxel in ascending input index:
 *   xyz    device, 3n doubles (interleaved): positions;
 *   lo, voxel, dims  host: grid lower corner, voxel side, voxels per axis;
 *   key    device, n u32: voxel key of each cell, input order;
 *   start  device, V + 1 u32, V = dims[0] dims[1] dims[2]: exclusive prefix
 *          sum of the voxel counts (cells of voxel v are start[v]..start[v+1]-1);
 *   order  device, n u32: input index of the cell at each sorted position;
 *   stream a cudaStream_t (NULL: the legacy default stream).
 * Limits: n <= 262,144 and V <= 524,288; larger sizes return MECH_E_ARG and
 * launch nothing.  The working memory is a fixed array of about 6.1 MiB in the
 * library's device data, held by every GPU that loads the library until the
 * process exits; the call itself allocates and frees nothing.  The first call
 * on each device looks up the device address of that array
 * (cudaGetSymbolAddress) with the device current; under lazy module loading
 * (the CUDA default) that first use is also when the driver loads the
 * library's device code and this array, which takes device memory.  So make
 * the first call on each device early -- a call with n = 0 (xyz, key and
 * order may then be NULL; start gets V + 1 zeros) does the set-up and nothing
 * else of note -- before the caller's allocator reserves the device's memory
 * and before any stream capture.
 * Cost: the cells of a voxel are put in input order by ranking each one
 * against the others of its voxel, so a voxel holding k cells costs k
 * comparisons per cell; the lanes of a warp read the same entries together,
 * so the whole call takes about sum over voxels of k^2 / 8 warp instructions
 * on top of linear work: at tissue densities (under ~10 cells per voxel)
 * linear, and at the limit of all 262,144 cells in one voxel about 8.6e9 warp
 * instructions, tens of milliseconds.  Asynchronous: the outputs are ready when the
 * stream reaches this work.  Every call uses the same array and leaves its
 * contents behind, so calls whose work overlaps on the GPU (other streams,
 * other host threads) race and corrupt each other's results: serialise them.
 */
MECH_API int mech_bin_noalloc(int64_t n, const double* xyz, const double lo[3], double voxel,
                              const int32_t dims[3], uint32_t* key, uint32_t* start, uint32_t* order,
                              void* stream);

/*
 * Fault injection for tests of the failure paths (host-armed; nothing here
 * makes a GPU fault, trap or hang).  MECH_FAULT_TILE_WAIT: the tile kernel's
 * copy barrier expects 16 bytes more than are copied, so its wait can never
 * complete; the wait gives up after 1 ms, the kernel sets its error flag and
 * returns, and the next synchronising call reports MECH_E_TIMEOUT.
 * MECH_FAULT_ALLOC (h may be NULL): the next device allocation by any handle
 * fails with MECH_E_OOM.  MECH_FAULT_NONE disarms both.  After any device
 * error the handle refuses mech_step and mech_write_positions (MECH_E_STATE)
 * until the whole state is reloaded with mech_load_state.
 */
#define MECH_FAULT_NONE 0
#define MECH_FAULT_TILE_WAIT 1
#define MECH_FAULT_ALLOC 2
MECH_API int mech_debug_inject(mech_t* h, int32_t fault);

typedef struct {
    int64_t n_cells;
    int32_t n_rep;
    int32_t mode;
    int64_t n_voxels;     /* total voxels of all replicate grids */
    int32_t dims[3];      /* grid of replicate 0 */
    double voxel;         /* internal voxel side */
    int64_t step;         /* steps taken */
    int32_t launches_per_step; /* kernel launches of one steady-state step */
    int32_t graph_steps;
    int64_t device_bytes; /* device memory held by the handle */
} mech_info_t;

MECH_API int mech_info(mech_t* h, mech_info_t* out);

/* Grid of replicate rep: lo[3], dims[3], voxel offset in the global index. */
MECH_API int mech_grid(mech_t* h, int32_t rep, double* lo3, int32_t* dims3, int64_t* voxel_base);

/* Release every device and host resource of the handle (NULL is a no-op). */
MECH_API int mech_destroy(mech_t* h);

/*
 * Substrate diffusion (the microenvironment solver and gradient regions of
 * Sec. 5.1-5.2, run on a 75^3-voxel domain in the paper).  S densities on
 * nx x ny x nz cubic voxels of side dx, array [s][z][y][x] (FP64), diffusion
 * coefficients D[s] and decay rates lambda[s] (both >= 0), no flux through
 * the faces.  mech_diffusion_step advances n_steps steps of length dt, each
 * three one-dimensional backward-Euler solves (x, then y, then z) with the
 * decay split equally among them, solved by the Thomas algorithm in FP64
 * with IEEE operations in a fixed order (the results are reproducible bit for
 * bit); asynchronous on the handle's stream.  mech_diffusion_gradient
 * computes the gradients (central differences inside, one-sided at the
 * faces; array [s][axis][z][y][x]) and copies them out when grad is not
 * NULL; synchronous.  Densities start at zero; write/read copy all S fields
 * (synchronous).
 */
typedef struct mech_diffusion mech_diffusion_t;

MECH_API int mech_diffusion_create(mech_diffusion_t** out, int64_t nx, int64_t ny, int64_t nz, int32_t n_substrates,
                                   double dx, const double* D, const double* lambda);
MECH_API int mech_diffusion_destroy(mech_diffusion_t* h);
MECH_API int mech_diffusion_set_stream(mech_diffusion_t* h, void* stream);
MECH_API int mech_diffusion_write(mech_diffusion_t* h, const double* rho);
MECH_API int mech_diffusion_read(mech_diffusion_t* h, double* rho);
MECH_API int mech_diffusion_step(mech_diffusion_t* h, double dt, int64_t n_steps);
MECH_API int mech_diffusion_gradient(mech_diffusion_t* h, double* grad);
MECH_API int mech_diffusion_sync(mech_diffusion_t* h);

#ifdef __cplusplus
}
#endif

#endif /* MECH_H */

/*
 * lbm.h -- C ABI of the GB300 pore-scale lattice Boltzmann library (liblbm.so).
 *
 * Method: Fattahi, Waluga, Wohlmuth & Ruede, "Large scale lattice Boltzmann
 * simulation for the coupling of free and porous media flow".  A D3Q19
 * two-relaxation-time scheme (Sec. 2.1, Eqs. (LBM), (TRT), (TRT2),
 * (equilibrium), (Macro), (collision), (streaming)) driven by a body force,
 * with central-linear-interpolation bounce-back on every wall link
 * (Sec. 2.2, Eq. (CLI); q = 1/2 is simple bounce-back, Eq. (noslip); links
 * without a second fluid node use bounce-back, and LBM_FLAG_CLI_SAFEGUARDS
 * extends that to links across a two-cell gap or with q < 0.1), on
 * voxelised sphere packings (Sec. 3.1), with plane averages of the stream-wise
 * velocity (Sec. 3.1) and the Darcy permeability (Eq. (Darcy)).
 *
 * Conventions shared by every call:
 *  - Return value: LBM_OK (0) on success, a negative LBM_E* code on failure.
 *    No C++ exception crosses the ABI.  lbm_status_string() names a code.
 *  - Geometry and solver handles are owned by the library and freed by their
 *    *_destroy call.  All device memory is owned by the caller: the solver
 *    lives in one caller-allocated device workspace of lbm_workspace_size()
 *    bytes (256-byte aligned) that must outlive the solver.
 *  - Streams: lbm_init() binds the solver to a CUDA stream (a cudaStream_t
 *    passed as void*, NULL = legacy default stream).  Device-side calls are
 *    asynchronous on that stream; calls that return host values synchronise
 *    that stream only.
 *  - Layouts: dense fields are [nz][ny][nx] with x fastest (cell index
 *    c = x + nx (y + ny z)); vectors are component-major [3][nz][ny][nx].
 *    Fluid cells are numbered 0..n_fluid-1 in increasing cell index.
 *  - D3Q19 ordering: k = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (1,1,0),
 *    (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1),
 *    (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1); the opposite of k >= 1 is k+1
 *    for odd k and k-1 for even k.
 *  - Lattice units throughout (dx = dt = 1, rho0 = 1).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LBM_OK 0
#define LBM_EINVAL (-1)       /* bad argument (NULL handle, size out of range, ...) */
#define LBM_ENOMEM (-2)       /* host allocation failed */
#define LBM_ECUDA (-3)        /* a CUDA runtime call failed */
#define LBM_EPACKING (-4)     /* target porosity unreachable without overlap */
#define LBM_ENAN (-5)         /* a NaN or Inf appeared in the velocity field */
#define LBM_ENOTCONVERGED (-6)/* lbm_run_until reached max_steps */
#define LBM_ETIMEOUT (-7)     /* a bounded device-side wait gave up; the solver
                                 then refuses lbm_step/lbm_run_until (also
                                 LBM_ETIMEOUT) until lbm_reset */
#define LBM_ESIZE (-8)        /* workspace too small or misaligned */

/* ---- storage precision of the populations ---- */
#define LBM_F32 0
#define LBM_F16 1
#define LBM_BF16 2

typedef struct lbm_geometry lbm_geometry;
typedef struct lbm_solver lbm_solver;

/* Box.  x and y are always periodic.  With periodic_z == 0 the cell layers
 * z = 0 and z = nz-1 are solid no-slip walls (Sec. 3.1: walls at top and
 * bottom, periodic stream- and span-wise); their surfaces lie at the link
 * fractions q_lo and q_hi from the adjacent fluid nodes (1/2 = half-way,
 * Eq. (noslip)).  Limits: 1 <= nx, ny, nz and nx*ny*nz < 2^31. */
typedef struct {
    int32_t nx, ny, nz;
    int32_t periodic_z;
    double q_lo, q_hi;
} lbm_box;

/* Seeded sphere placement standing in for the settled rigid-body packing of
 * Sec. 3.1 (the paper's particle code is not available).  Candidates draw, in
 * order, x in [0,nx), y in [0,ny), z in [layer_z0, layer_z1) and r in
 * [r_min, r_max) from SplitMix64 (Steele, Lea & Flood 2014) seeded with
 * `seed`, each value u = (next >> 11) 2^-53 scaled and rounded down to the
 * 2^-10 grid.  With allow_overlap == 0 a candidate closer than the radius sum
 * (minimum image) to an earlier sphere is rejected, and max_rejects
 * consecutive rejections give LBM_EPACKING.  Spheres are added until the voxel
 * porosity of the cells with ceil(layer_z0) <= z < ceil(layer_z1) (wall layers
 * excluded) is <= porosity; more than max_spheres gives LBM_EINVAL.
 * Requires 2 r_max < nx, ny (and nz when periodic). */
typedef struct {
    lbm_box box;
    double layer_z0, layer_z1;
    double r_min, r_max;
    double porosity;
    int32_t allow_overlap;
    uint64_t seed;
    int64_t max_spheres;
    int64_t max_rejects;
} lbm_sphere_params;

/* Variant of the odd (gather/scatter) step; both address the same slots and
 * give the same bits.  LBM_FLAG_NEIGHBOUR_TABLE reads the 18 neighbour indices of a cell
 * from the stored table (72 bytes per cell and odd step);
 * LBM_FLAG_ROW_NEIGHBOURS computes them from per-row fluid bitmasks (about
 * 4 bytes per cell, but two dependent loads before the gathers).  Neither:
 * the table, which measured faster for every storage type, with computed
 * indices in tiles of 256 cells whose planes and neighbour planes are all
 * fluid.  The table is also used whenever ny*nz does not fit beside x in
 * 32 bits. */
#define LBM_FLAG_NEIGHBOUR_TABLE 1
#define LBM_FLAG_ROW_NEIGHBOURS 2
/* Neighbour indices outside the computed tiles from the row bitmasks of the
 * tile's rows and their neighbour rows, which each block stages in shared
 * memory once per tile of 256 cells (about 4 bytes per cell and odd step,
 * the cell's packed position, instead of the table's 72); cells in the
 * first or last row of a periodic span, tiles across boxes and tiles whose
 * rows do not fit the staging buffer use the table.  Needs nx, ny <= 2048
 * and nz <= 1024 (else the table is used). */
#define LBM_FLAG_STAGED_NEIGHBOURS 256
/* Neighbour indices outside the computed tiles: the table's eight entries
 * without an x component, and the ten with one derived from them (fluid
 * cells are numbered along x-rows, so the fluid neighbour at x +- 1 of a
 * fluid cell j in the same row is j +- 1), reading the table only where that
 * cell is solid or the row wraps around: 36 bytes per cell and odd step plus
 * those reads, instead of 72. */
#define LBM_FLAG_DERIVED_NEIGHBOURS 2048
/* Scheduling switches.  By default lbm_step times a few grid sizes for each
 * step kernel during its first launches on solvers of more than ~4 waves of
 * blocks (synchronising the stream while it does so) and then replays the
 * steps in chunks as a CUDA graph.  These flags turn either off. */
#define LBM_FLAG_NO_GRAPH 4
#define LBM_FLAG_NO_AUTOTUNE 8
/* The even step always on its staged kernel (populations fetched into shared
 * memory by TMA bulk copies), which the autotuner otherwise tries as one of its
 * candidates.  Same arithmetic, same results. */
#define LBM_FLAG_STAGED_EVEN 64
/* Simple bounce-back (Eq. (noslip): every wall surface half-way along its
 * link, q = 1/2 forced) on every wall link instead of Eq. (CLI).  The link
 * fractions q are still computed and exported; every link reports the
 * bounce-back fallback. */
#define LBM_FLAG_SIMPLE_BOUNCE_BACK 32
/* Corner safeguards of Eq. (CLI).  By default (the paper's scheme) a wall
 * link uses Eq. (CLI) whenever its second fluid node x_f2 = x_f1 - e_k exists
 * and simple bounce-back only where x_f2 is solid.  With this flag two more
 * kinds of link take simple bounce-back: links whose x_f1 - 2 e_k is solid
 * (a two-cell gap, where the interpolations of the two walls feed each other)
 * and links with q < 0.1 (a = (1-2q)/(1+2q) > 2/3).  In sharp corners of
 * overlapping sphere packings (nodes with 10-14 of their 18 links cut) the
 * paper's update was observed to grow without bound; the safeguards keep it
 * bounded at the price of a half-way wall on those links. */
#define LBM_FLAG_CLI_SAFEGUARDS 128
/* Reference equilibria in translation-invariant planes (see lbm_recenter):
 * fully fluid planes whose neighbour planes are fully fluid store each
 * population relative to the equilibrium of the plane's mean velocity, which
 * lbm_recenter refreshes.  Storage rounding then acts on the small
 * non-equilibrium part only.  In FP16/BF16 storage, where that rounding
 * dominates, it cuts the steady-channel velocity error by two orders of
 * magnitude (measured: FP16 11% -> 0.03%, BF16 59% -> 0.4% of u_max on a
 * 16x16x34 channel) and is on by default; LBM_FLAG_NO_PLANE_REFERENCES turns
 * it off.  In FP32 storage the collision's own roundings dominate, so it is
 * off unless LBM_FLAG_PLANE_REFERENCES asks for it.  It costs the step
 * kernels one reference load and one addition per population in those
 * planes (measured 3% of the FP32 and 7% of the FP16 step on the
 * 256x256x512 channels). */
#define LBM_FLAG_PLANE_REFERENCES 512
#define LBM_FLAG_NO_PLANE_REFERENCES 1024

/* Flow parameters.  tau = 1/omega+ with 1/omega+ = 3 nu + 1/2 (Sec. 2.1);
 * lambda is the magic parameter (1/omega+ - 1/2)(1/omega- - 1/2), which fixes
 * omega- (Sec. 2.1; 3/16 puts bounce-back walls exactly half-way).  g is the
 * body force per unit mass (the source F_k = 3 w_k e_k.g of Eq. (collision)).
 * storage is LBM_F32, LBM_F16 or LBM_BF16; flags is 0 or an OR of the
 * LBM_FLAG_* values above (at most one neighbour variant). */
typedef struct {
    double tau;
    double lambda;
    double g[3];
    int32_t storage;
    int32_t flags;
} lbm_params;

typedef struct {
    int64_t n_cells;   /* nx*ny*nz */
    int64_t n_fluid;   /* fluid cells */
    int64_t n_links;   /* wall links (fluid cell, k) with a solid neighbour */
    int64_t n_spheres;
    double porosity;   /* voxel porosity of the placement layer (placement) or of the box */
} lbm_geometry_info;

/* ------------------------------------------------------------------------- */
/* Geometry (host side; the library owns the handle).                        */
/* ------------------------------------------------------------------------- */

/* Place spheres (see lbm_sphere_params) and voxelise them: a cell (integer
 * centre) is solid if it is a wall layer or lies within distance r of any
 * periodic image of a sphere.  *out receives a new handle.
 * Errors: LBM_EINVAL, LBM_EPACKING, LBM_ENOMEM. */
int lbm_geometry_from_spheres(const lbm_sphere_params *params, lbm_geometry **out);

/* Same from an explicit sphere list xyzr[n][4] = (x, y, z, r), copied.
 * Centres may lie outside the box (e.g. below the bottom wall, Sec. 3.1).
 * Errors: LBM_EINVAL (r <= 0, 2r >= a periodic extent), LBM_ENOMEM. */
int lbm_geometry_from_list(const lbm_box *box, const double *xyzr, int64_t n, lbm_geometry **out);

/* Counts of a geometry. */
int lbm_geometry_info_get(const lbm_geometry *geom, lbm_geometry_info *out);

/* Copy the sphere list into host xyzr[cap][4]; *n receives the count.
 * LBM_ESIZE if cap is too small. */
int lbm_geometry_spheres(const lbm_geometry *geom, double *xyzr, int64_t cap, int64_t *n);

/* Copy the solid mask (1 = solid) into host mask[nz][ny][nx]. */
int lbm_geometry_mask(const lbm_geometry *geom, uint8_t *mask);

void lbm_geometry_destroy(lbm_geometry *geom);

/* ------------------------------------------------------------------------- */
/* Solver (device side).                                                      */
/* ------------------------------------------------------------------------- */

/* Bytes of device workspace lbm_init needs for this geometry and params. */
int lbm_workspace_size(const lbm_geometry *geom, const lbm_params *params, size_t *bytes);

/* Build the device fluid list, neighbour table and wall-link list (with q) in
 * the caller's workspace, then initialise the populations to the equilibrium
 * f_k^eq(rho = 1, u0) of Eq. (equilibrium).  dev_u0 is a device velocity
 * field [3][nz][ny][nx] (float) or NULL for rest.  stream is a cudaStream_t
 * (NULL = default stream); the call returns after the set-up has completed on
 * it.  The workspace must be 256-byte aligned and at least
 * lbm_workspace_size() bytes (else LBM_ESIZE).  The geometry may be destroyed
 * after this call.  Errors: LBM_EINVAL, LBM_ESIZE, LBM_ECUDA, LBM_ENOMEM. */
int lbm_init(const lbm_geometry *geom, const lbm_params *params, void *dev_workspace, size_t bytes,
             const float *dev_u0, void *stream, lbm_solver **out);

/* ------------------------------------------------------------------------- */
/* Batches: several independent boxes (e.g. periodic REV cubes of uneven     */
/* size, Sec. 3: the REV scale) advanced together, one kernel launch per     */
/* step for all of them.  A batch solver answers every call above; its      */
/* fields are the parts' fields concatenated in part order (cells, fluid     */
/* cells and z planes), lbm_plane_average returns the parts' planes one      */
/* after the other, lbm_profile_residual returns the largest part residual,  */
/* lbm_recenter shifts each part by its own mean density, and                */
/* lbm_permeability is refused (use lbm_batch_permeability).  The row-bitmask */
/* neighbour variant is not available for batches.                          */
/* ------------------------------------------------------------------------- */
int lbm_batch_workspace_size(const lbm_geometry *const *geoms, int32_t n, const lbm_params *params,
                             size_t *bytes);
int lbm_batch_init(const lbm_geometry *const *geoms, int32_t n, const lbm_params *params, void *dev_workspace,
                   size_t bytes, const float *dev_u0, void *stream, lbm_solver **out);
int lbm_batch_parts(const lbm_solver *solver, int32_t *n_parts);
/* Counts of part `part` and the offsets of its first fluid cell, cell and z
 * plane in the concatenated arrays (any output may be NULL). */
int lbm_batch_part_info(const lbm_solver *solver, int32_t part, lbm_geometry_info *info, int64_t *fluid_offset,
                        int64_t *cell_offset, int64_t *plane_offset);
/* Permeability of every part over its whole box (Eq. (Darcy), as
 * lbm_permeability with z_lo = z_hi = -1): k_out[n_parts].  Synchronises. */
int lbm_batch_permeability(lbm_solver *solver, double *k_out);
/* Profile residual of every part: res_out[n_parts] (+inf on a part's first
 * call).  Synchronises. */
int lbm_batch_profile_residual(lbm_solver *solver, double *res_out);

/* Launch schedule in use: grid sizes of the even and odd step kernels (the
 * kernels loop over tiles of 256 fluid cells, so a grid smaller than the tile
 * count makes them persistent; grid_even = -1: the even step's staged kernel,
 * which fetches each tile's populations into shared memory with TMA bulk
 * copies, on one wave of resident blocks), whether the autotuner has
 * finished, and the steps per CUDA-graph replay (0: graphs off). */
int lbm_schedule(const lbm_solver *solver, int32_t *grid_even, int32_t *grid_odd, int32_t *tuned,
                 int32_t *graph_steps);

/* Re-initialise the populations of an existing solver (step count back to 0)
 * from dev_u0 (or rest when NULL); clears the stale state that a timed-out
 * step leaves (LBM_ETIMEOUT). */
int lbm_reset(lbm_solver *solver, const float *dev_u0);

/* Advance n >= 0 time steps (collision, Eq. (collision), then streaming,
 * Eq. (streaming), with Eq. (CLI) on every wall link), asynchronously on the
 * solver's stream. */
int lbm_step(lbm_solver *solver, int64_t n);

/* Moments of the current state (Eq. (Macro)): rho = sum_k f_k and the velocity
 * u = j + g/2 (j = sum_k e_k f_k, rho0 = 1; g/2 makes u the mean of the pre-
 * and post-collision momentum).  Dense device outputs dev_rho[nz][ny][nx] and
 * dev_u[3][nz][ny][nx] (float; either may be NULL); solid cells get 0.
 * Asynchronous on the solver's stream. */
int lbm_moments(lbm_solver *solver, float *dev_rho, float *dev_u);

/* Plane averages of the stream-wise velocity (Sec. 3.1), summed in FP64 on the
 * device: host_out[nz][3] = (sum_fluid u_x / (nx ny), sum_fluid u_x / n_fluid(z)
 * or 0 for an all-solid plane, n_fluid(z) / (nx ny)).  Synchronises the
 * stream. */
int lbm_plane_average(lbm_solver *solver, double *host_out);

/* Darcy permeability along x (Eq. (Darcy) with mu = rho0 nu, no mean pressure
 * gradient and the body force g_x): K = nu <u_x> / g_x with <u_x> the
 * superficial mean over the planes z_lo..z_hi (both -1: the whole box),
 * reduced in FP64 on the device.  Synchronises the stream.  LBM_EINVAL if
 * g_x == 0 or the window is out of range. */
int lbm_permeability(lbm_solver *solver, int32_t z_lo, int32_t z_hi, double *k_out);

/* Convergence residual ||u - u_prev||_2 / ||u||_2 over all fluid cells and
 * components (FP64 sums on the device), where u_prev is the velocity at the
 * previous call; the first call after lbm_init/lbm_reset returns +inf.
 * Synchronises the stream.  LBM_ENAN if the field holds a NaN or Inf. */
int lbm_residual(lbm_solver *solver, double *res_out);

/* Convergence residual of the plane-averaged stream-wise velocity (the
 * quantity Sec. 3.1 reports at steady state): ||P - P_prev||_2 / ||P||_2 over
 * the nz superficial plane averages P(z) of lbm_plane_average, against the
 * profile at the previous call (+inf on the first call after
 * lbm_init/lbm_reset).  Unlike the field residual it is not limited by the
 * slow drift of the local velocity that the mass imbalance of Eq. (CLI)
 * causes, nor by storage round-off.  Synchronises the stream.  LBM_ENAN on a
 * non-finite profile. */
int lbm_profile_residual(lbm_solver *solver, double *res_out);

/* Mean density deviation <rho - 1> over the fluid cells (FP64 sum on the
 * device).  The CLI rule (Eq. (CLI)) does not conserve mass exactly, so in a
 * steady flow this drifts linearly in time.  Synchronises the stream. */
int lbm_mass(lbm_solver *solver, double *mean_drho);

/* Remove the mean density deviation: the next lbm_step subtracts
 * w_k <rho - 1> from every population before its collision.  The scheme is
 * invariant under such a uniform shift (the TRT split, the source term and
 * Eq. (CLI), a w - a w + w = w, all commute with it), so velocities are
 * unchanged in exact arithmetic; it keeps the stored populations small so
 * that reduced-precision storage keeps its resolution in long runs.
 * With plane references (the FP16/BF16 default, LBM_FLAG_PLANE_REFERENCES
 * for FP32) it also refreshes the reference populations
 * of the solver's translation-invariant planes (fully fluid planes whose
 * neighbour planes are fully fluid too, e.g. the free channel above a porous
 * layer): there every slot stores its population minus the equilibrium
 * f^eq(1, u_z) of the plane's mean velocity, so that storage rounding acts on
 * the small non-equilibrium part only (rounding that is the same at every
 * cell of such a plane would otherwise act like a spurious body force).  The
 * next step switches to the new references; the stored values change, the
 * populations they represent do not.  *shift_out (may be NULL) receives the
 * scheduled shift.  Synchronises the stream. */
int lbm_recenter(lbm_solver *solver, double *shift_out);

#define LBM_CONVERGE_FIELD 0    /* lbm_residual */
#define LBM_CONVERGE_PROFILE 1  /* lbm_profile_residual */

/* Step in chunks of `interval` until the residual selected by `criterion`
 * (LBM_CONVERGE_FIELD or LBM_CONVERGE_PROFILE) is below tol, taking at least
 * one chunk; the density is re-centred (lbm_recenter) after every chunk.  *steps_done and *res_out receive the steps taken and the last
 * residual.  LBM_ENOTCONVERGED after max_steps, LBM_ENAN on divergence. */
int lbm_run_until(lbm_solver *solver, double tol, int64_t interval, int64_t max_steps, int32_t criterion,
                  int64_t *steps_done, double *res_out);

/* Checkpoint and resume (the paper has no counterpart; long runs to steady
 * state at 10^5-10^6 steps need it).  A checkpoint is a host byte buffer of
 * lbm_checkpoint_size() bytes holding the stored populations at the current
 * parity, the step count, the pending density shift, the reference
 * populations and the residual histories; not the lists, which follow from
 * the geometry.  lbm_save copies the state into host_buf (LBM_ESIZE if bytes
 * is too small; LBM_ETIMEOUT for a stale solver).  lbm_load restores it into
 * a solver created from the same geometry and the same tau, lambda, g,
 * storage and wall rule (else LBM_EINVAL); the steps after it give the same
 * bits as the uninterrupted run would.  Both synchronise the stream; the
 * buffer is caller-owned and may be written to a file as it is (host byte
 * order). */
int lbm_checkpoint_size(const lbm_solver *solver, size_t *bytes);
int lbm_save(lbm_solver *solver, void *host_buf, size_t bytes);
int lbm_load(lbm_solver *solver, const void *host_buf, size_t bytes);

/* Number of planes (over all parts) whose slots store populations relative
 * to the plane's reference equilibrium (LBM_FLAG_PLANE_REFERENCES, see
 * lbm_recenter): fully fluid planes whose neighbour planes are fully fluid
 * and lie in tiles of 256 cells that hold only such planes' cells; 0 when
 * plane references are off. */
int lbm_reference_planes(const lbm_solver *solver, int32_t *n_planes);

/* Steps taken since lbm_init/lbm_reset. */
int lbm_steps_done(const lbm_solver *solver, int64_t *steps);

/* Counts of the solver's device lists. */
int lbm_solver_info(const lbm_solver *solver, lbm_geometry_info *out);

/* Copy the device lists to host buffers (any may be NULL):
 * fluid_cell[n_fluid] cell index of each fluid cell; nbr[18][n_fluid] fluid
 * index of the neighbour along e_k (k = 1..18) or -1 when solid;
 * link_cell/link_k/link_q/link_fallback[n_links]: one record per wall link in
 * (cell, k) order with the link fraction q of Eq. (CLI) and 1 when the link
 * uses simple bounce-back (a = 0) instead: when its second fluid node
 * x_f2 = x_f1 - e_k is solid, and with LBM_FLAG_CLI_SAFEGUARDS also when
 * x_f1 - 2 e_k is solid (a two-cell gap) or when q < 0.1 (the wall within a
 * tenth of a link of the node); every link with LBM_FLAG_SIMPLE_BOUNCE_BACK.
 * Synchronises the stream. */
int lbm_export_lists(lbm_solver *solver, int32_t *fluid_cell, int32_t *nbr, int32_t *link_cell,
                     int8_t *link_k, double *link_q, uint8_t *link_fallback);

/* Self-test of failure detection: one warp on the solver's stream waits, with
 * the bounded mbarrier wait of the staged step kernels, on a barrier phase
 * that nothing completes; after max_polls polls (>= 1) it gives up and sets
 * the solver's status word as a step kernel would.  Synchronises and returns
 * what the synchronising calls return after such an event: LBM_ETIMEOUT,
 * with the word cleared.  The solver then treats its state as stale, as after
 * a real timeout (a block that gives up leaves its tile half-updated):
 * lbm_step and lbm_run_until return LBM_ETIMEOUT until lbm_reset, while the
 * read-only calls keep working.  Touches no populations itself. */
int lbm_wait_selftest(lbm_solver *solver, int32_t max_polls);

/* Shifted populations h_k = f_k - w_k of the current state (the streamed
 * populations of Eq. (streaming) at the current time) into the device buffer
 * dev_out[19][n_fluid] (float; may be NULL when n_fluid is 0).  Asynchronous. */
int lbm_populations(lbm_solver *solver, float *dev_out);

/* Plane averages without any device allocation (the paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory -- an application whose own pool allocator owns all device memory, or
 * a monitoring loop that must not stall, since cudaMalloc/cudaFree synchronise
 * the device).  Same result as lbm_plane_average, computed from a dense
 * velocity x-component dev_ux[nz][ny][nx] (float, e.g. from lbm_moments) and
 * the dense solid mask dev_solid[nz][ny][nx] (uint8, 1 = solid) that the
 * caller already holds on the current device; host_out[nz][3] as in
 * lbm_plane_average.  The per-plane scratch is a fixed array of
 * LBM_STATIC_MAX_PLANES planes compiled into the library and kept on every GPU
 * that loads it until the process exits; nz > LBM_STATIC_MAX_PLANES is
 * rejected with LBM_EINVAL.  The first call in each device context (the
 * current device's primary context; again after a cudaDeviceReset) looks up
 * the array's device address with cudaGetSymbolAddress, so make that first
 * call before any stream capture.  All calls share the array: calls that overlap on the GPU
 * (other streams or threads) race; each call overwrites every entry it uses.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 * Synchronises `stream` (a cudaStream_t, NULL = default stream). */
#define LBM_STATIC_MAX_PLANES 4096
int lbm_plane_average_static(const float *dev_ux, const uint8_t *dev_solid, int32_t nx, int32_t ny, int32_t nz,
                             double *host_out, void *stream);

void lbm_solver_destroy(lbm_solver *solver);

const char *lbm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */

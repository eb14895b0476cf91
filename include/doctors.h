/*
 * doctors.h - C-ABI of libdoctors, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of the deterministic CT dose method of Norris & Liu,
 * "Photon Fluence and Dose Estimation in Computed Tomography using a Discrete
 * Ordinates Boltzmann Solver" (arXiv:1811.12391):
 *
 *   1. uncollided point-source fluence per voxel and group by Siddon ray
 *      tracing (Sec. II.A, first-collision source method);
 *   2. multigroup discrete-ordinates source iteration of the collided
 *      problem, Eq. 2 with vacuum boundaries, step-differenced and swept as
 *      diagonal wavefronts over the eight octants;
 *   3. Legendre-moment scattering source (Eq. 2's kernel as a Legendre
 *      expansion), the scalar fluence of Eq. 3 and the dose tally (Sec. II.A,
 *      III.A: fluence times group-wise conversion factors);
 *   4. the discrete adjoint of 1-3 for gradients of a dose functional.
 *
 * Conventions
 *   - Every call returns an int status (DOCTORS_OK or a DOCTORS_ERR_* code);
 *     doctors_last_error() returns a thread-local description of the last
 *     failure.  On failure no output is written unless stated otherwise.
 *   - Voxel arrays are flat with x fastest: v = (k*ny + j)*nx + i.  Voxel
 *     (i,j,k) spans origin + [i,i+1)*dx (likewise y, z), in cm.
 *   - Group arrays are [G][V], group 0 the highest energy.
 *   - Cross sections are cm^-1 at unit density; the macroscopic value in a
 *     voxel is density[v] * table[mat[v]].  sigma_s holds the Legendre
 *     moments of the group-to-group scattering kernel, [n_mat][L+1][G][G]
 *     indexed (from, to); only downscatter (to >= from) is allowed.
 *   - A `mem` argument says where a caller buffer lives: DOCTORS_MEM_HOST or
 *     DOCTORS_MEM_DEVICE (device memory on the problem's device).  Caller
 *     buffers stay owned by the caller; the problem copies what it needs, so
 *     inputs may be freed after the call returns.  Device memory of the
 *     problem itself is owned by the handle and freed by doctors_destroy.
 *   - All GPU work is ordered on the CUDA stream given at creation.  Calls
 *     that return results to host memory synchronise that stream; calls that
 *     write device buffers are stream-ordered and do not synchronise.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef DOCTORS_H
#define DOCTORS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DOCTORS_OK                 0
#define DOCTORS_ERR_INVALID_ARG    1   /* a bad pointer, size, order or table */
#define DOCTORS_ERR_OOM            2   /* device allocation failed */
#define DOCTORS_ERR_CUDA           3   /* a CUDA runtime call failed */
#define DOCTORS_ERR_NOT_CONVERGED  4   /* iteration cap reached (results still written) */
#define DOCTORS_ERR_TIMEOUT        5   /* a bounded device-side wait gave up */
#define DOCTORS_ERR_STATE          6   /* call out of order (e.g. dose before solve) */

/* memory spaces of caller buffers */
#define DOCTORS_MEM_HOST    0
#define DOCTORS_MEM_DEVICE  1

/* source kinds (Sec. II.B: point sources, fan beams and cone beams) */
#define DOCTORS_SRC_POINT     0   /* isotropic point source outside the mesh */
#define DOCTORS_SRC_FAN_CONE  1   /* point source behind a rectangular fan x cone collimator */
#define DOCTORS_SRC_VOLUME    2   /* uniform isotropic volume source over the whole mesh */

/* which fluence doctors_get_fluence returns */
#define DOCTORS_FLUENCE_UNCOLLIDED  0
#define DOCTORS_FLUENCE_COLLIDED    1
#define DOCTORS_FLUENCE_TOTAL       2
#define DOCTORS_FLUENCE_ADJOINT     3   /* adjoint scalar fluence (importance) of the last adjoint solve */

/* spatial differencing of the sweep (doctors_options.differencing) */
#define DOCTORS_DIFF_STEP     0
#define DOCTORS_DIFF_DIAMOND  1

/* Voxel mesh (Sec. II.D: Cartesian voxel phantoms). */
typedef struct doctors_mesh {
    int nx, ny, nz;          /* voxels per axis, each >= 1 */
    double dx, dy, dz;       /* voxel size in cm, > 0 */
    double origin[3];        /* corner of voxel (0,0,0) in cm */
} doctors_mesh;

/* Solver options (Sec. II.D: quadrature order, Legendre order, groups). */
typedef struct doctors_options {
    int groups;              /* G, 1..64 */
    int sn_order;            /* N of the level-symmetric S_N set: 2,4,6,8,12,16 (N(N+2) directions) */
    int legendre;            /* L, 0..3: (L+1)^2 flux moments */
    double tol;              /* stop when, in every group, ||phi00_new - phi00_old||_2 / ||phi00_new||_2 < tol;
                                values below 1e-6 are raised to 1e-6 (FP32 sweep) */
    int max_iters;           /* source-iteration cap, >= 1 */
    int tile_x, tile_y;      /* sweep tile in voxels (0 = default: 8 x 8 for the dataflow sweep, else
                                16 x 16); tile_x*tile_y <= 256 */
    int angles_per_block;    /* directions per sweep block (0 = default: whole octants on the dataflow
                                sweep, else the largest of 12, 10, 9, 7, ... dividing it); must divide
                                N(N+2)/8; 21 and 36 (whole S12, S16 octants) on the dataflow sweep only */
    int sweep_kernel;        /* 0 = default (the fastest measured: dataflow with a face warp (7) where
                                it applies, else plain dataflow (4), else chained (3)),
                                1 = CUDA-core transforms, one task (tile, octant, direction block,
                                group) per CTA, 3 = CUDA-core transforms, each CTA running a chain of
                                tasks of a stage back to back in one hyperplane pipeline,
                                4 = dataflow: one launch per sweep, CTAs take tasks from a queue and
                                wait (bounded) on their upstream tiles' face fluxes plane by plane;
                                needs angles_per_block = N(N+2)/8 with N <= 8, 12 or 16 (whole
                                octants), or angles_per_block = 12 at S16 (one launch per block of
                                12 directions).  A wait that gives up makes the solve return
                                DOCTORS_ERR_TIMEOUT,
                                5 = dataflow with the transforms split out: a pass turns the source
                                moments into angular sources of all directions, the sweep reads and
                                writes one angular record per cell, a pass turns the angular fluence
                                back into moments (whole octants of S2..S8 only; two more arrays
                                of G x N(N+2) x V floats, padded),
                                7 = dataflow with a face warp: one more warp per CTA fetches and
                                waits for the incoming face fluxes, the column threads only sweep
                                (same conditions as 4, P1 or P3, tile_x + tile_y <= 64),
                                8 = as 5 with the two transform passes on the tensor cores
                                (tcgen05, 3xTF32 with FP32 accumulation; P3 only).
                                2 and 6 are not offered (DOCTORS_ERR_INVALID_ARG): a sweep with
                                the transforms on mma.sync tensor cores and a dataflow sweep of two
                                groups per task, both measured slower than 1, 3, 4 and 7 on
                                every workload, were taken out */
    int device_loop;         /* 1 = run the source iteration as one CUDA graph whose while loop is
                                decided on the device (no host round trip per iteration) */
    int differencing;        /* spatial scheme of the sweep (the paper does not state one):
                                DOCTORS_DIFF_STEP (0, default): every outgoing face flux is the cell
                                flux, psi = (q + sum_d c_d psi_in,d) / (sigma_t + sum_d c_d);
                                DOCTORS_DIFF_DIAMOND (1): the cell flux is the mean of each face pair,
                                psi = (q + 2 sum_d c_d psi_in,d) / (sigma_t + 2 sum_d c_d) and
                                psi_out,d = 2 psi - psi_in,d, with no negative-flux fixup
                                (c_d = |Omega_d| / delta_d).  Diamond differencing runs on the dataflow
                                sweep only: sweep_kernel 0 or 4, angles_per_block = N(N+2)/8, N <= 8
                                or N = 12, 16 */
    int reserved[5];         /* must be zero */
} doctors_options;

/* One source (Sec. II.B: position, energy distribution, azimuthal and polar
 * opening angles).  A point source must lie outside the mesh.  The emission
 * is weight * spectrum[g] photons per source particle in group g, isotropic
 * per 4 pi, masked by the collimator: a voxel centre c is lit when, with
 * u = c - pos, along = u.axis > 0, |u.perp| <= tan(fan_deg/2) * along and
 * |u.up| <= (z_half_iso / iso_dist) * along, where perp = (-a_y, a_x, 0) /
 * |(a_x, a_y)| ((1,0,0) if the axis is along z) and up = axis x perp; the
 * test is taken in FP32.  A volume source emits weight * spectrum[g] photons
 * per cm^3 in group g everywhere in the mesh. */
typedef struct doctors_source {
    int kind;                /* DOCTORS_SRC_* */
    double pos[3];           /* cm (point kinds) */
    double axis[3];          /* unit beam axis, source -> isocentre (fan/cone) */
    double fan_deg;          /* full in-plane opening angle (fan/cone) */
    double z_half_iso;       /* beam half-height at the isocentre distance, cm (fan/cone) */
    double iso_dist;         /* source-to-isocentre distance, cm (fan/cone) */
    double weight;           /* per-view weight (tube-current weight) */
    const double *spectrum;  /* [G], host memory */
} doctors_source;

/* Solve report. */
typedef struct doctors_result {
    int iterations;          /* sweeps performed */
    int converged;           /* 1 if every group met the tolerance */
    double residual;         /* max over groups of the last relative change (FP64) */
    double balance_rel;      /* |sum source - sum absorption - leakage| / sum source of the last sweep (FP64) */
    double tol_used;         /* tolerance actually applied */
    double cell_updates;     /* voxel x direction x group updates performed */
    double ms_raytrace;      /* device time of ray trace + first-collision source */
    double ms_iterate;       /* device time of the source iteration */
    double ms_sweep;         /* device time of the sweep launches alone (summed over iterations) */
    double ms_total;         /* device time of the whole call */
    long long launches;      /* kernels launched by the call */
} doctors_result;

typedef struct doctors_problem doctors_problem;

/* Create a problem on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream); all later work is ordered on
 * it.  Validates the mesh and options (DOCTORS_ERR_INVALID_ARG), builds the
 * level-symmetric quadrature (Sec. II.D, Eq. 3) and the harmonics tables,
 * and allocates the device state (DOCTORS_ERR_OOM).  *out is set only on
 * success. */
int doctors_create_problem(const doctors_mesh *mesh, const doctors_options *opt,
                           void *cuda_stream, doctors_problem **out);

/* Set the voxel materials and cross sections (Sec. II.B: CT data converted
 * to dosimetrically equivalent materials; Eq. 2's sigma_t and Legendre
 * scattering moments).  mat [V] uint8 (< n_mat) and density [V] float32 (>= 0;
 * NULL = all 1) live in `mem`; sigma_t [n_mat][G] and sigma_s
 * [n_mat][L+1][G][G] (from, to) are host doubles, n_mat 1..8.  Rejects
 * upscatter, negative values and sum_g' sigma_s,0(g->g') > sigma_t(g).
 * Invalidates any previous solution. */
int doctors_set_materials(doctors_problem *p, int n_mat, const uint8_t *mat, const float *density,
                          const double *sigma_t, const double *sigma_s, int mem);

/* Set the sources (Sec. II.B; Sec. II.C: several concurrent projections form
 * a CT scan and are superposed in one problem).  n_src 1..4096, host array.
 * Invalidates any previous solution. */
int doctors_set_source(doctors_problem *p, int n_src, const doctors_source *src);

/* Solve: Siddon ray trace of the uncollided fluence of every point source
 * and its first-collision source (Sec. II.A), then source iteration of the
 * collided problem (Eq. 2, vacuum boundaries) with step-differenced (or, per
 * options.differencing, diamond-differenced) octant wavefront sweeps, all
 * active groups per sweep.  Synchronises the stream.  Returns
 * DOCTORS_ERR_NOT_CONVERGED (results kept) if max_iters is reached.  `info`
 * may be NULL. */
int doctors_solve(doctors_problem *p, doctors_result *info);

/* Copy a group fluence [G][V] float32 (Eq. 3's scalar fluence; uncollided,
 * collided or their sum, or the adjoint scalar fluence of the last adjoint
 * solve) into `out` in `mem`.  DOCTORS_ERR_STATE before a successful solve
 * (or, for DOCTORS_FLUENCE_ADJOINT, before an adjoint solve). */
int doctors_get_fluence(doctors_problem *p, int which, float *out, int mem);

/* Dose tally (Sec. II.A, III.A): dose[v] = sum_g k[mat v][g] * density[v] *
 * (phi_u + phi_c)[g][v], accumulated in FP64.  k [n_mat][G] host doubles
 * (energy-deposition weights or fluence-to-dose factors); dose [V] float64
 * in `mem`.  DOCTORS_ERR_STATE before a successful solve. */
int doctors_dose(doctors_problem *p, const double *k, double *dose, int mem);

/* Dose tally that allocates nothing (the paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as code
 * inside a framework whose caching allocator owns the device memory, or
 * real-time and embedded callers that forbid allocation after start-up).
 * Same result as doctors_dose, written to `dose` [V] float64, which must be
 * device memory on the problem's device; k [n_mat][G] is host memory.  The
 * factor table is staged in a fixed array inside the library's device image
 * (at most 256 = n_mat * G entries; larger tables are rejected with
 * DOCTORS_ERR_INVALID_ARG), held by every GPU that loads the library until
 * the process exits.  All calls share that array: calls that overlap on the
 * GPU race on it.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, once per device, cached for the life of the
 * process: the cache assumes one context per device, so do not use it across
 * cudaDeviceReset); make that first call before any stream capture.
 * Stream-ordered, does not synchronise: k is copied with cudaMemcpyAsync on
 * the problem's stream.  From pageable host memory the copy is staged before
 * the call returns, so k may change at once; from pinned host memory the copy
 * runs when the stream reaches it, so k must stay unchanged until then (and,
 * under stream capture, for the life of the captured graph, which reads k on
 * every replay).  DOCTORS_ERR_STATE before a successful solve;
 * DOCTORS_ERR_INVALID_ARG for null or non-finite arguments; on either error
 * nothing is written. */
int doctors_dose_noalloc(doctors_problem *p, const double *k, double *dose);

/* Adjoint solve and gradients (no counterpart in the paper; the discrete
 * adjoint of the operator above).  For J = sum_{g,v} response[g][v] *
 * (phi_u + phi_c)[g][v] with response [G][V] float64 in `mem`, solves the
 * adjoint problem (directions reversed, scattering transposed) and writes,
 * for every non-NULL output (float64, in `mem`):
 *   d_weights [n_src]  dJ/d weight of each source,
 *   d_spectrum [G]     dJ/d spectrum[g], the spectrum taken as shared by all
 *                      point sources (sum over sources of weight * partial),
 *   d_density [V]      dJ/d density[v] through the transport (attenuation of
 *                      the uncollided rays, collisions and scattering); any
 *                      explicit density dependence of `response` is the
 *                      caller's.
 * Requires a successful doctors_solve (DOCTORS_ERR_STATE).  Synchronises.
 * `info` (may be NULL) reports the adjoint iteration. */
int doctors_adjoint_solve(doctors_problem *p, const double *response, int mem, double *d_weights,
                          double *d_spectrum, double *d_density, doctors_result *info);

/* Region-of-interest dose (Sec. II.A, III.A: the dose tally, summed over a
 * region with voxel weights).  J = sum_v roi[v] * dose[v], dose as in
 * doctors_dose, summed in FP64 on the device in a fixed order (the same
 * inputs give the same bits).  k [n_mat][G] host doubles, finite; roi [V]
 * float64 in `mem` (finite); *J is host memory; dose [V] float64 in `mem`
 * or NULL.  Host inputs are copied before the call returns.  DOCTORS_ERR_STATE
 * before a successful solve; DOCTORS_ERR_INVALID_ARG for null or non-finite
 * inputs, with no output written.  Synchronises. */
int doctors_roi_dose(doctors_problem *p, const double *k, const double *roi, int mem, double *J,
                     double *dose);

/* Gradients of the region-of-interest dose J above (no counterpart in the
 * paper; the discrete adjoint of Eq. 2 and the chain rule through the ray
 * trace and the tally).  Forms the adjoint response
 * r[g][v] = roi[v] * k[mat v][g] * density[v] on the device, solves the
 * adjoint as doctors_adjoint_solve does, and writes *J (host) and every
 * non-NULL output (float64, in `mem`): d_weights [n_src], d_spectrum [G] as
 * doctors_adjoint_solve, and d_density [V] = the full dJ/d density[v]: the
 * transport part plus the dose's own density factor
 * roi[v] * sum_g k[mat v][g] * (phi_u + phi_c)[g][v].  Argument rules as
 * doctors_roi_dose; `info` (may be NULL) reports the adjoint iteration;
 * DOCTORS_ERR_NOT_CONVERGED keeps the outputs.  Synchronises. */
int doctors_roi_gradients(doctors_problem *p, const double *k, const double *roi, int mem, double *J,
                          double *d_weights, double *d_spectrum, double *d_density, doctors_result *info);

/* Test hook for the dataflow sweep's bounded waits (sweep_kernel 4 or 5): from the
 * next sweep on, the sweep task numbered `task` (stage-major order) does not
 * write the face fluxes it owes its downstream tiles, so their waits run out;
 * the solve then returns DOCTORS_ERR_TIMEOUT and resets the sweep's queue and
 * face buffers.  task < 0 clears the hook.  DOCTORS_ERR_STATE if the problem's
 * sweep is not the dataflow kernel.  The paper has no counterpart. */
int doctors_debug_withhold_faces(doctors_problem *p, int task);

/* Test hook: the voxel index list and segment lengths of the ray from
 * source `src` to the centre of voxel `voxel`, as walked by the ray-trace
 * kernel (FP32, from the target back toward the source; see Sec. II.A).
 * idx and len are host arrays of capacity cap; *n receives the count.
 * DOCTORS_ERR_INVALID_ARG if cap is too small or src is not a point source. */
int doctors_debug_ray_indices(doctors_problem *p, int src, int voxel, int32_t *idx, float *len,
                              int cap, int *n);

/* CT numbers -> materials and densities (Sec. II.B: the reconstructed CT
 * image is converted into dosimetrically equivalent materials through a
 * calibration; the paper cites a stoichiometric calibration it does not
 * print).  Applies any piecewise calibration, voxel by voxel:
 *   material: bin b = the number of thresholds t_i with t_i <= hu (so a CT
 *     number equal to a threshold falls in the upper bin),
 *     mat_out = bin_material[b]; thresholds [n_thresholds] strictly
 *     ascending, finite, 0..31 of them; bin_material [n_thresholds + 1];
 *   density: piecewise linear through the knots (hu_knots[k], rho_knots[k]),
 *     k = 0..n_knots-1 (1..32 knots, CT numbers strictly ascending, densities
 *     finite and >= 0), constant rho_knots[0] below the first knot and
 *     rho_knots[n_knots-1] at or above the last; within hu_knots[k] <= hu <
 *     hu_knots[k+1]:  t = (hu - hu_knots[k]) / (hu_knots[k+1] - hu_knots[k]),
 *     rho = rho_knots[k] + t * (rho_knots[k+1] - rho_knots[k]), each operation
 *     an FP32 operation rounded to nearest, in that order (no fused
 *     multiply-add).
 * A NaN CT number gives bin 0 and rho_knots[0].
 * hu [n] float32, mat_out [n] uint8, rho_out [n] float32: all host or all
 * device memory per `mem` (device: on the current device); the tables are
 * host memory.  Device memory: stream-ordered on `cuda_stream` (NULL: the
 * legacy default stream), does not synchronise; host memory: staged
 * through temporary device buffers, synchronises.  The outputs feed
 * doctors_set_materials.  DOCTORS_ERR_INVALID_ARG for bad tables or null
 * arrays (checked before any device work). */
int doctors_ct_to_materials(const float *hu, size_t n, int n_thresholds, const float *thresholds,
                            const uint8_t *bin_material, int n_knots, const float *hu_knots,
                            const float *rho_knots, uint8_t *mat_out, float *rho_out, int mem,
                            void *cuda_stream);

/* Level-symmetric quadrature and real spherical harmonics as used by the
 * sweep (Sec. II.D, Eq. 3).  Host only, needs no GPU.  dirs [A][3], w [A],
 * R [A][(L+1)^2] host doubles (any may be NULL), A = N(N+2), directions
 * octant-major.  *n_dirs receives A. */
int doctors_quadrature(int sn_order, int legendre, double *dirs, double *w, double *R, int *n_dirs);

/* Solve several problems (e.g. the views of an axial scan, or phantoms of
 * different mesh sizes) as one batch (Sec. II.C: a CT scan is many
 * concurrent projections).  After each problem's ray trace, one CUDA graph
 * holds every problem's source iteration inside a device-side while loop:
 * per iteration, every live problem's scattering source, all its wavefront
 * stages and its FP64 residual, then a one-thread decision that retires the
 * problems that have converged (their kernels return at entry from then on)
 * and ends the loop when all are retired.  Everything runs on the first
 * problem's stream; all problems must be on one device and have materials
 * and sources set.  results[i] (array may be NULL) receives problem i's
 * report; the batch's device time is in every report's ms_total. */
int doctors_solve_batch(doctors_problem **problems, int n, doctors_result *results);

/* Sweep schedule chosen by doctors_autotune. */
typedef struct doctors_tuning {
    int tile_x, tile_y;      /* tile of columns */
    int angles_per_block;    /* directions per CTA */
    int sweep_kernel;        /* 1 CUDA-core, 3 chained, 4 dataflow, 5 dataflow with split transforms,
                                7 dataflow with a face warp, 8 split transforms on the tensor cores
                                (as doctors_options) */
    double ms_per_sweep;     /* measured time of one full sweep of this problem */
    int candidates;          /* schedules timed (0 if taken from the cache) */
} doctors_tuning;

/* Autotune the wavefront schedule (tile shape, directions per CTA and the
 * moment-transform path) of a problem whose materials and sources are set:
 * each candidate schedule is timed on two sweeps of the problem's own
 * first-collision source with CUDA events, and the fastest is installed.
 * Results are cached per (mesh size, S_N order, Legendre order, groups) for
 * the life of the process.  Synchronises; invalidates any solution.  `out`
 * may be NULL. */
int doctors_autotune(doctors_problem *p, doctors_tuning *out);

/* Release the problem and its device memory.  NULL is ignored. */
void doctors_destroy(doctors_problem *p);

/* Thread-local description of the last error ("" if none). */
const char *doctors_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DOCTORS_H */

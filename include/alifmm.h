/*
 * alifmm.h -- C ABI of the GB300 (sm_103a) ALI-FMM travel-time library.
 *
 * The library computes first-arrival qP travel-time fields in 2D heterogeneous
 * orthotropic media with the Anisotropic Locally Interpolated Fast Marching
 * Method of Ludlam, Tant, Dolean and Curtis ("Travel times and ray paths for
 * acoustic and elastic waves in generally anisotropic media", arXiv 2302.10988),
 * for many sources and many media samples at once; it then traces rays back
 * through those fields and returns the adjoint gradient of a receiver-time
 * misfit with respect to region orientations.
 *
 * Problem statement (Sec. 2 and Sec. 6 of the paper): a stiffness tensor and a
 * density per material, a grain-orientation map on a grid, and source and
 * receiver nodes go in; travel-time fields, receiver times and ray paths come
 * out.
 *
 * Conventions (all entry points)
 *  - Grid node (i, j) is at x = i*h, y = j*h.  Fields are stored row-major,
 *    node (i, j) of a field at offset j*nx + i.
 *  - A "field" is one (sample b, source s) pair, numbered f = b*S + s.  The
 *    fields of a plan are packed back to back; alf_plan_field_offset() gives
 *    the first node of each.
 *  - Angles are radians.  An orientation is the CCW angle from +x to the
 *    material's phase-angle-zero axis (the axis along which the qP phase
 *    speed is sqrt(c22/rho)), Sec. 3.2.
 *  - SI units: Pa, kg/m^3, m, s.
 *  - Unless a parameter says "host", pointers are CUDA device pointers owned
 *    by the caller; the library never frees them.  The library owns only the
 *    workspaces inside alf_ctx and alf_plan.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call that takes a stream only enqueues work on it and
 *    returns without synchronising, unless stated otherwise.
 *  - Every call returns an alf_status.  Arguments are validated on the host
 *    before anything is launched; on failure nothing is enqueued and
 *    alf_last_error() describes the problem.  Kernels never trap: device-side
 *    failures (no convergence, an incomplete ray, an adjoint sweep that could
 *    not release every node) are written to the plan's status words and read
 *    back by alf_sync_status().
 */
#ifndef ALIFMM_H
#define ALIFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ALF_OK = 0,
    ALF_ERR_INVALID_ARG = 1,          /* a pointer, size or option is out of range */
    ALF_ERR_NONPHYSICAL_MATERIAL = 2, /* rho <= 0, non-finite stiffness, or an in-plane stiffness that is not
                                         positive definite (c22, c33, c44 > 0 and c22 c33 > c23^2) */
    ALF_ERR_OUT_OF_GRID = 3,          /* a source or receiver node lies outside its grid */
    ALF_ERR_CUDA = 4,                 /* a CUDA runtime call failed (message has the CUDA error) */
    ALF_ERR_OOM = 5,                  /* a workspace allocation failed */
    ALF_ERR_NOT_CONVERGED = 6,        /* the sweeps hit their visit cap before reaching the fixed point */
    ALF_ERR_RAY_INCOMPLETE = 7,       /* a ray hit its point cap before reaching its target */
    ALF_ERR_UNSUPPORTED = 8,          /* a feature not available in this build */
    ALF_ERR_INCONSISTENT_RECORDS = 9  /* alf_backward: some node was never released by the reverse sweep
                                         (the records or times do not come from one solve of this plan) */
} alf_status;

typedef enum { ALF_FP64 = 0, ALF_FP32 = 1 } alf_precision;

/* Straight-ray (group) speed model, used by the near-source initialisation,
 * by the no-stencil fallback and by ray segments:
 *  ALF_GROUP_PAPER: the paper's group->phase inversion (Sec. 3.2, Eqs.
 *                   eigen_eq2, eigen_eq3, lambda_1): the phase angle whose qP
 *                   polarisation lies along the group angle, |V| = |v|/cos(theta-phi);
 *  ALF_GROUP_EXACT: the ray velocity of the qP slowness curve, psi = theta +
 *                   atan(v'/v), |V| = sqrt(v^2 + v'^2), by an FP64 Newton solve. */
typedef enum { ALF_GROUP_PAPER = 0, ALF_GROUP_EXACT = 1 } alf_group_model;

/* Near-source initialisation (Sec. 4.4):
 *  ALF_INIT_RADIUS:    nodes within Chebyshev distance init_radius of the
 *                      source get straight-ray times (exact while the medium
 *                      around the source is homogeneous);
 *  ALF_INIT_HIERARCHY: the paper's refined grids (densities level_density[],
 *                      out to level_radius[] original cells), straight rays
 *                      inside the source cell on the finest one; each level
 *                      stops at the first node on the boundary of its square
 *                      (in key order) and hands its known nodes that coincide
 *                      with the next level's nodes to it as frozen nodes.
 *                      Level grids are at most 2^16 nodes.  alf_backward does
 *                      not differentiate this initialisation
 *                      (ALF_ERR_UNSUPPORTED). */
typedef enum { ALF_INIT_RADIUS = 0, ALF_INIT_HIERARCHY = 1 } alf_init_mode;

/* One material: 6x6 Voigt stiffness (Pa) and density (kg/m^3).  Only the
 * YZ-plane entries c22 = c[1][1], c23 = c[1][2], c33 = c[2][2], c44 = c[3][3]
 * enter the in-plane qP speed (Sec. 3.2); a material with c22 == c33 and
 * c23 == c22 - 2*c44 is treated as isotropic with speed sqrt(c22/rho). */
typedef struct {
    double c[6][6];
    double rho;
} alf_material;

typedef struct {
    int precision;          /* alf_precision of the sweeps and of every float output */
    int group_model;        /* alf_group_model */
    int init_mode;          /* alf_init_mode */
    int init_radius;        /* ALF_INIT_RADIUS: 0..8 (default 2) */
    int n_levels;           /* ALF_INIT_HIERARCHY: 1..4 levels (default 3) */
    int level_density[4];   /* odd, decreasing, > 1 (default 27, 9, 3) */
    int level_radius[4];    /* original cells, increasing (default 1, 6, 13) */
    int plane_step;         /* ray tracer plane spacing, cells (default 4) */
    int ray_halfwidth;      /* candidate nodes each side of the predicted crossing (default 8, max 16) */
    double stop_radius;     /* stop when this close to the target, cells (default 1.6) */
    int max_ray_points;     /* points per ray including both ends (default 512) */
    int max_rounds;         /* livelock guard: sweep rounds per field <= max_rounds * (nx + ny) (default 64) */
    int sweep;              /* sweep schedule: 1 = all fields advance in lockstep rounds, each round a few
                               kernels over the whole batch; 2 = one warp owns each field and runs all
                               its rounds inside one launch (suits many fields; needs nx*ny/8 bytes of
                               shared memory per warp, nx*ny <= 2^18); 3 = one CTA owns each field,
                               one launch (suits few large fields); 4 = active tiles: one CTA per field
                               iterates F on 8 x 8 tiles in shared memory until no node of a tile changes
                               and wakes the neighbouring tiles that read a changed border (no front band;
                               never chosen by 0 or by alf_plan_autotune); 0 = choose (2 when it fits and
                               the fields fill the GPU, else 3), default 0 */
    int ray_family;         /* planes of the ray tracer (Sec. 5.1): 0 = the set most perpendicular to the
                               ray at every step (default); 1..4 = one fixed set: x = c, y = c, x - y = c,
                               x + y = c; 5 = the fastest of the four fixed sets (Table 3 compares them) */
    int keep_records;       /* 1: keep per-node stencil records for alf_backward (default 0) */
    double band_cells;      /* sweep schedule: nodes later than the front by more than this many
                               cell-crossing times wait for the front (default 2; <= 0: no band) */
    int use_graph;          /* 1: replay the sweep rounds from a CUDA graph (default 1) */
    int time_kernels;       /* 1: time the evaluation kernel with CUDA events (alf_plan_stats; default 0) */
    int velocity_table;     /* 1: the local update takes the qP phase speed by linear interpolation in a table
                               of phase speeds at integer degrees (Sec. 3; Table 2 compares it with solving
                               the Christoffel matrix at run time, 0, the default).  Group speeds (source
                               initialisation, fallback, rays) are unchanged.  alf_backward refuses it. */
    int cta_threads;        /* sweep 3: threads of the CTA that owns a field, 64, 128, 256 or 512 (2 to 16
                               warps); 0 = choose (default): 512 for FP32 batches with no more fields than
                               SMs, else 256.  alf_plan_autotune chooses it among the four. */
    int cta_cluster;        /* sweep 3: CTAs of 512 threads that share one field as a thread-block cluster on
                               as many SMs, 1, 2, 4 or 8; 0 = choose (default): for FP32 batches with no more
                               fields than SMs, the largest that keeps fields x cluster <= SMs and leaves at
                               least 2^19 nodes of the largest field per SM, else 1 */
    int subgrid;            /* global sub-grid size s (Sec. 4.5, Table 2; Sec. 5.1), odd, 1..21 (default 1):
                               the plan solves every sample on its grid refined s times in each direction,
                               (nx - 1) s + 1 by (ny - 1) s + 1 nodes of spacing h / s, each fine node taking
                               the region of the nearest original node; sources and receivers sit at the
                               fine nodes (i s, j s).  Fields, records, ray points and every field offset are
                               those of the fine grid; the original nodes are every s-th fine node.
                               init_radius, level_radius, plane_step, ray_halfwidth and stop_radius stay in
                               original cells (the plan multiplies them by s); level_density is relative to
                               the fine grid. */
    int wave_mode;          /* 0 = qP (default); 1 = qSV, the smaller in-plane eigenvalue of the Christoffel
                               matrix; 2 = SH, its out-of-plane eigenvalue c66 cos^2 + c55 sin^2 (Sec. 7: S-wave
                               times from the other eigenvalues of Sec. 3.2).  The local update takes the
                               mode's phase speed.  For the shear modes group speeds (initialisation, fallback,
                               rays) are the envelope 1/V(psi) = max over phase angles theta of
                               cos(theta - psi) / v(theta) -- the eikonal's solution around a point source,
                               single valued where the qSV ray surface has cusps -- tabulated per material at
                               1/8 degree on the device and interpolated; group_model is then not used.  At
                               most 4096 materials. */
} alf_options;

/* Fills `opt` with the defaults listed above.  Never fails. */
void alf_default_options(alf_options* opt);

/* Geometry of a batch: nsamples media on their own grids, all sharing the
 * region->material table, each with the same number of sources and receivers.
 * Every pointer here is HOST memory, read during alf_plan_create() only.
 *  nx[b], ny[b]   grid size of sample b, 2..16384 each, nx*ny <= 2^28
 *  h[b]           node spacing of sample b (m), > 0
 *  region_map     uint16 region id per node, samples packed back to back,
 *                 sample b is [ny[b]][nx[b]]; may be NULL when region_map32 is given
 *  region_map32   the same with uint32 ids, for more than 65,536 regions (a
 *                 per-node orientation map is nregions = nx*ny with region id
 *                 = node index); used instead of region_map when not NULL
 *  nregions       1..2^28, with nsamples * nregions <= 2^30
 *  region_material[r]  material index of region r (< nmaterials); may be NULL when region_material32 is given
 *  region_material32    the same with uint32 indices, for more than 65,536 materials (a per-node stiffness
 *                 map is one material per region); used instead of region_material when not NULL
 *  nmaterials     1..2^28 (velocity_table: at most 65,536)
 *  src_ij[b][s][2], rec_ij[b][r][2]  (i, j) nodes, inside the sample's grid */
typedef struct {
    int nsamples;
    const int32_t* nx;
    const int32_t* ny;
    const double* h;
    const uint16_t* region_map;
    int nregions;
    const uint16_t* region_material;
    int nmaterials;
    const alf_material* materials;
    int nsources;
    const int32_t* src_ij;
    int nreceivers;
    const int32_t* rec_ij;
    const uint32_t* region_map32;
    const uint32_t* region_material32;
} alf_geometry;

typedef struct alf_ctx alf_ctx;
typedef struct alf_plan alf_plan;

/* Context on one CUDA device (made current for every call of the context).
 * Errors: ALF_ERR_INVALID_ARG (out == NULL), ALF_ERR_CUDA (no such device, or
 * not an sm_103 device). */
alf_status alf_create(alf_ctx** out, int cuda_device);
alf_status alf_destroy(alf_ctx* ctx);
/* Message of the last failed call on `ctx` (thread-unsafe; "" if none). */
const char* alf_last_error(const alf_ctx* ctx);

/* Builds a plan: validates materials (Sec. 3.2 constants), grids, sources and
 * receivers; uploads the geometry and allocates the sweep workspaces (per-CTA
 * active lists and bitmaps, per-region tables).  Options are copied; NULL
 * means defaults.  Synchronous. */
alf_status alf_plan_create(alf_ctx* ctx, const alf_geometry* geom, const alf_options* opt, alf_plan** out);
alf_status alf_plan_destroy(alf_plan* plan);
/* Node offset of field f in the packed times buffer; total_nodes for f = nfields. */
size_t alf_plan_field_offset(const alf_plan* plan, int field);
int alf_plan_nfields(const alf_plan* plan);
/* Options in effect (after autotuning, if it ran); `sweep` is the schedule in use (1, 2 or 3). */
alf_status alf_plan_options(const alf_plan* plan, alf_options* out);

/* Forward solve (Secs. 2, 4): for every field, the near-source initialisation
 * then the ALI local update iterated to its fixed point (the heap FMM's
 * result) by sweep rounds: each round re-evaluates, in a field, the dirty
 * nodes (those whose neighbourhood changed) near the front, until every dirty
 * set is empty.  Sweeps 2 and 3 run every field's rounds inside one launch
 * (one warp, one CTA or one cluster of CTAs per field, fields taken from a
 * queue), so the call only enqueues work on `stream` (it waits only when the
 * plan times its kernels).  Sweep 1 enqueues lockstep rounds over all fields
 * and synchronises `stream` every 32 rounds to read the remaining work, so it
 * returns once the rounds are done (the finalisation and receiver gather are
 * still enqueued, not waited for).  Every schedule reaches the same fixed
 * point, bit for bit.
 *  region_theta   [nsamples][nregions] double, orientation of each region
 *  times          [total nodes] float (ALF_FP32) or double (ALF_FP64), output
 *  rec_times      [nsamples][nsources][nreceivers], same dtype, output; may be NULL
 *  records        [total nodes] uint8 stencil record per node, output; may be NULL:
 *                 0..31 stencil row 2*(pair-1)+(member-1) (Sec. 4.1 tables),
 *                 32+k fallback through diamond slot k, 254 frozen, 255 none.
 *                 Diamond slot order: (-1,0) (1,0) (0,-1) (0,1) (-1,-1) (1,-1)
 *                 (-1,1) (1,1) (-2,0) (2,0) (0,-2) (0,2).
 * Status is recorded per plan; read it with alf_sync_status(). */
alf_status alf_solve(alf_plan* plan, const double* region_theta, void* times, void* rec_times, uint8_t* records,
                     void* stream);

/* After alf_solve, the three calls below read its outputs and write disjoint
 * workspaces of the plan, so they may run at the same time on different
 * streams (each ordered after the solve by the caller).  Two calls of the same
 * function on one plan must not overlap. */

/* FP64 convergence check (the precision policy's final check): evaluates the
 * local update F in double precision at every node of a solved field and
 * writes per field the largest |F64(tau) - tau| / tau and the number of nodes
 * whose FP64 stencil record differs from `records` (if given).
 *  times        solved fields (precision of the plan), input
 *  records      records of that solve, or NULL
 *  max_rel      [nfields] double, output
 *  n_flips      [nfields] int32, output (0 when records is NULL) */
alf_status alf_check64(alf_plan* plan, const double* region_theta, const void* times, const uint8_t* records,
                       double* max_rel, int32_t* n_flips, void* stream);

/* The same FP64 check, also returning every node's FP64 value and stencil
 * record (for node-by-node comparison with a reference evaluation):
 *  check_times    [total nodes] double, output: U(S_D) in FP64, where S_D is
 *                 the node's frozen neighbours and those whose key (tau,
 *                 index) precedes its own; frozen nodes and nodes without a
 *                 value keep their time; may be NULL
 *  check_records  [total nodes] uint8, output: the record of that value
 *                 (codes as in alf_solve; 254 frozen, 255 none); may be NULL
 *                 (not both)
 * Other arguments as alf_check64. */
alf_status alf_check64_nodes(alf_plan* plan, const double* region_theta, const void* times, const uint8_t* records,
                             double* check_times, uint8_t* check_records, double* max_rel, int32_t* n_flips,
                             void* stream);

/* alf_solve followed by alf_check64 of the fields it solved, with the records
 * of the solve: the same outputs, bit for bit, as the two calls in turn.  With
 * the CTA-per-field sweep (schedule 3) in FP32, without a velocity table,
 * clusters of one CTA and no kernel timing, the check runs inside the solve
 * kernel, on each field right after its sweep converges and while the field is
 * still in L2 (one launch, no second pass over the fields); otherwise the check
 * is launched after the solve on `stream`.  The check reads the field before
 * the frozen marks are cleared and takes |tau| of every value, as the
 * separate check reads the cleared field.
 *  max_rel    [nfields] double, output, as alf_check64
 *  n_flips    [nfields] int32, output: nodes whose FP64 record differs from
 *             the one this solve wrote to `records` (0 when records is NULL)
 * Other arguments as alf_solve.  Status and errors as alf_solve. */
alf_status alf_solve_check64(alf_plan* plan, const double* region_theta, void* times, void* rec_times,
                             uint8_t* records, double* max_rel, int32_t* n_flips, void* stream);

/* Ray tracing (Sec. 5.1) for every (sample, source, receiver): the ray starts
 * at the receiver and walks plane by plane to the source through the source's
 * field (reciprocity), choosing the plane family most perpendicular to the last
 * segment and the lowest parabola vertex of cost(C) = |BC|/V_group + tau(C).
 *  times      solved fields, input
 *  ray_pts    [nsamples][nsources][nreceivers][max_ray_points][2] (x, y) in
 *             grid units, same dtype as times, output
 *  ray_npts   [.. same ..] int32 point count, output
 *  ray_time   [.. same ..] time integrated along the path through the
 *             nearest-node cells, same dtype, output; may be NULL
 *  ray_status [.. same ..] int32: 0 ok, 1 point cap reached, output; may be NULL */
alf_status alf_trace_rays(alf_plan* plan, const double* region_theta, const void* times, void* ray_pts,
                          int32_t* ray_npts, void* ray_time, int32_t* ray_status, void* stream);

/* Gradient of ray times along fixed paths (Sec. 5.1 integration; the paper's
 * motivation for ray paths, Sec. 1, is exactly this use in inversions): with
 * each ray's polyline held fixed, its time is the sum over pieces of
 * len h / V(dir - theta_region), and this returns, for every region,
 * dL/dtheta = sum over rays of dL/dT_ray * dT_ray/dtheta_region.  Cheaper than
 * alf_backward (no sweep) and first order in the path, which is optimal.
 *  ray_pts, ray_npts  the output of alf_trace_rays for the same plan
 *  dL_dray      [nsamples][nsources][nreceivers], dtype of the plan, input
 *  dL_dtheta    [nsamples][nregions] double, output (overwritten)
 * May run beside alf_check64 and alf_backward (it writes only dL_dtheta). */
alf_status alf_ray_gradient(alf_plan* plan, const double* region_theta, const void* ray_pts, const int32_t* ray_npts,
                            const void* dL_dray, double* dL_dtheta, void* stream);

/* The traced ray paths (Sec. 5.1) packed back to back, for a compact copy or
 * store: ray r's points are packed_pts[offsets[r] .. offsets[r + 1]).  Only the
 * points a ray has are read (its count clamped to 0..max_ray_points).
 *  ray_pts, ray_npts  the output of alf_trace_rays for the same plan, input
 *  packed_pts         [total points][2], the precision of the plan, output;
 *                     capacity for nrays * max_ray_points points covers any case
 *  offsets            [nrays + 1] int64, output: the points of the rays before
 *                     r (exclusive prefix sum of the counts); offsets[nrays] is
 *                     the total
 * nrays = nsamples * nsources * nreceivers, in the order of alf_trace_rays.
 * Device buffers, caller-owned; asynchronous on `stream`.  Returns
 * ALF_ERR_INVALID_ARG for a null pointer or a plan without receivers. */
alf_status alf_pack_rays(alf_plan* plan, const void* ray_pts, const int32_t* ray_npts, void* packed_pts,
                         int64_t* offsets, void* stream);

/* Adjoint (reverse-mode) gradient of the receiver times: given dL/dT at every
 * receiver, returns dL/dtheta for every region, by differentiating the chosen
 * stencil (or fallback) of every node and the straight-ray initialisation,
 * swept in reverse causal order.  Needs a plan created with keep_records = 1
 * and init_mode = ALF_INIT_RADIUS, and the times and records of the same solve.
 *  dL_drec      [nsamples][nsources][nreceivers], dtype of the plan, input
 *  dL_dtheta    [nsamples][nregions] double, output (overwritten) */
alf_status alf_backward(alf_plan* plan, const double* region_theta, const void* times, const uint8_t* records,
                        const void* dL_drec, double* dL_dtheta, void* stream);

/* Synchronises `stream` and returns in *worst (host) the first non-OK device
 * status recorded by the plan since the last call (then clears it), and the
 * matching alf_status as the return value. */
alf_status alf_sync_status(alf_plan* plan, void* stream, int32_t* worst);

/* Work counters of the last alf_solve (synchronises `stream`). */
typedef struct {
    uint64_t node_evaluations; /* evaluations of the local operator in the sweep */
    uint64_t rounds;           /* sweep rounds (sweep 1: of the whole batch; 2, 3: of the slowest field) */
    uint64_t nodes;            /* nodes of the plan */
    uint64_t eval_launches;    /* launches timed (option time_kernels = 1): the evaluation kernel of every
                                  round (sweep 1) or the one field-resident sweep kernel (sweep 2, 3) */
    double eval_ms;            /* their device time, measured with CUDA events on the solve's stream */
    uint64_t kernel_launches;  /* kernel launches issued by the library so far (whole process) */
    uint64_t dirty_entries;    /* dirty-list entries the rounds scanned (sweeps 2 and 3; 0 for sweep 1) */
} alf_stats;
alf_status alf_plan_stats(alf_plan* plan, void* stream, alf_stats* out);

/* Picks the sweep's launch parameters for this plan by timing full solves
 * of its batch (the faster of two per candidate) and keeps the fastest: the
 * schedule (unless the options fix it), the front band width (1..6 cells,
 * in half cells between 1 and 2.5)
 * and, for sweep 1, the evaluation CTA size (128 or 256 threads), for sweep 3
 * the threads per field's CTA (64..512, unless fixed) and, where the fields
 * leave SMs idle, a cluster of 2, 4 or 8 CTAs per field.  `times` and
 * `records` (may be NULL) are scratch outputs of those solves.  Synchronous. */
alf_status alf_plan_autotune(alf_plan* plan, const double* region_theta, void* times, uint8_t* records,
                             void* stream);

/* Velocity model on the device, for checks: out[k] = phase speed (kind 0, 2,
 * 4) or group speed (kind 1, 3, 5) of the qP (kinds 0, 1), qSV (2, 3) or SH
 * (4, 5) mode of material *mat (host) at angle angles[k] relative to the
 * material axis, computed in `precision`; qP group speeds by `group_model`,
 * shear group speeds by the envelope table (see alf_options.wave_mode).
 *  angles, out  device double arrays of n entries */
alf_status alf_eval_velocity(alf_ctx* ctx, const alf_material* mat, int kind, int group_model, int precision,
                             const double* angles, double* out, int n, void* stream);

/* Forward solve of ONE field that allocates no device memory (the paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- an application whose device memory belongs to another
 * allocator, or a latency-bound loop in which cudaMalloc/cudaFree, which can
 * synchronise the device, are not allowed).  It runs the lockstep-round
 * kernels of alf_solve (sweep 1) in FP32 with the radius initialisation and
 * the plan's default front band (2 cell-crossing times), but keeps every
 * workspace in a fixed device array inside the library (about 8 MB per GPU
 * that loads the library, held until the process exits).
 * Limits: nx*ny <= 512*512 nodes, nregions <= 1024, nmaterials <= 64,
 * init_radius <= 8; larger inputs are rejected with ALF_ERR_INVALID_ARG and a
 * message in err.
 *  cuda_device              device to run on (made current)
 *  materials[nmaterials]    host
 *  region_material[nregions], region_theta[nregions] (double), region_map[ny][nx]   device, input;
 *                           every region id must be < nregions and every material id < nmaterials (checked
 *                           on the device before any other kernel runs: ALF_ERR_INVALID_ARG otherwise)
 *  h, (si, sj)              spacing (m) and source node
 *  group_model              alf_group_model
 *  max_rounds               cap on the sweep rounds (0: 64 (nx + ny)); a field still changing after it
 *                           returns ALF_ERR_NOT_CONVERGED
 *  times[ny][nx]            device float, output (caller-owned)
 *  stream                   cudaStream_t as void*; the call synchronises it
 *  err, err_len             host buffer for a message (may be NULL)
 * The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress), so make it before any stream capture.  All calls
 * share the array: calls whose work overlaps on the GPU (other streams or
 * host threads) race on it.  Returns ALF_OK, ALF_ERR_INVALID_ARG,
 * ALF_ERR_OUT_OF_GRID, ALF_ERR_NONPHYSICAL_MATERIAL, ALF_ERR_CUDA or
 * ALF_ERR_NOT_CONVERGED. */
alf_status alf_solve_field_noalloc(int cuda_device, const alf_material* materials, int nmaterials,
                                   const uint16_t* region_material, int nregions, const double* region_theta,
                                   const uint16_t* region_map, int nx, int ny, double h, int si, int sj,
                                   int init_radius, int group_model, int max_rounds, float* times, void* stream,
                                   char* err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* ALIFMM_H */

/*
 * pcdf.h -- C ABI of the predicted composite distance field library (GB300,
 * sm_103a).
 *
 * The library builds the distance fields of Finean et al., "Motion Planning
 * in Dynamic Environments Using Context-Aware Human Trajectory Prediction"
 * (arXiv 2201.05058):
 *   - Sec. 6: a distance field of the static environment, a field per dynamic
 *     obstacle (the human primitive, a cylinder in the paper, a capsule here)
 *     at each predicted position, and the composite field taken as their
 *     per-voxel minimum;
 *   - Sec. 8: a sequence of n composite fields, one per predicted timestep,
 *     where obstacle factor i reads field min(i, n);
 *   - Sec. 7: the GPMP2 hinge-loss obstacle cost on the distance field,
 *     evaluated here at robot body-sphere centres by trilinear interpolation,
 *     and its gradient with respect to the centres.
 *
 * Conventions for every call
 *   Grid: int32 nx, ny, nz in [1, PCDF_MAX_DIM]; voxel edge vox (metres, finite,
 *   > 0); origin = world position of the grid corner.  Arrays are [nz][ny][nx],
 *   x fastest.  Voxel (i, j, k) has its centre at
 *   origin + (i + 1/2, j + 1/2, k + 1/2) * vox.
 *
 *   Signed squared EDT S (int32, voxel-index units): for a free voxel, the
 *   minimum of |v - u|^2 over occupied in-grid voxels u; for an occupied voxel,
 *   minus the minimum over free in-grid voxels.  An empty opposite set gives
 *   +PCDF_INF / -PCDF_INF.  S is never 0.  Cells outside the grid are neither
 *   occupied nor free.
 *
 *   Float field (fp32, metres): sign(S) * sqrtf((float)|S|) * vox with an IEEE
 *   round-to-nearest square root and product; +/-PCDF_INF gives +/-inf.
 *
 *   Capsule: 7 int32 (ax, ay, az, bx, by, bz, r) in 1/16-voxel fixed point
 *   measured from the grid corner, so the centre of voxel (i, j, k) is
 *   16 * (i, j, k) + 8.  A voxel belongs to the capsule iff its centre lies in
 *   the closed set of points within r of segment a-b (exact integer test).
 *   With PCDF_CYLINDER set in the radius word the primitive is the closed
 *   finite cylinder instead: points whose projection falls on the segment and
 *   whose distance to its line is at most r.  Coordinates must lie in
 *   [PCDF_CAP_MIN, PCDF_CAP_MAX] and 0 <= r <= PCDF_CAP_MAX_R.
 *
 *   Memory: device pointers are owned by the caller; the library keeps none
 *   past the call and allocates nothing.  Calls that need scratch take a
 *   caller-owned device workspace and report its size through the matching
 *   *_workspace_bytes query.  Pointers marked "host" are read during the call
 *   only.  The one exception is the context (pcdf_create): it owns a scratch
 *   buffer that it allocates and grows itself, for callers that prefer not to
 *   size workspaces.
 *
 *   Asynchrony: every device call is enqueued on `stream` (a cudaStream_t; NULL
 *   is the legacy default stream) and returns without waiting for the GPU.
 *   Host-side argument checks happen before anything is enqueued.
 *
 *   Errors: 0 on success, else a negative PCDF_E* code; pcdf_last_error()
 *   returns a message for the calling thread's last failure.
 */
#ifndef PCDF_H
#define PCDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PCDF_OK 0
#define PCDF_EINVAL (-1)   /* bad size, pointer, alignment or capsule range */
#define PCDF_ENOMEM (-2)   /* workspace smaller than the size query returned */
#define PCDF_ECUDA (-3)    /* a CUDA launch or runtime call failed */
#define PCDF_ETIMEOUT (-4) /* a bounded wait inside the batched kernel expired */

#define PCDF_INF 2147483647
#define PCDF_MAX_DIM 512
#define PCDF_MAX_T 1024
#define PCDF_MAX_H 64
#define PCDF_CAP_MIN (-8192)
#define PCDF_CAP_MAX 16384
#define PCDF_CAP_MAX_R 8192
/* OR-ed into a capsule's radius word: the primitive is the finite cylinder of
 * radius r around segment a-b with flat ends at a and b (the paper's human
 * primitive, Sec. 6) instead of the capsule; a != b is required. */
#define PCDF_CYLINDER (1 << 30)

typedef struct pcdf_grid {
    int32_t nx, ny, nz;
    float vox;
    float origin[3];
} pcdf_grid;

/* Message describing the calling thread's most recent failed call ("" if none). */
const char *pcdf_last_error(void);

/* pcdf_bounds_check  the debug build's index checks (no counterpart in the
 * paper; the stand-in for a memory checker).  The library compiled with
 * PCDF_CHECK_BOUNDS (libpcdf_checked.so) tests every global and shared index
 * of the static EDT, the capsule field, the composite z pass, the column
 * maxima and the cost query and its backward before the access; a failed
 * test skips the access (nothing traps) and records the first failure and a
 * count on the device.  This call waits for the device, then returns in
 * *first (nullable) the first failing check as (16-bit hash of its source
 * file name) << 16 | line, 0 if none, and in *count (nullable) the number of
 * failed checks; reset != 0 clears both.  In the normal build it returns
 * PCDF_EINVAL (and zeros). */
int pcdf_bounds_check(uint32_t *first, uint32_t *count, int32_t reset);

/* ABI version (major * 100 + minor). */
int pcdf_version(void);

/* ---------------------------------------------------------------------------
 * Static environment field (Sec. 6: the environment's distance field, computed
 * once or maintained).
 *
 * occ        device uint8 [nz][ny][nx], nonzero = occupied.
 * static_sq  device int32 [nz][ny][nx], out: signed squared EDT S.
 * static_sdf device fp32 [nz][ny][nx] or NULL, out: float field.
 * workspace  device, >= pcdf_static_workspace_bytes() bytes, 256-byte aligned.
 * ------------------------------------------------------------------------- */
int pcdf_static_workspace_bytes(const pcdf_grid *grid, size_t *bytes);
int pcdf_build_static_sdf(const pcdf_grid *grid, const uint8_t *occ, int32_t *static_sq, float *static_sdf,
                          void *workspace, size_t workspace_bytes, void *stream);

/* Allocation-free variant of pcdf_build_static_sdf (the paper has no
 * counterpart; it exists for callers that cannot allocate device memory when
 * they need the field, such as real-time loops that forbid allocation after
 * start-up or hosts whose device memory belongs to another runtime).  Same
 * arguments and result as pcdf_build_static_sdf, without a workspace: the
 * scratch is a fixed array inside the library (about 12 MB on every device
 * that loads it, held until exit), so grids are limited to
 * PCDF_NOALLOC_MAX_VOXELS voxels (larger grids fail with PCDF_EINVAL and
 * nothing is enqueued).  Allocates nothing itself.  CUDA loads the library's
 * modules lazily, so the driver allocates the array when the first call on a
 * device loads it: that call can fail with PCDF_ECUDA (out of memory), and a
 * caller that must not fail later makes its first call at start-up.  Every
 * call whose stream is not being captured looks up the array's device address
 * (cudaGetSymbolAddress, with the call's device current), so a device reset
 * between calls is harmless.  A call made while its stream is being captured
 * does not look the address up: it reuses the last one found on the device,
 * and fails with PCDF_EINVAL if there is none, so the first call on a device
 * should come before any stream capture.  All calls share
 * the array: calls that overlap on the GPU race on it and must be serialised
 * by the caller.  No part of the array needs to start at zero. */
#define PCDF_NOALLOC_MAX_VOXELS 2097152
int pcdf_build_static_sdf_noalloc(const pcdf_grid *grid, const uint8_t *occ, int32_t *static_sq, float *static_sdf,
                                  void *stream);

/* ---------------------------------------------------------------------------
 * Static-map utilities of the mapping pipeline (Sec. 8).
 *
 * pcdf_filter_voxels  clean-up of the static voxel map: out = occ with every
 *     occupied voxel cleared whose 26 in-grid neighbours hold fewer than
 *     min_neighbours (0..27) occupied voxels.  The paper clears voxels with
 *     fewer than five connected voxels (min_neighbours = 5 reads "connected"
 *     as the 26-neighbourhood).  occ, out: device uint8 [nz][ny][nx], nonzero
 *     = occupied, distinct buffers; out holds 0/1.
 * pcdf_collapse_2d  the 2-D map of the prediction module: out2d[j][i] = 1 iff
 *     occ[k][j][i] != 0 for some k in [z0, z1) (clipped to the grid; an empty
 *     range gives zeros).  out2d: device uint8 [ny][nx].  Its EDT is
 *     pcdf_build_static_sdf on the grid {nx, ny, 1}.
 * ------------------------------------------------------------------------- */
int pcdf_filter_voxels(const pcdf_grid *grid, const uint8_t *occ, int32_t min_neighbours, uint8_t *out, void *stream);
int pcdf_collapse_2d(const pcdf_grid *grid, const uint8_t *occ, int32_t z0, int32_t z1, uint8_t *out2d, void *stream);

/* ---------------------------------------------------------------------------
 * Predicted composite fields (Sec. 6 composition; Sec. 8 sequence of n fields).
 *
 * For t = 0..T-1:  comp[t] = min(S_static, S_dyn[t])  per voxel, where S_dyn[t]
 * is the signed squared EDT of the voxels inside any of the H capsules at t.
 *
 * static_sq  device int32 [nz][ny][nx] (from pcdf_build_static_sdf).
 * static_sdf device fp32 [nz][ny][nx] or NULL: the float field that
 *            pcdf_build_static_sdf produced with static_sq.  When given, the
 *            float output copies it wherever the static field wins the min
 *            instead of recomputing the square root (same bits either way; a
 *            float field that does not belong to static_sq gives wrong output).
 * caps       HOST int32 [T][H][7] capsules (see conventions); may be NULL iff
 *            H == 0 (then every comp[t] equals the static field).
 * comp_sq    device int32 [T][nz][ny][nx] or NULL.
 * comp_sdf   device fp32 [T][nz][ny][nx] or NULL (at least one output non-NULL).
 * workspace  device, >= pcdf_composite_workspace_bytes(grid, T, H, caps).
 * 1 <= T <= PCDF_MAX_T, 0 <= H <= PCDF_MAX_H.
 * ------------------------------------------------------------------------- */
int pcdf_composite_workspace_bytes(const pcdf_grid *grid, int32_t T, int32_t H, const int32_t *caps,
                                   size_t *bytes);
int pcdf_build_predicted_composite(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf,
                                   int32_t T, int32_t H, const int32_t *caps, int32_t *comp_sq, float *comp_sdf,
                                   void *workspace, size_t workspace_bytes, void *stream);

/* The z-slab [zlo, zlo + S) of voxel slices that some capsule of some t
 * touches (S = 0: no capsule touches the grid).  The dynamic field's sites all
 * lie in it; the workspace holds one int32 per slab voxel per t and one
 * int32 per column (x, y): the largest static value of the column. */
int pcdf_composite_slab(const pcdf_grid *grid, int32_t T, int32_t H, const int32_t *caps, int32_t *zlo,
                        int32_t *S);

/* The two stages of pcdf_build_predicted_composite, for callers that want to
 * overlap or time them separately (same arguments and workspace; the
 * workspace carries the dynamic intermediate from the first to the second):
 *   prepare: the capsule row pass and y pass over the z-slab the capsules touch;
 *   finish:  the static column maxima, then the fused z pass, composite min
 *            and float epilogue for every t (where a column's largest static
 *            value is no larger than the humans' least 2-D partial, or a z lies
 *            far enough from the slab, the output is the static field without
 *            evaluating the humans' envelope). */
int pcdf_composite_prepare(const pcdf_grid *grid, int32_t T, int32_t H, const int32_t *caps, void *workspace,
                           size_t workspace_bytes, void *stream);
int pcdf_composite_finish(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf, int32_t T,
                          int32_t H, const int32_t *caps, int32_t *comp_sq, float *comp_sdf, void *workspace,
                          size_t workspace_bytes, void *stream);

/* The finish stage for the fields t = t0 .. t0 + nt - 1 only (0 <= t0,
 * nt >= 1, t0 + nt <= T): the outputs are the same [T][nz][ny][nx] arrays,
 * indexed by the absolute t, and only the range's fields are written.  A
 * caller can copy finished fields to the host while later ones are computed
 * (each call also recomputes the static column maxima). */
int pcdf_composite_finish_range(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf, int32_t T,
                                int32_t H, const int32_t *caps, int32_t t0, int32_t nt, int32_t *comp_sq,
                                float *comp_sdf, void *workspace, size_t workspace_bytes, void *stream);

/* One map update (Sec. 6, Sec. 8): the static field of occ and the T composite
 * fields, with the same results as pcdf_build_static_sdf (static_sq, and
 * static_sdf if non-NULL) followed by pcdf_build_predicted_composite, on two
 * streams of the same device: the capsules' x+y pass runs on side_stream
 * beside the static build on `stream`, and the composite's z stage on
 * `stream` once both are done.  side_stream first waits for the work already
 * on `stream`, and `stream` waits for side_stream's pass, so the call is
 * ordered on `stream` like a one-stream call (events between the streams;
 * nothing synchronises the host; capturable in a CUDA graph from `stream`).
 * workspace: pcdf_update_workspace_bytes(grid, T, H, caps) bytes, 256-byte
 * aligned (the static build's scratch, then the composite's). */
int pcdf_update_workspace_bytes(const pcdf_grid *grid, int32_t T, int32_t H, const int32_t *caps, size_t *bytes);
int pcdf_update_fields(const pcdf_grid *grid, const uint8_t *occ, int32_t T, int32_t H, const int32_t *caps,
                       int32_t *static_sq, float *static_sdf, int32_t *comp_sq, float *comp_sdf, void *workspace,
                       size_t workspace_bytes, void *stream, void *side_stream);

/* ---------------------------------------------------------------------------
 * From-scratch comparator (Sec. 6 benchmark: a full exact EDT per subsequent
 * field instead of the composition).
 *
 * For t = 0..T-1: sq[t] = signed squared EDT of (occ OR capsules at t).
 * Arguments as above; occ is the device occupancy of the static map.
 * ------------------------------------------------------------------------- */
int pcdf_scratch_workspace_bytes(const pcdf_grid *grid, int32_t T, int32_t H, size_t *bytes);
int pcdf_build_from_scratch(const pcdf_grid *grid, const uint8_t *occ, int32_t T, int32_t H, const int32_t *caps,
                            int32_t *sq, float *sdf, void *workspace, size_t workspace_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Translated primitive field (Sec. 6: the field of the human primitive is
 * computed once and composited at each tracked or predicted position).
 *
 * The template of a primitive cap (HOST int32 [7], fixed point as above,
 * capsule or cylinder) is the signed squared EDT of its voxels on a box: on
 * each axis the voxels whose centres 16 i + 8 lie in
 * [min(a, b) - r, max(a, b) + r], widened by R >= 0 voxels on every side.
 * Box voxel (i, j, k) is map voxel lo + (i, j, k) for the primitive where cap
 * puts it.
 *
 * pcdf_template_box: lo[3] and dims[3] (x, y, z) of that box (HOST outputs).
 *   PCDF_EINVAL if some axis holds no voxel centre of the primitive's range,
 *   a coordinate or radius is out of range, or a side exceeds PCDF_MAX_DIM.
 * pcdf_build_template: tmpl = device int32 [dz][dy][dx], the signed squared
 *   EDT of the primitive's voxels inside the box (interior voxels negative,
 *   +/-PCDF_INF where the opposite set is empty).  workspace: device,
 *   256-byte aligned, >= pcdf_template_workspace_bytes(cap, R).
 *
 * pcdf_composite_translated: for t = 0..T-1,
 *   comp[t](v) = min(static_sq(v), min_h P(v - lo[t][h]))
 * where P is the template inside its box and +INF outside, and lo is HOST
 * int32 [T][H][3], the map index (x, y, z) of the box's voxel 0 for primitive
 * h at t (the template's own lo plus an integer voxel move; each entry within
 * [-PCDF_MAX_DIM, PCDF_MAX_DIM]).  dims: HOST int32 [3], the template's box;
 * R: the widening the template was built with (0 <= 2 R < every side).  The
 * primitive's voxels lie in the box less R per side, so a voxel whose static
 * value is at most its squared gap to that inner box skips the template read
 * (same result: the template is at least that gap there).
 * static_sq, static_sdf, comp_sq and comp_sdf as for the composite above
 * (H = 0: every output is the static field).  No workspace.
 *
 * Exactness.  The output equals pcdf_build_predicted_composite of the moved
 * primitives wherever (1) the static value is at most R^2 or the voxel lies
 * inside every placed box (outside its box a primitive is more than R voxels
 * away), (2) each moved primitive and the free voxels next to it lie inside
 * the grid (the composite path counts in-grid voxels only), and (3) the
 * primitives of one t share no voxel and touch no face (otherwise their
 * interior values are the min over the primitives, not those of the union).
 * The translation is exact only for integer voxel moves; a primitive at a
 * sub-voxel position needs its own template.
 * ------------------------------------------------------------------------- */
/* pcdf_field_max: *out (device int32) = the largest value v of sq[0..n) with
 * 0 < v < PCDF_INF, or 0 if there is none; with R the least integer whose
 * square is at least that value, condition (1) above holds wherever the
 * static field is finite.  sq: device int32 [n]. */
int pcdf_field_max(const int32_t *sq, int64_t n, int32_t *out, void *stream);
/* pcdf_template_radius: *R (HOST) = the least integer R >= 0 with R * R >=
 * max_value, for max_value (>= 0) as pcdf_field_max returns it; with that R
 * the template covers every voxel whose static value is finite (condition (1)
 * above).  PCDF_EINVAL for a negative max_value or a NULL R. */
int pcdf_template_radius(int32_t max_value, int32_t *R);
/* pcdf_lattice_placements: the box placements lo (HOST int32 [T][H][3]) of
 * primitives caps (HOST int32 [T][H][7]) that are all ref_cap (HOST int32 [7],
 * whose template box starts at ref_lo, HOST int32 [3]) moved by whole voxels:
 * lo[t][h] = ref_lo + (a[t][h] - a_ref) / 16 per axis.  PCDF_EINVAL (nothing
 * written) if some primitive has another radius or axis, a move that is not a
 * multiple of 16 (one voxel), or a placement outside [-PCDF_MAX_DIM,
 * PCDF_MAX_DIM]. */
int pcdf_lattice_placements(const int32_t *caps, int32_t T, int32_t H, const int32_t *ref_cap, const int32_t *ref_lo,
                            int32_t *lo);
int pcdf_template_box(const int32_t *cap, int32_t R, int32_t *lo, int32_t *dims);
int pcdf_template_workspace_bytes(const int32_t *cap, int32_t R, size_t *bytes);
int pcdf_build_template(const int32_t *cap, int32_t R, int32_t *tmpl, void *workspace, size_t workspace_bytes,
                        void *stream);
int pcdf_composite_translated(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf, int32_t T,
                              int32_t H, const int32_t *tmpl, const int32_t *dims, int32_t R, const int32_t *lo,
                              int32_t *comp_sq, float *comp_sdf, void *stream);

/* ---------------------------------------------------------------------------
 * Hinge obstacle cost at body spheres (Sec. 7 hinge form, GPMP2 obstacle
 * factor; Sec. 8 field assignment).
 *
 * For sphere q with centre c and radius r (spheres device fp32 [N][4],
 * 16-byte aligned) and time index s = tidx[q] (device int32 [N]):
 *   t = clamp(s, 0, T-1);
 *   per axis u = (c - origin) / vox - 1/2 in fp32, clamped to [0, n-1]
 *   (NaN -> 0), lower corner i0 = min(floor(u), n-2) (0 if n == 1);
 *   d = trilinear interpolation of sdf[t] (device fp32 [T][nz][ny][nx]), lerped
 *   along x, then y, then z; any -inf corner gives d = -inf, else any +inf
 *   corner gives d = +inf;
 *   h[q] = max(0, eps + r - d)  (device fp32 [N], out).
 * n_oob: device int32 or NULL; if given, the number of spheres clamped on some
 * axis is ADDED to *n_oob (the caller zeroes it).
 * N may be 0 (nothing is launched).
 * ------------------------------------------------------------------------- */
int pcdf_query_cost(const pcdf_grid *grid, const float *sdf, int32_t T, const float *spheres, const int32_t *tidx,
                    int64_t N, float eps, float *h, int32_t *n_oob, void *stream);

/* Backward of pcdf_query_cost: with the same inputs and upstream gradient
 * grad_h (device fp32 [N]),
 *   grad_c[q] = -grad_h[q] * grad_c d(c)   where h > 0 and d is finite, else 0
 *   (device fp32 [N][3], out; the gradient of d is the analytic derivative of
 *   the trilinear interpolant divided by vox, zero along clamped or
 *   single-voxel axes);
 *   grad_r[q] = grad_h[q] * [h > 0 and d finite]  (device fp32 [N] or NULL). */
int pcdf_query_cost_backward(const pcdf_grid *grid, const float *sdf, int32_t T, const float *spheres,
                             const int32_t *tidx, int64_t N, float eps, const float *grad_h, float *grad_c,
                             float *grad_r, void *stream);

/* ---------------------------------------------------------------------------
 * Batched environments in one persistent launch (an extension beyond the
 * paper: many maps of uneven size, horizon and human count updated together).
 *
 * For every environment e: the static signed squared EDT of occ (as
 * pcdf_build_static_sdf) and its T composite fields comp_sq[t] (as
 * pcdf_build_predicted_composite), int32 only.  Results are bit-identical to
 * the per-environment calls and independent of the tile shapes.
 *
 * pcdf_batch_create   builds the host-side plan (work items, capsule tables,
 *                     workspace layout); allocates host memory only; reads
 *                     each environment's HOST capsules; needs the current
 *                     device to query occupancy.
 * pcdf_batch_upload   copies the plan into the workspace (host-to-device
 *                     copies on `stream`; not capturable; repeat it whenever
 *                     the workspace or the environments' device pointers
 *                     change).
 * pcdf_batch_run      resets the counters and launches the persistent kernel:
 *                     no host synchronisation, capturable in a CUDA graph.
 * pcdf_batch_error    synchronises `stream` and reports PCDF_ETIMEOUT if a
 *                     dependency wait inside the last run timed out (then the
 *                     outputs are not valid), else PCDF_OK.
 * pcdf_batch_autotune times every candidate tile shape (rows per row-pass
 *                     item, slab slices per capsule item, time steps per
 *                     composite item) with `reps` runs each, synchronising
 *                     `stream`, and returns the fastest; the workspace must
 *                     hold pcdf_batch_autotune_workspace_bytes().
 * ------------------------------------------------------------------------- */
typedef struct pcdf_env {
    pcdf_grid grid;
    int32_t T, H;
    const int32_t *caps; /* HOST [T][H][7]; NULL iff H == 0 */
    const uint8_t *occ;  /* device [nz][ny][nx] */
    int32_t *comp_sq;    /* device [T][nz][ny][nx], out */
} pcdf_env;

typedef struct pcdf_batch_tiles {
    int32_t row_rows;   /* rows per row-pass item (<= 0: 32) */
    int32_t dyn_slices; /* slab slices per capsule-field item (<= 0: 1) */
    int32_t comp_t;     /* time steps per composite item (<= 0: 1) */
} pcdf_batch_tiles;

typedef struct pcdf_batch pcdf_batch;

int pcdf_batch_create(const pcdf_env *envs, int32_t n_env, const pcdf_batch_tiles *tiles, pcdf_batch **out);
void pcdf_batch_destroy(pcdf_batch *batch);
int pcdf_batch_workspace_bytes(const pcdf_batch *batch, size_t *bytes);
int pcdf_batch_tiles_used(const pcdf_batch *batch, pcdf_batch_tiles *tiles);
int pcdf_batch_upload(pcdf_batch *batch, void *workspace, size_t workspace_bytes, void *stream);
int pcdf_batch_run(const pcdf_batch *batch, void *workspace, void *stream);
int pcdf_batch_error(const pcdf_batch *batch, const void *workspace, void *stream, int32_t *code);
/* pcdf_batch_block_stage  testing aid for the failure path: raises the
 * completion target of one stage (0 rows, 1 y pass, 2 z pass) of environment
 * `env` above any item count, so that the items that wait on it (the y, z
 * and first-launch items after it) can only give up when their bounded wait
 * (about a second) expires.  After the first expiry every later wait gives
 * up at once, so no item reads unfinished inputs: the waiting items are
 * skipped, the second launch (the composite items) skips everything,
 * pcdf_batch_error then reports PCDF_ETIMEOUT, and the outputs of the run
 * are not valid.  The capsule stage (3) has no waiter in the first launch and
 * is refused (PCDF_EINVAL).  Takes effect at the next pcdf_batch_upload; a
 * new batch starts unblocked. */
int pcdf_batch_block_stage(pcdf_batch *batch, int32_t env, int32_t stage);
int pcdf_batch_autotune_workspace_bytes(const pcdf_env *envs, int32_t n_env, size_t *bytes);
int pcdf_batch_autotune(const pcdf_env *envs, int32_t n_env, void *workspace, size_t workspace_bytes, void *stream,
                        int32_t reps, pcdf_batch_tiles *best, float *best_ms);

/* ---------------------------------------------------------------------------
 * Context: the handle of the paper's interface (a device, a stream and scratch
 * that the library owns), over the workspace calls above.
 *
 * pcdf_create         binds a context to `device` (0 <= device < the device
 *                     count; PCDF_EINVAL otherwise) and `stream` (a
 *                     cudaStream_t of that device, NULL: the legacy default
 *                     stream); allocates nothing on the device.
 * pcdf_destroy        releases the scratch (stream-ordered on the context's
 *                     stream) and the handle; NULL is ignored.
 * pcdf_scratch_bytes  an upper bound of the scratch any call of a context
 *                     needs for `grid` with up to T fields and H humans (the
 *                     composite bound assumes capsules touching every slice);
 *                     host only.
 * pcdf_ctx_reserve    grows the scratch to at least `bytes` now (for example
 *                     to pcdf_scratch_bytes at start-up), so that later calls
 *                     allocate nothing.
 * pcdf_ctx_*          the workspace call of the same name (same arguments,
 *                     results and checks) on the context's device and stream
 *                     with the context's scratch.  When the scratch is smaller
 *                     than the call needs, it is released and reallocated
 *                     first (cudaFreeAsync / cudaMallocAsync on the context's
 *                     stream; PCDF_ENOMEM if that fails).  The calls are
 *                     asynchronous; calls sharing a context must share its
 *                     stream order (one thread at a time).
 * pcdf_build_batched  the batched environments (pcdf_batch_* with the default
 *                     tiles): plans, uploads into the scratch and runs them,
 *                     the run as a CUDA graph when use_graph is 1 (0: plain
 *                     launches; other values PCDF_EINVAL); synchronises the
 *                     context's stream and returns PCDF_ETIMEOUT if a
 *                     dependency wait inside the run expired.
 * ------------------------------------------------------------------------- */
typedef struct pcdf_ctx pcdf_ctx;
int pcdf_create(pcdf_ctx **out, int32_t device, void *stream);
void pcdf_destroy(pcdf_ctx *ctx);
int pcdf_scratch_bytes(const pcdf_grid *grid, int32_t T, int32_t H, size_t *bytes);
int pcdf_ctx_reserve(pcdf_ctx *ctx, size_t bytes);
int pcdf_ctx_build_static_sdf(pcdf_ctx *ctx, const pcdf_grid *grid, const uint8_t *occ, int32_t *static_sq,
                              float *static_sdf);
int pcdf_ctx_build_predicted_composite(pcdf_ctx *ctx, const pcdf_grid *grid, const int32_t *static_sq,
                                       const float *static_sdf, int32_t T, int32_t H, const int32_t *caps,
                                       int32_t *comp_sq, float *comp_sdf);
int pcdf_ctx_build_from_scratch(pcdf_ctx *ctx, const pcdf_grid *grid, const uint8_t *occ, int32_t T, int32_t H,
                                const int32_t *caps, int32_t *sq, float *sdf);
int pcdf_ctx_query_cost(pcdf_ctx *ctx, const pcdf_grid *grid, const float *sdf, int32_t T, const float *spheres,
                        const int32_t *tidx, int64_t N, float eps, float *h, int32_t *n_oob);
int pcdf_ctx_query_cost_backward(pcdf_ctx *ctx, const pcdf_grid *grid, const float *sdf, int32_t T,
                                 const float *spheres, const int32_t *tidx, int64_t N, float eps, const float *grad_h,
                                 float *grad_c, float *grad_r);
int pcdf_build_batched(pcdf_ctx *ctx, const pcdf_env *envs, int32_t n_env, int32_t use_graph);

/* ---------------------------------------------------------------------------
 * Learned surrogate of the dynamic field: a BF16 MLP with FP32 accumulation
 * (an extension beyond the paper).  16 inputs (PCDF_MLP_IN features, then
 * zero pads; the weights of the pad inputs stay zero) -> 256 -> 256 -> 256 -> 1, ReLU after the hidden layers.
 *
 * State: one device buffer of pcdf_mlp_state_bytes(), 256-byte aligned,
 * holding the FP32 parameter vector, the two Adam moments and the gradient
 * (each PCDF_MLP_PARAMS_PAD floats, in that order), then the BF16 copies of the
 * weight matrices (PCDF_MLP_BF16_WEIGHTS values).  Parameter vector order:
 * W1 [256][16], b1 [256], W2 [256][256], b2, W3 [256][256], b3, w4 [256], b4;
 * the BF16 copies hold W1, W2, W3, w4 in the same layouts.  Layer l computes
 * relu(x W_l^T + b_l); activations and input gradients are stored in BF16.
 *
 * x: device BF16 bits [M][16] (16-byte aligned); y, target: device FP32 [M].
 * The three padding columns of x (after the PCDF_MLP_IN features) are
 * ignored: the kernels put 1 there and the first layer's bias in the matching
 * columns of W1.
 *
 * All passes run on the 5th-generation tensor cores (tcgen05.mma, BF16
 * operands in shared memory, FP32 accumulators in tensor memory) in
 * persistent warp-specialised kernels over 128-row tiles.  A bounded wait on
 * the tensor cores or the copies that expires (about a second) gives NaN: in
 * y for the tiles concerned, in the loss and in the gradient of b4.
 *
 * pcdf_mlp_forward  y and the hidden activations, stored in the workspace.
 * pcdf_mlp_backward  one training step's products: the forward pass (y), the
 * loss mean((y - t)^2) (written to *loss if non-NULL) and the gradient
 * (overwritten).  With dy = 2 (y - t) / M (FP32), D3 = dy * w4 where H3 > 0
 * (FP32 product rounded to BF16), D_l = D_{l+1} W_{l+1} where H_l > 0 (FP32
 * sum rounded to BF16), grad W_l = D_l^T H_{l-1} (H_0 = x) and grad b_l = the
 * column sums of D_l (FP32 sums in an unspecified order: atomics).  D3 is
 * rebuilt on chip from dy and the mask of H3 wherever it is used.
 *
 * Workspace: pcdf_mlp_workspace_bytes(M), 256-byte aligned.  For T = ceil(M /
 * 128) tiles it holds, in this order: H1, H2, H3, D2, D1 (T x 65536 bytes
 * each: H_l = relu(Z_l), D_l = dL/dZ_l, BF16), the x tiles as multiplied (T x
 * 4096 bytes), the ReLU masks of H1, H2, H3 (T x 4096 bytes each) and dy (T x
 * 128 FP32, 0 past M).  A tile is stored in the tensor-core operand layout:
 * element (m, k) of an [M][256] matrix at byte 65536 (m / 128) + 4096 ((m %
 * 128) / 8) + 128 (k / 8) + 16 (m % 8) + 2 (k % 8); of x, 4096 (m / 128) +
 * 256 ((m % 128) / 8) + 128 (k / 8) + 16 (m % 8) + 2 (k % 8).  Mask word (t,
 * j, r) at 4 (1024 t + 128 j + r) of its section holds the flags H_l(128 t +
 * r, k) > 0 of the 32 columns k = 32 j + 8 g + c: byte g, bit c / 2 for even
 * c and bit 4 + (c - 1) / 2 for odd c (a NaN activation counts as > 0).  Rows
 * past M in the last tile hold the network of zero features (H) and zeros
 * (D).  pcdf_mlp_forward stores H1, H2, H3, the x tiles and the masks of H1
 * and H2; pcdf_mlp_backward stores H1, H2, D2, D1, the x tiles, the three
 * masks and dy (H3 is left as it was).
 * pcdf_mlp_adam applies one Adam step (bias-corrected, step >= 1) to the FP32
 * parameters and refreshes the BF16 copies.
 * ------------------------------------------------------------------------- */
#define PCDF_MLP_IN 13
#define PCDF_MLP_IN_PAD 16
#define PCDF_MLP_WIDTH 256
#define PCDF_MLP_PARAMS 136193
#define PCDF_MLP_PARAMS_PAD 136196
#define PCDF_MLP_BF16_WEIGHTS 135424

int pcdf_mlp_state_bytes(size_t *bytes);
int pcdf_mlp_workspace_bytes(int64_t M, size_t *bytes);
int pcdf_mlp_init(void *state, uint64_t seed, void *stream);
int pcdf_mlp_forward(const void *state, const uint16_t *x, int64_t M, float *y, void *workspace,
                     size_t workspace_bytes, void *stream);
/* pcdf_mlp_infer  y = network(x) for M rows in one fused launch (no
 * workspace) on the legacy mma.sync tensor-core path, kept as the baseline:
 * each CTA keeps a 64-row tile's activations in shared memory and streams the
 * hidden weights.  Same arithmetic as the tcgen05 passes up to the order of
 * the FP32 sums (y within FP32 rounding of theirs, not bit-identical).  x
 * device BF16 bits [M][16] (16-byte aligned), y device fp32 [M]. */
int pcdf_mlp_infer(const void *state, const uint16_t *x, int64_t M, float *y, void *stream);

/* pcdf_mlp_infer_tc  y alone, with no workspace: a persistent kernel (one
 * CTA per SM) walks 128-row tiles; one thread issues tcgen05.mma, a producer
 * warp streams the x tiles and the hidden weights (bulk copies from a packed
 * copy in the state that pcdf_mlp_init and pcdf_mlp_adam keep current; the
 * state is only read here), and eight epilogue warps read each layer back
 * with tcgen05.ld for the bias, ReLU and BF16 rounding, overlapping the next
 * layer's products.  The same kernel, products and rounding as
 * pcdf_mlp_forward and pcdf_mlp_backward: y is bit-identical to theirs. */
int pcdf_mlp_infer_tc(const void *state, const uint16_t *x, int64_t M, float *y, void *stream);
/* pcdf_mlp_infer_tc_count  pcdf_mlp_infer_tc over the first *count rows of x
 * (count: device int32, read by the kernel, clamped to [0, M_max]), so that
 * a row count produced on the device (pcdf_surrogate_select) needs no host
 * round trip; x and y hold M_max rows, y past the count is left unwritten. */
int pcdf_mlp_infer_tc_count(const void *state, const uint16_t *x, int64_t M_max, const int32_t *count, float *y,
                            void *stream);
int pcdf_mlp_backward(void *state, const uint16_t *x, const float *target, int64_t M, float *y, float *loss,
                      void *workspace, size_t workspace_bytes, void *stream);
int pcdf_mlp_adam(void *state, float lr, float beta1, float beta2, float eps, int32_t step, void *stream);

/* ---------------------------------------------------------------------------
 * Surrogate queries (an extension beyond the paper).
 *
 * Features of a point p (metres) at time index t of a horizon T for one
 * capsule (a, b, r): two zeros; the height of p above the grid floor in
 * units of 2 m; 2 t / (T - 1) - 1 (0 if T == 1); p - a and p - b in units of
 * 2 m; r in units of 2 m; the continuous signed distance |p - n| - r from p to
 * the capsule (n the nearest axis point) in units of 2 m; the axis parameter
 * of n scaled to [-1, 1]; three zeros.  (The capsule enters relative to the
 * point and only the floor fixes a position, so a network trained in one
 * grid serves any grid of the same voxel size; the network learns the exact
 * voxel field's departure from the continuous distance.)
 *
 * pcdf_surrogate_samples  M training rows from exact dynamic fields
 *     fields  device fp32 [n_fields][nz][ny][nx] (float fields of one capsule
 *             each, e.g. composites with an empty static map);
 *     caps    device int32 [n_fields][7], tf device int32 [n_fields] (time
 *             index of each field for the t feature, horizon T);
 *     point i: with probability `near` within 1 m of the capsule axis, else
 *     uniform in the grid; a counter hash of (seed, i) draws it;
 *     x out device BF16 bits [M][16]; target out device fp32 [M]: the
 *     trilinear value of the field at the point minus the continuous signed
 *     distance from the point to the capsule (the network learns that
 *     departure).
 * pcdf_surrogate_features  rows (q * H + h) for sphere q and capsule h of time
 *     clamp(tidx[q], 0, T - 1); caps device int32 [T][H][7]; x out [N * H][16].
 * pcdf_surrogate_finish  from the network outputs y [N * H] (device fp32):
 *     with D_h = continuous signed distance to capsule h + y[q * H + h],
 *     d = trilinear over the query's cell of min(static corner value,
 *     min_h (D_h + u_h . (corner - p))), u_h the unit vector from
 *     capsule h's nearest axis point to p (the dynamic value extrapolated to
 *     the corners along its distance gradient); rows with y_index -1 count as
 *     +INF.  With bounds (device fp32 [N][2] from pcdf_surrogate_select,
 *     8-byte aligned): d is clamped to [d_lo, d_hi], and a query is answered
 *     exactly when its decision is not certain (d_lo < eps + r <= d_hi) or
 *     when it is certainly active (d_hi < eps + r), has a network row and
 *     |d - (eps + r)| < band; every other decision (h > 0 or not) is the
 *     exact path's by construction.  With bounds NULL (to measure the
 *     network): a query with a network row is answered exactly when
 *     |d - (eps + r)| < band.  Exact answers take the corner voxels of the
 *     cell from static_sq and an exact local search over the capsules'
 *     voxels, interpolated like pcdf_query_cost (same bits as the exact
 *     composite path); h[q] = max(0, eps + r - d) (device fp32 [N]), d_out
 *     (nullable) the distance used; n_fallback (device int32, nullable) the
 *     number of exact answers.  caps_host: HOST int32 [T][H][7].  Workspace:
 *     pcdf_surrogate_finish_workspace_bytes(T, H, N).
 * ------------------------------------------------------------------------- */
int pcdf_surrogate_samples(const pcdf_grid *grid, const float *fields, const int32_t *caps, const int32_t *tf,
                           int32_t n_fields, int32_t T, int64_t M, uint64_t seed, float near, uint16_t *x,
                           float *target, void *stream);
int pcdf_surrogate_features(const pcdf_grid *grid, const float *spheres, const int32_t *tidx, int64_t N, int32_t T,
                            int32_t H, const int32_t *caps, uint16_t *x, void *stream);
int pcdf_surrogate_finish_workspace_bytes(int32_t T, int32_t H, int64_t N, size_t *bytes);
int pcdf_surrogate_finish(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf,
                          const float *spheres, const int32_t *tidx, int64_t N, int32_t T, int32_t H,
                          const int32_t *caps_host, const float *y, const int32_t *y_index, const float *bounds,
                          float eps, float band, float *h, float *d_out, int32_t *n_fallback, void *workspace,
                          size_t workspace_bytes, void *stream);

/* pcdf_surrogate_finish_slab  the same, with the exact answers taken from the
 * 2-D partial field of the capsule slab that pcdf_composite_prepare left in
 * comp_workspace (prepare run on the same grid, T, H and caps, earlier on the
 * stream; comp_workspace_bytes >= pcdf_composite_workspace_bytes): each
 * corner's dynamic value is the minimum over its column's slab sites, the
 * integers the composite z pass produces, at a few loads per corner instead
 * of a search over the capsules' voxels.
 * Both finish calls, pcdf_surrogate_select and pcdf_mlp_infer_tc_count make
 * no host synchronisation and copy nothing from host memory (the capsules
 * reach the device as kernel parameters), so a plan step of
 * pcdf_composite_prepare, select, inference and finish can be captured in a
 * CUDA graph and replayed on new sphere contents. */
int pcdf_surrogate_finish_slab(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf,
                               const float *spheres, const int32_t *tidx, int64_t N, int32_t T, int32_t H,
                               const int32_t *caps_host, const void *comp_workspace, size_t comp_workspace_bytes,
                               const float *y, const int32_t *y_index, const float *bounds, float eps, float band,
                               float *h, float *d_out, int32_t *n_fallback, void *workspace, size_t workspace_bytes,
                               void *stream);

/* pcdf_surrogate_select  the certificate of every query and the rows the
 * network must answer.  Query q: sphere (p, r) at time t = clamp(tidx[q], 0,
 * T - 1), capsules caps DEVICE int32 [T][H][7] (H <= 64).  bounds[q] (device
 * fp32 [N][2], 8-byte aligned, out) = (d_lo, d_hi) with d_lo <= d <= d_hi
 * for the exact composite path's distance d, from:
 *   - the exact static corner values of the query's cell (static_sdf);
 *   - at a corner outside capsule h (continuous signed distance D > 0 from
 *     the voxel centre), the exact field of the capsule's voxels lies in
 *     [D, D + sqrt(3) vox] (the lower end always; the upper end when
 *     r >= 14/16 voxel and the capsule lies inside the grid, else +inf);
 *     inside it (D <= 0) it is at most D (no lower end);
 *   - the humans' field is the min over the capsules outside them and at
 *     most that min inside them; the composite is min(static, humans) and
 *     the trilinear weights are non-negative;
 *   - a margin of 1e-4 m on each side for FP32 rounding.
 * Row i = q * H + h needs the network if capsule h can lie below the static
 * field at some corner (its lower end is below the static value there) and,
 * with mode 0, if the query is certainly active (d_hi < eps + r), the only
 * queries whose cost uses the network's value; mode 1 keeps every row where
 * the capsule can matter (to measure the network).  Kept rows get their
 * features in x (BF16 bits [<= N * H][16]) at slot y_index[i] (device int32
 * [N * H]; -1 for a skipped row), slots taken in an unspecified order;
 * *count (device int32) receives the number kept.  The network runs on
 * x[0 .. *count) and pcdf_surrogate_finish(_slab) reads its output through
 * y_index (a NULL y_index there means y holds every row in order). */
int pcdf_surrogate_select(const pcdf_grid *grid, const float *static_sdf, const float *spheres, const int32_t *tidx,
                          int64_t N, int32_t T, int32_t H, const int32_t *caps, float eps, int32_t mode, uint16_t *x,
                          int32_t *y_index, int32_t *count, float *bounds, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PCDF_H */

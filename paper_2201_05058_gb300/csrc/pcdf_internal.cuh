// Internal declarations shared by the CUDA translation units of libpcdf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pcdf.h"

// ---------------------------------------------------------------------------
// Bounds checks (debug build).  Compiled with PCDF_CHECK_BOUNDS (and
// relocatable device code, so that every file shares one error word), the
// kernels of the hot path test each global and shared index before the
// access: PCDF_IN(i, n) is false when i lies outside [0, n), and then records
// the first failing check (a 16-bit hash of its file name, its line) and a
// count in g_bounds_error, and the access is skipped; nothing traps.  In the
// normal build PCDF_IN is the constant true and costs nothing.
// ---------------------------------------------------------------------------
namespace pcdf {

__host__ __device__ constexpr unsigned file_tag(const char *s, const char *base = nullptr, unsigned h = 5381)
{
    // djb2 hash of the part after the last '/'
    return !base ? file_tag(s, s, h)
                 : (*s == 0 ? (h & 0xffffu)
                            : (*s == '/' ? file_tag(s + 1, s + 1, 5381) : file_tag(s + 1, base, h * 33u + (unsigned char)*s)));
}

template <unsigned V>
struct TagConst {
    static constexpr unsigned value = V;
};

#ifdef PCDF_CHECK_BOUNDS
extern __device__ unsigned int g_bounds_error[2];  // [0] first failing check: tag << 16 | line; [1] count
__host__ __device__ __forceinline__ bool bounds_ok(long long i, long long n, unsigned code)
{
    if (i >= 0 && i < n)
        return true;
#ifdef __CUDA_ARCH__
    atomicCAS(&g_bounds_error[0], 0u, code);
    atomicAdd(&g_bounds_error[1], 1u);
#else
    (void)code;
#endif
    return false;
}
#define PCDF_IN(i, n)                                                                                               \
    (::pcdf::bounds_ok((long long)(i), (long long)(n),                                                             \
                       (::pcdf::TagConst<::pcdf::file_tag(__FILE__)>::value << 16) | (unsigned)__LINE__))
#else
#define PCDF_IN(i, n) true
#endif

}  // namespace pcdf

namespace pcdf {

// 1-D distances along x are stored as int16 with the sign of the voxel's own
// state (+ free, - occupied) and magnitude = distance to the nearest voxel of
// the other state on the row; kInf16 marks "none on this row".
constexpr int16_t kInf16 = 0x7FFF;
constexpr int32_t kInf32 = PCDF_INF;

// One capsule with its voxel-index bounding box, clipped to the grid (lo > hi
// on some axis when the capsule covers no voxel centre of the grid).
struct alignas(16) CapInfo {
    int32_t a[3];
    int32_t b[3];
    int32_t r;
    int32_t lo[3];
    int32_t hi[3];
    int32_t cyl;     // finite cylinder (flat ends) instead of a capsule
    int32_t pad[2];
};
static_assert(sizeof(CapInfo) == 64, "CapInfo layout");

// Capsules handed to one row-pass launch by value (kernel parameters are
// copied at launch, so the host array may be reused as soon as the call
// returns and nothing has to be staged in device memory).
constexpr int kMaxCapsPerLaunch = 384;
struct CapBatch {
    int32_t count;
    int32_t pad[3];
    CapInfo caps[kMaxCapsPerLaunch];
};

// Slab slices of equal capsule cross-sections: rep[t * S + e] is the first
// slab slice of time t whose voxel set in every capsule equals slice e's
// (upright capsules: every slice between the caps; cap slices at the same
// distance from their cap centres).  Only those slices are computed, and
// every reader of the slab partials goes through the map.  A kernel
// parameter like CapBatch; on = 0: the identity.
constexpr int kSlabMapMax = 4096;
struct SlabMap {
    int32_t on;
    int32_t S;
    uint8_t rep[kSlabMapMax];
};

// Columns handled by one CTA of the lower-envelope pass (the CTA has two
// threads per column, one per site set).
constexpr int kEnvCols = 32;

// ---------------------------------------------------------------------------
// launchers (edt.cu); all return cudaError_t of the launch
// ---------------------------------------------------------------------------

// Row pass along x.  Rows of slices z = z0 .. z0 + nslices - 1; for every t in
// [0, n_t) the output block t is g16 + t * nslices * ny * nx and the capsules
// of that t are caps->caps[t * H .. t * H + H - 1].
//   mode 0: occupancy only (occ is indexed by absolute z; caps unused)
//   mode 1: occupancy OR capsules
//   mode 2: capsules only
cudaError_t launch_pass_x(int mode, const uint8_t *occ, const CapBatch *caps, int H, int nx, int ny, int z0,
                          int nslices, int n_t, int16_t *g16, cudaStream_t stream);

// Exact signed EDT of a whole grid (edt_full.cu): row bits of the occupancy
// (mode 0), of the occupancy OR the capsules caps->caps[0 .. H) (mode 1) or of
// the capsules alone (mode 2), then the fused x+y pass and the z pass; sq and
// (nullable) sdf are [nz][ny][nx].  ws holds full_edt_scratch() bytes
// (256-byte aligned): row words, their carries and the 2-D partial field.
// colmax (nullable): receives the largest value of every column of sq, as
// launch_colmax would write it.
size_t full_edt_scratch(int nx, int ny, int nz, size_t *bits_off, size_t *carry_off, size_t *mid_off);
cudaError_t launch_full_edt(int mode, const uint8_t *occ, const CapBatch *caps, int H, int nx, int ny, int nz,
                            int32_t *sq, float *sdf, float vox, void *ws, cudaStream_t stream,
                            int32_t *colmax = nullptr);

// Lower-envelope pass over ncols columns: element e of column c lives at
// (c / nx) * outer_stride + (c % nx) + e * stride, e in [0, n).
cudaError_t launch_envelope_i16(const int16_t *in, int32_t *out, int n, int nx, long long ncols,
                                long long outer_stride, long long stride, cudaStream_t stream);

// Analytic x+y passes of the capsule field over the slab slices zlo .. zlo+S-1
// for t = t0 .. t0 + n_t - 1 (capsules of local t at caps->caps[t * H ...]);
// output dyn_mid[t][s][y][x], signed 2-D partial squared distances.  `cap` is
// the per-thread stack capacity; dyn_xy_fits tells whether it fits on chip.
bool dyn_xy_fits(int ny, int H, int cap);
cudaError_t launch_dyn_xy(const CapBatch *caps, const SlabMap *map, int H, int nx, int ny, int zlo, int S, int t0,
                          int n_t, int cap,
                          int32_t *dyn_mid, cudaStream_t stream);

// colmax[y][x] = largest value of the column (x, y) of sq [nz][ny][nx].
cudaError_t launch_colmax(const int32_t *sq, int nx, int ny, int nz, int32_t *colmax, cudaStream_t stream);

// z-pass of the dynamic field over the slab [zlo, zlo + S) fused with the
// composite min against static_sq and the float epilogue, for t = t0 ..
// t0 + nt - 1 (outputs and slab indexed by the absolute t).
// static_sdf (nullable) is the float field of static_sq; where the static
// field wins the min it is copied instead of recomputed.  colmax holds the
// column maxima of static_sq (launch_colmax): columns and z ranges where the
// static field provably wins skip the envelope.
cudaError_t launch_composite_z(const int32_t *static_sq, const float *static_sdf, const int32_t *colmax,
                               const int32_t *dyn_mid, const SlabMap *map, int nx, int ny, int nz, int zlo, int S,
                               int t0, int nt, int32_t *comp_sq, float *comp_sdf, float vox, cudaStream_t stream);

// Copies static_sq into t = t0 .. t0 + nt - 1 of comp (and its float field)
// when no capsule touches the grid.
cudaError_t launch_broadcast_static(const int32_t *static_sq, long long V, int t0, int nt, int32_t *comp_sq,
                                    float *comp_sdf, float vox, cudaStream_t stream);

// query.cu
struct QueryGrid {
    int n[3];
    float origin[3];
    float vox;
};
cudaError_t launch_query_cost(const QueryGrid &g, const float *sdf, int T, const float4 *spheres,
                              const int32_t *tidx, long long N, float eps, float *h, int32_t *n_oob,
                              cudaStream_t stream);
cudaError_t launch_query_cost_backward(const QueryGrid &g, const float *sdf, int T, const float4 *spheres,
                                       const int32_t *tidx, long long N, float eps, const float *grad_h,
                                       float *grad_c, float *grad_r, cudaStream_t stream);

}  // namespace pcdf

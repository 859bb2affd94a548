// Translated primitive field (Sec. 6): the field of one human primitive is
// computed once, as the exact signed EDT of its voxels on a box around it, and
// composited with the static field at every predicted position by the same
// per-voxel min as the composite path.  A position is an integer voxel offset
// of the box (the translation is exact only on the lattice), so an output
// voxel reads the template at its own index minus the box's placement.
//
// Box: on each axis the voxels whose centres 16 i + 8 lie in
// [min(a, b) - r, max(a, b) + r] (fixed point), widened by R voxels on every
// side.  Outside the box the primitive's field is taken as +INF; it is in fact
// larger than R^2 there, so wherever the static value is at most R^2 the
// output is the exact composite.
//
// k_composite_translated: each warp owns kTrRowIters output rows (y, z) of
// one t, lanes over x in 16-byte groups of 4 voxels (two groups per lane in
// flight); each CTA owns a block of rows and the T CTAs of a row block are
// adjacent, so the static rows come from DRAM once (prefetched into L2 by
// those CTAs together).  The boxes that cross a row are found from the
// placements alone (kernel parameters), so rows outside every box are plain
// copies of the static row.
#include <cuda_runtime.h>

#include <cmath>

#include <algorithm>
#include <cstring>
#include <vector>

#include "edt_common.cuh"
#include "host.h"

namespace pcdf {
namespace {

constexpr int kTrWarps = 8;        // warps (rows in flight) per CTA
constexpr int kTrRowIters = 8;     // rows per warp: a CTA owns kTrWarps * kTrRowIters rows
constexpr int kMaxPlacements = 1536;

// Box placements of one launch: place[lt * H + h] = (x, y, z) map index of the
// box's voxel 0 for local time lt and primitive h.  Passed by value.
struct TmplPlacement {
    int4 place[kMaxPlacements];
};

// The template's value at the W voxels from (x, y, z) on, for the boxes that
// reach them, min'ed into d; a voxel whose static value sv is no larger than
// its squared gap to a box's inner box (the template box less R per side,
// which holds every voxel of the primitive) skips that box: the template is
// at least the gap there, so the static value wins either way.
template <int W>
__device__ __forceinline__ void template_min(int x, int y, int z, const int32_t *sv,
                                             const int32_t *__restrict__ tmpl, int dx, int dy, int dz, int R,
                                             const int4 *pl, int H, int32_t *d)
{
    int32_t smax = sv[0];
#pragma unroll
    for (int i = 1; i < W; ++i)
        smax = max(smax, sv[i]);
    for (int h = 0; h < H; ++h) {
        const int4 p = pl[h];
        const int j = y - p.y, k = z - p.z;
        if ((unsigned)j >= (unsigned)dy || (unsigned)k >= (unsigned)dz)
            continue;
        const int u0 = x - p.x;
        if (u0 + W <= 0 || u0 >= dx)
            continue;  // the group lies beside the box
        const int gy = max(0, max(R - j, j - (dy - 1 - R)));
        const int gz = max(0, max(R - k, k - (dz - 1 - R)));
        const int gyz = gy * gy + gz * gz;
        // the group's least gap (its voxel nearest the inner box) bounds all W
        const int gx0 = max(0, max(R - (u0 + W - 1), u0 - (dx - 1 - R)));
        const int lb0 = gx0 * gx0 + gyz;
        if (lb0 > 0 && smax <= lb0)
            continue;
        const int32_t *trow = tmpl + ((long long)k * dy + j) * dx;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const int u = u0 + i;
            if ((unsigned)u >= (unsigned)dx)
                continue;
            const int gx = max(0, max(R - u, u - (dx - 1 - R)));
            const int lb = gx * gx + gyz;
            if (lb > 0 && sv[i] <= lb)
                continue;
            d[i] = min(d[i], __ldg(trow + u));
        }
    }
}

// W voxels from (x, y, z): the static values come in with the call; the
// template is min'ed in and both outputs are stored.
template <bool kSq, bool kSdfOut, bool kStaticSdf, int W>
__device__ __forceinline__ void translated_finish(int x, int y, int z, int off, const int32_t *sv, const float *sf,
                                                  const int32_t *__restrict__ tmpl, int dx, int dy, int dz, int R,
                                                  const int4 *pl, int H, int32_t *__restrict__ oq,
                                                  float *__restrict__ of, float vox)
{
    int32_t d[W];
#pragma unroll
    for (int i = 0; i < W; ++i)
        d[i] = kInf32;
    template_min<W>(x, y, z, sv, tmpl, dx, dy, dz, R, pl, H, d);
    int32_t cv[W];
    float f[W];
    bool any = false;  // some voxel of the group where the template is nearer
#pragma unroll
    for (int i = 0; i < W; ++i) {
        cv[i] = min(sv[i], d[i]);
        any |= d[i] < sv[i];
    }
    if (kStaticSdf && !any) {
#pragma unroll
        for (int i = 0; i < W; ++i)
            f[i] = sf[i];
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i)
            f[i] = (kStaticSdf && sv[i] <= d[i]) ? sf[i] : sq_to_sdf_fast(cv[i], vox);
    }
    if (W == 4) {
        if (kSq)
            __stcs(reinterpret_cast<int4 *>(oq + off), make_int4(cv[0], cv[1], cv[2], cv[3]));
        if (kSdfOut)
            __stcs(reinterpret_cast<float4 *>(of + off), make_float4(f[0], f[1], f[2], f[3]));
    } else {
        if (kSq)
            __stcs(oq + off, cv[0]);
        if (kSdfOut)
            __stcs(of + off, f[0]);
    }
}

template <bool kStaticSdf, int W>
__device__ __forceinline__ void load_static(int off, const int32_t *__restrict__ static_sq,
                                            const float *__restrict__ static_sdf, int32_t *sv, float *sf)
{
    if (W == 4) {
        const int4 a = __ldg(reinterpret_cast<const int4 *>(static_sq + off));
        sv[0] = a.x, sv[1] = a.y, sv[2] = a.z, sv[3] = a.w;
        if (kStaticSdf) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(static_sdf + off));
            sf[0] = f.x, sf[1] = f.y, sf[2] = f.z, sf[3] = f.w;
        }
    } else {
        sv[0] = __ldg(static_sq + off);
        if (kStaticSdf)
            sf[0] = __ldg(static_sdf + off);
    }
}

template <bool kSq, bool kSdfOut, bool kStaticSdf>
__global__ void __launch_bounds__(32 * kTrWarps)
    k_composite_translated(const int32_t *__restrict__ static_sq, const float *__restrict__ static_sdf,
                           const int32_t *__restrict__ tmpl, int dx, int dy, int dz, int R,
                           const __grid_constant__ TmplPlacement pl, int H, int nx, int ny, int nz, int t0, int nt,
                           int32_t *__restrict__ comp_sq, float *__restrict__ comp_sdf, float vox, int vec)
{
    const int lt = (int)(blockIdx.x % nt);
    const long long blk = blockIdx.x / nt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long nrows = (long long)ny * nz;
    const long long V = nrows * nx;
    const int4 *place = pl.place + lt * H;
    int32_t *oq = kSq ? comp_sq + (long long)(t0 + lt) * V : nullptr;
    float *of = kSdfOut ? comp_sdf + (long long)(t0 + lt) * V : nullptr;
    if (vec) {
        // the CTA's static rows are one contiguous range; the nt CTAs of the
        // row block split its L2 prefetch in 4 KB pieces (16-byte aligned,
        // whole multiples of 16 bytes: nx % 4 == 0, aligned fields)
        const long long r0 = blk * kTrRowIters * kTrWarps;
        const long long r1 = min(r0 + kTrRowIters * kTrWarps, nrows);
        const long long e0 = r0 * nx, e1 = r1 * nx;
        for (long long a = e0 + (long long)(lt + nt * (int)threadIdx.x) * 1024; a < e1;
             a += (long long)nt * blockDim.x * 1024) {
            const uint32_t bytes = (uint32_t)(min(a + 1024, e1) - a) * 4u;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_sq + a), "r"(bytes) : "memory");
            if (kStaticSdf)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_sdf + a), "r"(bytes)
                             : "memory");
        }
    }
    for (int it = 0; it < kTrRowIters; ++it) {
        const long long row = (blk * kTrRowIters + it) * kTrWarps + warp;
        if (row >= nrows)
            return;  // warp-uniform; later rows of this warp are larger still
        const int y = (int)(row % ny), z = (int)(row / ny);
        const int base = (int)(row * nx);  // within one field: V <= 512^3 < 2^31
        if (vec) {
            // two groups of 4 per lane in flight: both loaded before either is stored
            for (int x = 4 * lane; x < nx; x += 256) {
                const bool two = x + 128 < nx;
                int32_t sv0[4], sv1[4];
                float sf0[4], sf1[4];
                load_static<kStaticSdf, 4>(base + x, static_sq, static_sdf, sv0, sf0);
                if (two)
                    load_static<kStaticSdf, 4>(base + x + 128, static_sq, static_sdf, sv1, sf1);
                translated_finish<kSq, kSdfOut, kStaticSdf, 4>(x, y, z, base + x, sv0, sf0, tmpl, dx, dy, dz, R,
                                                               place, H, oq, of, vox);
                if (two)
                    translated_finish<kSq, kSdfOut, kStaticSdf, 4>(x + 128, y, z, base + x + 128, sv1, sf1, tmpl,
                                                                   dx, dy, dz, R, place, H, oq, of, vox);
            }
        } else {
            for (int x = lane; x < nx; x += 32) {
                int32_t sv[1];
                float sf[1];
                load_static<kStaticSdf, 1>(base + x, static_sq, static_sdf, sv, sf);
                translated_finish<kSq, kSdfOut, kStaticSdf, 1>(x, y, z, base + x, sv, sf, tmpl, dx, dy, dz, R, place,
                                                               H, oq, of, vox);
            }
        }
    }
}

template <bool kSq, bool kSdfOut, bool kStaticSdf>
cudaError_t launch_tr(unsigned nblk, const int32_t *static_sq, const float *static_sdf, const int32_t *tmpl,
                      const int *dims, int R, const TmplPlacement &pl, int H, int nx, int ny, int nz, int t0, int nt,
                      int32_t *comp_sq, float *comp_sdf, float vox, int vec, cudaStream_t st)
{
    k_composite_translated<kSq, kSdfOut, kStaticSdf><<<nblk, 32 * kTrWarps, 0, st>>>(
        static_sq, static_sdf, tmpl, dims[0], dims[1], dims[2], R, pl, H, nx, ny, nz, t0, nt, comp_sq, comp_sdf, vox,
        vec);
    return cudaGetLastError();
}

// Largest finite positive value of a field (0 if none): per-thread maxima,
// a shared-memory tree per CTA, one atomicMax per CTA.
__global__ void __launch_bounds__(256) k_finite_max(const int32_t *__restrict__ sq, long long n,
                                                     int32_t *__restrict__ out)
{
    __shared__ int32_t part[256];
    int32_t m = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t v = __ldg(sq + i);
        if (v < kInf32)
            m = max(m, v);
    }
    part[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            part[threadIdx.x] = max(part[threadIdx.x], part[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        atomicMax(out, part[0]);
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// The template box of a primitive (see the file comment); -1 when some axis
// holds no voxel centre of the primitive's range.
int template_box(const int32_t *cap, int R, int lo[3], int dims[3])
{
    const int32_t r = cap[6] & ~PCDF_CYLINDER;
    for (int a = 0; a < 3; ++a) {
        const long long mn = (long long)std::min(cap[a], cap[3 + a]) - r;
        const long long mx = (long long)std::max(cap[a], cap[3 + a]) + r;
        const long long first = host::floordiv(mn - 8 + 15, 16);  // least i with 16 i + 8 >= mn
        const long long last = host::floordiv(mx - 8, 16);        // greatest i with 16 i + 8 <= mx
        if (last < first)
            return -1;
        lo[a] = (int)(first - R);
        dims[a] = (int)(last - first + 1 + 2LL * R);
    }
    return 0;
}

int check_primitive(const int32_t *cap, int R, int lo[3], int dims[3])
{
    using host::fail;
    if (!cap)
        return fail(PCDF_EINVAL, "cap is NULL");
    if (R < 0 || R > PCDF_MAX_DIM)
        return fail(PCDF_EINVAL, "R = %d outside [0, %d]", R, PCDF_MAX_DIM);
    for (int a = 0; a < 6; ++a)
        if (cap[a] < PCDF_CAP_MIN || cap[a] > PCDF_CAP_MAX)
            return fail(PCDF_EINVAL, "primitive coordinate %d = %d outside [%d, %d]", a, cap[a], PCDF_CAP_MIN,
                        PCDF_CAP_MAX);
    const int32_t r = cap[6] & ~PCDF_CYLINDER;
    if (r < 0 || r > PCDF_CAP_MAX_R)
        return fail(PCDF_EINVAL, "primitive radius %d outside [0, %d]", r, PCDF_CAP_MAX_R);
    if ((cap[6] & PCDF_CYLINDER) && cap[0] == cap[3] && cap[1] == cap[4] && cap[2] == cap[5])
        return fail(PCDF_EINVAL, "cylinder with a zero-length axis");
    if (template_box(cap, R, lo, dims))
        return fail(PCDF_EINVAL, "no voxel centre lies within the primitive's range on some axis");
    for (int a = 0; a < 3; ++a)
        if (dims[a] > PCDF_MAX_DIM)
            return fail(PCDF_EINVAL, "template box side %d > %d (reduce R)", dims[a], PCDF_MAX_DIM);
    return PCDF_OK;
}

pcdf_grid box_grid(const int dims[3])
{
    pcdf_grid g;
    std::memset(&g, 0, sizeof(g));
    g.nx = dims[0];
    g.ny = dims[1];
    g.nz = dims[2];
    g.vox = 1.f;
    return g;
}

}  // namespace
}  // namespace pcdf

using namespace pcdf;
using namespace pcdf::host;

extern "C" {

int pcdf_template_box(const int32_t *cap, int32_t R, int32_t *lo, int32_t *dims)
{
    if (!lo || !dims)
        return fail(PCDF_EINVAL, "lo and dims must be non-NULL");
    int l[3], d[3];
    if (int rc = check_primitive(cap, R, l, d))
        return rc;
    for (int a = 0; a < 3; ++a) {
        lo[a] = l[a];
        dims[a] = d[a];
    }
    return PCDF_OK;
}

int pcdf_field_max(const int32_t *sq, int64_t n, int32_t *out, void *stream)
{
    if (n < 0 || (n > 0 && !sq) || !out)
        return fail(PCDF_EINVAL, "sq (n > 0) and out must be non-NULL, n >= 0");
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t), st);
    if (e == cudaSuccess && n > 0) {
        int sms = 0;
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) {
            const long long want = (n + 255) / 256;
            const unsigned nblk = (unsigned)std::min<long long>(want, 8LL * std::max(sms, 1));
            k_finite_max<<<nblk, 256, 0, st>>>(sq, n, out);
            e = cudaGetLastError();
        }
    }
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "field max");
}

int pcdf_template_radius(int32_t max_value, int32_t *R)
{
    if (!R)
        return fail(PCDF_EINVAL, "R is NULL");
    if (max_value < 0)
        return fail(PCDF_EINVAL, "max_value = %d < 0", max_value);
    // integer square root, rounded up: the least r with r * r >= max_value
    long long r = (long long)std::sqrt((double)max_value);
    while (r * r < max_value)
        ++r;
    while (r > 0 && (r - 1) * (r - 1) >= max_value)
        --r;
    *R = (int32_t)r;
    return PCDF_OK;
}

int pcdf_lattice_placements(const int32_t *caps, int32_t T, int32_t H, const int32_t *ref_cap, const int32_t *ref_lo,
                            int32_t *lo)
{
    if (T < 1 || T > PCDF_MAX_T || H < 0 || H > PCDF_MAX_H)
        return fail(PCDF_EINVAL, "T = %d or H = %d out of range", T, H);
    if (!ref_cap || !ref_lo || (H > 0 && (!caps || !lo)))
        return fail(PCDF_EINVAL, "caps, ref_cap, ref_lo and lo must be non-NULL");
    // check everything before writing anything
    for (long long q = 0; q < (long long)T * H; ++q) {
        const int32_t *c = caps + 7 * q;
        if (c[6] != ref_cap[6])
            return fail(PCDF_EINVAL, "primitive %lld has another radius or kind than the reference", q);
        for (int a = 0; a < 3; ++a) {
            const long long d = (long long)c[a] - ref_cap[a];
            if ((long long)c[3 + a] - ref_cap[3 + a] != d)
                return fail(PCDF_EINVAL, "primitive %lld has another axis than the reference", q);
            if (d % 16 != 0)
                return fail(PCDF_EINVAL, "primitive %lld is not a whole-voxel move of the reference", q);
            const long long p = (long long)ref_lo[a] + d / 16;
            if (p < -PCDF_MAX_DIM || p > PCDF_MAX_DIM)
                return fail(PCDF_EINVAL, "placement of primitive %lld outside [%d, %d]", q, -PCDF_MAX_DIM,
                            PCDF_MAX_DIM);
        }
    }
    for (long long q = 0; q < (long long)T * H; ++q)
        for (int a = 0; a < 3; ++a)
            lo[3 * q + a] = ref_lo[a] + (caps[7 * q + a] - ref_cap[a]) / 16;
    return PCDF_OK;
}

int pcdf_template_workspace_bytes(const int32_t *cap, int32_t R, size_t *bytes)
{
    if (!bytes)
        return fail(PCDF_EINVAL, "bytes is NULL");
    int l[3], d[3];
    if (int rc = check_primitive(cap, R, l, d))
        return rc;
    const pcdf_grid g = box_grid(d);
    *bytes = full_edt_ws(&g);
    return PCDF_OK;
}

int pcdf_build_template(const int32_t *cap, int32_t R, int32_t *tmpl, void *workspace, size_t workspace_bytes,
                        void *stream)
{
    int l[3], d[3];
    if (int rc = check_primitive(cap, R, l, d))
        return rc;
    if (!tmpl || !workspace)
        return fail(PCDF_EINVAL, "tmpl and workspace must be non-NULL");
    if (!aligned(workspace, kAlign))
        return fail(PCDF_EINVAL, "workspace must be %zu-byte aligned", kAlign);
    const pcdf_grid g = box_grid(d);
    if (workspace_bytes < full_edt_ws(&g))
        return fail(PCDF_ENOMEM, "workspace %zu bytes < %zu needed", workspace_bytes, full_edt_ws(&g));
    // the primitive in the box's frame: box voxel i is map voxel lo + i
    int32_t c[7];
    for (int a = 0; a < 3; ++a) {
        c[a] = cap[a] - 16 * l[a];
        c[3 + a] = cap[3 + a] - 16 * l[a];
    }
    c[6] = cap[6];
    std::vector<CapInfo> ci;
    int zlo = 0, zhi = -1;
    if (int rc = make_capinfo(&g, 1, 1, c, ci, &zlo, &zhi))
        return rc;
    static thread_local CapBatch batch;
    batch.count = 1;
    batch.caps[0] = ci[0];
    return run_full_edt(&g, 2, nullptr, &batch, 1, tmpl, nullptr, workspace, (cudaStream_t)stream);
}

int pcdf_composite_translated(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf, int32_t T,
                              int32_t H, const int32_t *tmpl, const int32_t *dims, int32_t R, const int32_t *lo,
                              int32_t *comp_sq, float *comp_sdf, void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (T < 1 || T > PCDF_MAX_T)
        return fail(PCDF_EINVAL, "T = %d outside [1, %d]", T, PCDF_MAX_T);
    if (H < 0 || H > PCDF_MAX_H)
        return fail(PCDF_EINVAL, "H = %d outside [0, %d]", H, PCDF_MAX_H);
    if (!static_sq || (!comp_sq && !comp_sdf))
        return fail(PCDF_EINVAL, "static_sq and at least one output must be non-NULL");
    int d[3] = {1, 1, 1};
    if (H > 0) {
        if (!tmpl || !dims || !lo)
            return fail(PCDF_EINVAL, "tmpl, dims and lo must be non-NULL when H > 0");
        for (int a = 0; a < 3; ++a) {
            if (dims[a] < 1 || dims[a] > PCDF_MAX_DIM)
                return fail(PCDF_EINVAL, "template side %d outside [1, %d]", dims[a], PCDF_MAX_DIM);
            d[a] = dims[a];
            if (R < 0 || 2LL * R >= dims[a])
                return fail(PCDF_EINVAL, "R = %d must satisfy 0 <= 2 R < every template side", R);
        }
        for (long long q = 0; q < 3LL * T * H; ++q)
            if (lo[q] < -PCDF_MAX_DIM || lo[q] > PCDF_MAX_DIM)
                return fail(PCDF_EINVAL, "placement %lld = %d outside [%d, %d]", q / 3, lo[q], -PCDF_MAX_DIM,
                            PCDF_MAX_DIM);
    }
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    const int vec = nx % 4 == 0 && aligned16(static_sq) && (!static_sdf || aligned16(static_sdf)) &&
                    (!comp_sq || aligned16(comp_sq)) && (!comp_sdf || aligned16(comp_sdf));
    const long long nrows = (long long)ny * nz;
    const long long rows_per_cta = (long long)kTrWarps * kTrRowIters;
    const long long nblk_rows = (nrows + rows_per_cta - 1) / rows_per_cta;
    const int t_chunk = H > 0 ? std::max(1, kMaxPlacements / H) : PCDF_MAX_T;
    static thread_local TmplPlacement pl;
    for (int t0 = 0; t0 < T; t0 += t_chunk) {
        const int nt = std::min(t_chunk, T - t0);
        for (int lt = 0; lt < nt; ++lt)
            for (int h = 0; h < H; ++h) {
                const int32_t *p = lo + 3LL * ((long long)(t0 + lt) * H + h);
                pl.place[lt * H + h] = make_int4(p[0], p[1], p[2], 0);
            }
        const unsigned nblk = (unsigned)(nblk_rows * nt);
        cudaError_t e;
        const cudaStream_t st = (cudaStream_t)stream;
        if (comp_sq && comp_sdf)
            e = static_sdf ? launch_tr<true, true, true>(nblk, static_sq, static_sdf, tmpl, d, R, pl, H, nx, ny, nz, t0,
                                                         nt, comp_sq, comp_sdf, grid->vox, vec, st)
                           : launch_tr<true, true, false>(nblk, static_sq, static_sdf, tmpl, d, R, pl, H, nx, ny, nz,
                                                          t0, nt, comp_sq, comp_sdf, grid->vox, vec, st);
        else if (comp_sq)
            e = launch_tr<true, false, false>(nblk, static_sq, static_sdf, tmpl, d, R, pl, H, nx, ny, nz, t0, nt,
                                              comp_sq, comp_sdf, grid->vox, vec, st);
        else
            e = static_sdf ? launch_tr<false, true, true>(nblk, static_sq, static_sdf, tmpl, d, R, pl, H, nx, ny, nz,
                                                          t0, nt, comp_sq, comp_sdf, grid->vox, vec, st)
                           : launch_tr<false, true, false>(nblk, static_sq, static_sdf, tmpl, d, R, pl, H, nx, ny, nz,
                                                           t0, nt, comp_sq, comp_sdf, grid->vox, vec, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "translated composite");
    }
    return PCDF_OK;
}

}  // extern "C"

// Host-side helpers of the C ABI: argument checks, capsule tables and the
// plan (slab, workspace layout) of a composite request.  Host code only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "host.h"

namespace pcdf {
namespace host {

thread_local char g_err[512] = "";

const char *last_error() { return g_err; }

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    return fail(PCDF_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int check_grid(const pcdf_grid *g)
{
    if (!g)
        return fail(PCDF_EINVAL, "grid is NULL");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->nx > PCDF_MAX_DIM || g->ny > PCDF_MAX_DIM ||
        g->nz > PCDF_MAX_DIM)
        return fail(PCDF_EINVAL, "grid dims %d x %d x %d outside [1, %d]", g->nx, g->ny, g->nz, PCDF_MAX_DIM);
    if (!std::isfinite(g->vox) || !(g->vox > 0.f))
        return fail(PCDF_EINVAL, "voxel size must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(g->origin[a]))
            return fail(PCDF_EINVAL, "origin must be finite");
    return PCDF_OK;
}

long long nvox(const pcdf_grid *g) { return (long long)g->nx * g->ny * g->nz; }

// floor(a / b) for b > 0
long long floordiv(long long a, long long b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Capsule ranges and the voxel-index bounding box of its voxel centres: a
// centre 16 i + 8 can lie within r of the segment only if it lies within
// [min(a, b) - r, max(a, b) + r] on every axis.
int make_capinfo(const pcdf_grid *g, int T, int H, const int32_t *caps, std::vector<pcdf::CapInfo> &out,
                 int *zlo, int *zhi)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    out.resize((size_t)T * H);
    *zlo = n[2];
    *zhi = -1;
    for (long long q = 0; q < (long long)T * H; ++q) {
        const int32_t *c = caps + 7 * q;
        for (int a = 0; a < 6; ++a)
            if (c[a] < PCDF_CAP_MIN || c[a] > PCDF_CAP_MAX)
                return fail(PCDF_EINVAL, "capsule %lld coordinate %d = %d outside [%d, %d]", q, a, c[a],
                            PCDF_CAP_MIN, PCDF_CAP_MAX);
        const bool cyl = (c[6] & PCDF_CYLINDER) != 0;
        const int32_t r = c[6] & ~PCDF_CYLINDER;
        if (r < 0 || r > PCDF_CAP_MAX_R)
            return fail(PCDF_EINVAL, "capsule %lld radius %d outside [0, %d]", q, r, PCDF_CAP_MAX_R);
        if (cyl && c[0] == c[3] && c[1] == c[4] && c[2] == c[5])
            return fail(PCDF_EINVAL, "cylinder %lld has a zero-length axis", q);
        pcdf::CapInfo &ci = out[q];
        std::memset(&ci, 0, sizeof(ci));
        ci.cyl = cyl;
        bool empty = false;
        for (int a = 0; a < 3; ++a) {
            ci.a[a] = c[a];
            ci.b[a] = c[3 + a];
            // the capsule's box also bounds the cylinder (a subset of it)
            const long long mn = std::min(c[a], c[3 + a]) - (long long)r;
            const long long mx = std::max(c[a], c[3 + a]) + (long long)r;
            long long lo = floordiv(mn - 8 + 15, 16);  // ceil((mn - 8) / 16)
            long long hi = floordiv(mx - 8, 16);
            lo = std::max(lo, 0LL);
            hi = std::min(hi, (long long)n[a] - 1);
            ci.lo[a] = (int32_t)lo;
            ci.hi[a] = (int32_t)hi;
            empty |= lo > hi;
        }
        ci.r = r;
        if (empty) {
            for (int a = 0; a < 3; ++a) {
                ci.lo[a] = 1;
                ci.hi[a] = 0;
            }
            continue;
        }
        *zlo = std::min(*zlo, ci.lo[2]);
        *zhi = std::max(*zhi, ci.hi[2]);
    }
    return PCDF_OK;
}

int check_caps_args(int T, int H, const int32_t *caps)
{
    if (T < 1 || T > PCDF_MAX_T)
        return fail(PCDF_EINVAL, "T = %d outside [1, %d]", T, PCDF_MAX_T);
    if (H < 0 || H > PCDF_MAX_H)
        return fail(PCDF_EINVAL, "H = %d outside [0, %d]", H, PCDF_MAX_H);
    if (H > 0 && !caps)
        return fail(PCDF_EINVAL, "caps is NULL with H = %d", H);
    return PCDF_OK;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Static (or union) signed EDT of one grid: row bits (mode 0 occupancy, 1
// occupancy OR the capsules of one t, 2 the capsules alone), fused x+y pass,
// z pass with optional float epilogue.
int run_full_edt(const pcdf_grid *g, int mode, const uint8_t *occ, const pcdf::CapBatch *caps, int H, int32_t *sq,
                 float *sdf, void *ws, cudaStream_t st, int32_t *colmax)
{
    cudaError_t e = pcdf::launch_full_edt(mode, occ, caps, H, g->nx, g->ny, g->nz, sq, sdf, g->vox, ws, st, colmax);
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "full EDT");
}

size_t full_edt_ws(const pcdf_grid *g)
{
    size_t bo, co, mo;
    return pcdf::full_edt_scratch(g->nx, g->ny, g->nz, &bo, &co, &mo);
}



namespace {

// The z-dependence of a capsule's voxel set in slice k, as a key: two slices
// with equal keys hold the same voxels of it.  For a capsule whose axis is
// upright (a and b share x and y) the exact predicate at a voxel centre p
// (16k + 8 along z) reduces to: below the segment |p - a|^2 <= r^2, above it
// |p - b|^2 <= r^2, which depend on z only through |p_z - a_z| or |p_z - b_z|
// (one key per distance, the same for both caps), and between them
// (p_x - a_x)^2 + (p_y - a_y)^2 <= r^2, the same in every slice; a cylinder
// holds that disk between its end planes and nothing elsewhere.  Any other
// capsule gets a key of its own in every slice.
constexpr long long kKeyEmpty = -1, kKeyMid = -2;
long long slice_key(const CapInfo &c, int k)
{
    if (c.lo[0] > c.hi[0])
        return kKeyEmpty;  // no voxel of the grid
    if (c.a[0] != c.b[0] || c.a[1] != c.b[1])
        return (1LL << 40) + k;
    const long long pz = 16LL * k + 8, za = std::min(c.a[2], c.b[2]), zb = std::max(c.a[2], c.b[2]);
    if (c.cyl)
        return pz >= za && pz <= zb ? kKeyMid : kKeyEmpty;
    if (pz > za && pz < zb)
        return kKeyMid;
    const long long dz = pz <= za ? za - pz : pz - zb;
    return dz > c.r ? kKeyEmpty : dz;
}

void plan_slab_map(int T, int H, CompositePlan &p)
{
    p.rep.clear();
    if (p.S <= 0 || p.S > 255 || (long long)T * p.S > kSlabMapMax)
        return;
    p.rep.resize((size_t)T * p.S);
    std::map<std::vector<long long>, int> first;  // key vector -> first slice of this t holding it
    std::vector<long long> key(std::max(H, 0));
    for (int t = 0; t < T; ++t) {
        first.clear();
        for (int e = 0; e < p.S; ++e) {
            for (int h = 0; h < H; ++h)
                key[h] = slice_key(p.ci[(size_t)t * H + h], p.zlo + e);
            const auto it = first.emplace(key, e).first;
            p.rep[(size_t)t * p.S + e] = (uint8_t)it->second;
        }
    }
}

}  // namespace

void slab_map(const CompositePlan &p, SlabMap &m)
{
    m.on = p.rep.empty() ? 0 : 1;
    m.S = p.S;
    if (m.on)
        std::memcpy(m.rep, p.rep.data(), p.rep.size());
}

int plan_composite(const pcdf_grid *grid, int T, int H, const int32_t *caps, CompositePlan &p)
{
    if (int rc = check_grid(grid))
        return rc;
    if (int rc = check_caps_args(T, H, caps))
        return rc;
    if (H > 0)
        if (int rc = make_capinfo(grid, T, H, caps, p.ci, &p.zlo, &p.zhi))
            return rc;
    p.S = p.zhi >= p.zlo ? p.zhi - p.zlo + 1 : 0;
    p.slab = (long long)T * p.S * grid->nx * grid->ny;
    // stack bound of the analytic kernel: rows holding a run (<= sum of the
    // capsules' y extents) plus two free rows per run (one run per capsule)
    int ext_max = 0;
    for (int t = 0; t < T; ++t) {
        int ext = 0;
        for (int h = 0; h < H; ++h) {
            const pcdf::CapInfo &c = p.ci[(size_t)t * H + h];
            if (c.lo[0] <= c.hi[0])
                ext += c.hi[1] - c.lo[1] + 1;
        }
        ext_max = std::max(ext_max, ext);
    }
    p.cap = std::min(ext_max + 2 * H + 2, grid->ny + 2);
    p.fused = H <= pcdf::kMaxCapsPerLaunch && pcdf::dyn_xy_fits(grid->ny, H, p.cap);
    plan_slab_map(T, H, p);
    if (p.S == 0)
        p.need = 0;
    else if (p.fused)
        p.need = align_up((size_t)p.slab * sizeof(int32_t));
    else
        p.need = align_up((size_t)p.slab * sizeof(int16_t)) + align_up((size_t)p.slab * sizeof(int32_t));
    if (p.S > 0) {  // column maxima of the static field
        p.colmax_off = p.need;
        p.need += align_up((size_t)grid->nx * grid->ny * sizeof(int32_t));
    }
    return PCDF_OK;
}

int32_t *plan_mid(const CompositePlan &p, void *workspace)
{
    return p.fused ? (int32_t *)workspace
                   : (int32_t *)((char *)workspace + align_up((size_t)p.slab * sizeof(int16_t)));
}

int check_ws(const CompositePlan &p, void *workspace, size_t workspace_bytes)
{
    if (p.S == 0)
        return PCDF_OK;
    if (!workspace || !aligned(workspace, kAlign))
        return fail(PCDF_EINVAL, "workspace must be non-NULL and %zu-byte aligned", kAlign);
    if (workspace_bytes < p.need)
        return fail(PCDF_ENOMEM, "workspace %zu bytes < %zu needed", workspace_bytes, p.need);
    return PCDF_OK;
}

int composite_prepare(const pcdf_grid *grid, int T, int H, const CompositePlan &p, void *workspace,
                      cudaStream_t st)
{
    if (p.S == 0)
        return PCDF_OK;
    int32_t *mid = plan_mid(p, workspace);
    const long long sliceN = (long long)grid->nx * grid->ny;
    // capsules travel as kernel parameters, in chunks of whole time steps
    const int t_chunk = std::max(1, pcdf::kMaxCapsPerLaunch / std::max(H, 1));
    static thread_local pcdf::CapBatch batch;
    if (p.fused) {
        static thread_local pcdf::SlabMap map;
        slab_map(p, map);
        for (int t0 = 0; t0 < T; t0 += t_chunk) {
            const int nt = std::min(t_chunk, T - t0);
            batch.count = nt * H;
            std::memcpy(batch.caps, p.ci.data() + (size_t)t0 * H, sizeof(pcdf::CapInfo) * nt * H);
            cudaError_t e =
                pcdf::launch_dyn_xy(&batch, &map, H, grid->nx, grid->ny, p.zlo, p.S, t0, nt, p.cap, mid, st);
            if (e != cudaSuccess)
                return cuda_fail(e, "dynamic x+y pass");
        }
        return PCDF_OK;
    }
    int16_t *g16 = (int16_t *)workspace;
    for (int t0 = 0; t0 < T; t0 += t_chunk) {
        const int nt = std::min(t_chunk, T - t0);
        batch.count = nt * H;
        std::memcpy(batch.caps, p.ci.data() + (size_t)t0 * H, sizeof(pcdf::CapInfo) * nt * H);
        cudaError_t e = pcdf::launch_pass_x(2, nullptr, &batch, H, grid->nx, grid->ny, p.zlo, p.S, nt,
                                            g16 + (long long)t0 * p.S * sliceN, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "dynamic row pass");
    }
    cudaError_t e = pcdf::launch_envelope_i16(g16, mid, grid->ny, grid->nx, (long long)grid->nx * T * p.S, sliceN,
                                              grid->nx, st);
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "dynamic y pass");
}

int composite_finish(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf, int t0, int nt,
                     const CompositePlan &p, int32_t *comp_sq, float *comp_sdf, void *workspace, cudaStream_t st,
                     bool have_colmax)
{
    cudaError_t e;
    if (p.S == 0) {
        e = pcdf::launch_broadcast_static(static_sq, nvox(grid), t0, nt, comp_sq, comp_sdf, grid->vox, st);
        return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "broadcast");
    }
    const int32_t *mid = plan_mid(p, workspace);
    int32_t *colmax = (int32_t *)((char *)workspace + p.colmax_off);
    if (!have_colmax) {
        e = pcdf::launch_colmax(static_sq, grid->nx, grid->ny, grid->nz, colmax, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "static column maxima");
    }
    static thread_local pcdf::SlabMap map;
    slab_map(p, map);
    e = pcdf::launch_composite_z(static_sq, static_sdf, colmax, mid, &map, grid->nx, grid->ny, grid->nz, p.zlo, p.S,
                                 t0, nt, comp_sq, comp_sdf, grid->vox, st);
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "composite z pass");
}


}  // namespace host
}  // namespace pcdf

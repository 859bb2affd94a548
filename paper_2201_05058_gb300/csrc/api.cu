// Host side of the C ABI declared in include/pcdf.h: argument checks,
// workspace carving and the launch sequence of each entry point.  Nothing here
// allocates device memory or synchronises the stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "host.h"

using namespace pcdf::host;

#ifdef PCDF_CHECK_BOUNDS
namespace pcdf {
__device__ unsigned int g_bounds_error[2];  // see PCDF_IN in pcdf_internal.cuh
}
#endif

extern "C" {

const char *pcdf_last_error(void) { return last_error(); }

int pcdf_bounds_check(uint32_t *first, uint32_t *count, int32_t reset)
{
#ifdef PCDF_CHECK_BOUNDS
    unsigned int v[2] = {0u, 0u};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpyFromSymbol(v, pcdf::g_bounds_error, sizeof(v));
    if (e == cudaSuccess && reset) {
        const unsigned int zero[2] = {0u, 0u};
        e = cudaMemcpyToSymbol(pcdf::g_bounds_error, zero, sizeof(zero));
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "bounds-check word");
    if (first)
        *first = v[0];
    if (count)
        *count = v[1];
    return PCDF_OK;
#else
    (void)reset;
    if (first)
        *first = 0;
    if (count)
        *count = 0;
    return fail(PCDF_EINVAL, "not a bounds-checked build (compiled without PCDF_CHECK_BOUNDS)");
#endif
}

int pcdf_version(void) { return 100; }

int pcdf_static_workspace_bytes(const pcdf_grid *grid, size_t *bytes)
{
    if (int rc = check_grid(grid))
        return rc;
    if (!bytes)
        return fail(PCDF_EINVAL, "bytes is NULL");
    *bytes = full_edt_ws(grid);
    return PCDF_OK;
}

int pcdf_build_static_sdf(const pcdf_grid *grid, const uint8_t *occ, int32_t *static_sq, float *static_sdf,
                          void *workspace, size_t workspace_bytes, void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (!occ || !static_sq || !workspace)
        return fail(PCDF_EINVAL, "occ, static_sq and workspace must be non-NULL");
    if (!aligned(workspace, kAlign))
        return fail(PCDF_EINVAL, "workspace must be %zu-byte aligned", kAlign);
    if (workspace_bytes < full_edt_ws(grid))
        return fail(PCDF_ENOMEM, "workspace %zu bytes < %zu needed", workspace_bytes, full_edt_ws(grid));
    static pcdf::CapBatch none;  // unused by the occupancy-only row pass
    return run_full_edt(grid, 0, occ, &none, 0, static_sq, static_sdf, workspace, (cudaStream_t)stream);
}

int pcdf_composite_workspace_bytes(const pcdf_grid *grid, int32_t T, int32_t H, const int32_t *caps,
                                   size_t *bytes)
{
    if (!bytes)
        return fail(PCDF_EINVAL, "bytes is NULL");
    CompositePlan p;
    if (int rc = plan_composite(grid, T, H, caps, p))
        return rc;
    *bytes = p.need;
    return PCDF_OK;
}

int pcdf_composite_slab(const pcdf_grid *grid, int32_t T, int32_t H, const int32_t *caps, int32_t *zlo,
                        int32_t *S)
{
    if (!zlo || !S)
        return fail(PCDF_EINVAL, "zlo and S must be non-NULL");
    CompositePlan p;
    if (int rc = plan_composite(grid, T, H, caps, p))
        return rc;
    *zlo = p.S ? p.zlo : 0;
    *S = p.S;
    return PCDF_OK;
}

int pcdf_build_predicted_composite(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf,
                                   int32_t T, int32_t H, const int32_t *caps, int32_t *comp_sq, float *comp_sdf,
                                   void *workspace, size_t workspace_bytes, void *stream)
{
    CompositePlan p;
    if (int rc = plan_composite(grid, T, H, caps, p))
        return rc;
    if (!static_sq || (!comp_sq && !comp_sdf))
        return fail(PCDF_EINVAL, "static_sq and at least one output must be non-NULL");
    if (int rc = check_ws(p, workspace, workspace_bytes))
        return rc;
    if (int rc = composite_prepare(grid, T, H, p, workspace, (cudaStream_t)stream))
        return rc;
    return composite_finish(grid, static_sq, static_sdf, 0, T, p, comp_sq, comp_sdf, workspace, (cudaStream_t)stream);
}

int pcdf_composite_prepare(const pcdf_grid *grid, int32_t T, int32_t H, const int32_t *caps, void *workspace,
                           size_t workspace_bytes, void *stream)
{
    CompositePlan p;
    if (int rc = plan_composite(grid, T, H, caps, p))
        return rc;
    if (int rc = check_ws(p, workspace, workspace_bytes))
        return rc;
    return composite_prepare(grid, T, H, p, workspace, (cudaStream_t)stream);
}

int pcdf_composite_finish(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf, int32_t T,
                          int32_t H, const int32_t *caps, int32_t *comp_sq, float *comp_sdf, void *workspace,
                          size_t workspace_bytes, void *stream)
{
    CompositePlan p;
    if (int rc = plan_composite(grid, T, H, caps, p))
        return rc;
    if (!static_sq || (!comp_sq && !comp_sdf))
        return fail(PCDF_EINVAL, "static_sq and at least one output must be non-NULL");
    if (int rc = check_ws(p, workspace, workspace_bytes))
        return rc;
    return composite_finish(grid, static_sq, static_sdf, 0, T, p, comp_sq, comp_sdf, workspace, (cudaStream_t)stream);
}

int pcdf_composite_finish_range(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf, int32_t T,
                                int32_t H, const int32_t *caps, int32_t t0, int32_t nt, int32_t *comp_sq,
                                float *comp_sdf, void *workspace, size_t workspace_bytes, void *stream)
{
    CompositePlan p;
    if (int rc = plan_composite(grid, T, H, caps, p))
        return rc;
    if (!static_sq || (!comp_sq && !comp_sdf))
        return fail(PCDF_EINVAL, "static_sq and at least one output must be non-NULL");
    if (t0 < 0 || nt < 1 || t0 + nt > T)
        return fail(PCDF_EINVAL, "time range [%d, %d) outside [0, %d)", t0, t0 + nt, T);
    if (int rc = check_ws(p, workspace, workspace_bytes))
        return rc;
    return composite_finish(grid, static_sq, static_sdf, t0, nt, p, comp_sq, comp_sdf, workspace, (cudaStream_t)stream);
}

int pcdf_scratch_workspace_bytes(const pcdf_grid *grid, int32_t T, int32_t H, size_t *bytes)
{
    if (int rc = check_grid(grid))
        return rc;
    if (T < 1 || T > PCDF_MAX_T || H < 0 || H > PCDF_MAX_H)
        return fail(PCDF_EINVAL, "T or H out of range");
    if (!bytes)
        return fail(PCDF_EINVAL, "bytes is NULL");
    *bytes = full_edt_ws(grid);
    return PCDF_OK;
}

int pcdf_build_from_scratch(const pcdf_grid *grid, const uint8_t *occ, int32_t T, int32_t H, const int32_t *caps,
                            int32_t *sq, float *sdf, void *workspace, size_t workspace_bytes, void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (int rc = check_caps_args(T, H, caps))
        return rc;
    if (!occ || !sq || !workspace)
        return fail(PCDF_EINVAL, "occ, sq and workspace must be non-NULL");
    if (!aligned(workspace, kAlign))
        return fail(PCDF_EINVAL, "workspace must be %zu-byte aligned", kAlign);
    if (workspace_bytes < full_edt_ws(grid))
        return fail(PCDF_ENOMEM, "workspace %zu bytes < %zu needed", workspace_bytes, full_edt_ws(grid));
    std::vector<pcdf::CapInfo> ci;
    int zlo = 0, zhi = -1;
    if (H > 0)
        if (int rc = make_capinfo(grid, T, H, caps, ci, &zlo, &zhi))
            return rc;
    const long long V = nvox(grid);
    static thread_local pcdf::CapBatch batch;
    for (int t = 0; t < T; ++t) {
        batch.count = H;
        if (H > 0)
            std::memcpy(batch.caps, ci.data() + (size_t)t * H, sizeof(pcdf::CapInfo) * H);
        if (int rc = run_full_edt(grid, H > 0 ? 1 : 0, occ, &batch, H, sq + (long long)t * V,
                                  sdf ? sdf + (long long)t * V : nullptr, workspace, (cudaStream_t)stream))
            return rc;
    }
    return PCDF_OK;
}

static int check_query(const pcdf_grid *grid, const float *sdf, int32_t T, const float *spheres,
                       const int32_t *tidx, int64_t N)
{
    if (int rc = check_grid(grid))
        return rc;
    if (T < 1 || T > PCDF_MAX_T)
        return fail(PCDF_EINVAL, "T = %d outside [1, %d]", T, PCDF_MAX_T);
    if (N < 0)
        return fail(PCDF_EINVAL, "N < 0");
    if (N > 0 && (!sdf || !spheres || !tidx))
        return fail(PCDF_EINVAL, "sdf, spheres and tidx must be non-NULL");
    if (!aligned(spheres, 16))
        return fail(PCDF_EINVAL, "spheres must be 16-byte aligned");
    return PCDF_OK;
}

static pcdf::QueryGrid qgrid(const pcdf_grid *g)
{
    pcdf::QueryGrid q;
    q.n[0] = g->nx;
    q.n[1] = g->ny;
    q.n[2] = g->nz;
    for (int a = 0; a < 3; ++a)
        q.origin[a] = g->origin[a];
    q.vox = g->vox;
    return q;
}

int pcdf_query_cost(const pcdf_grid *grid, const float *sdf, int32_t T, const float *spheres, const int32_t *tidx,
                    int64_t N, float eps, float *h, int32_t *n_oob, void *stream)
{
    if (int rc = check_query(grid, sdf, T, spheres, tidx, N))
        return rc;
    if (N > 0 && !h)
        return fail(PCDF_EINVAL, "h must be non-NULL");
    cudaError_t e = pcdf::launch_query_cost(qgrid(grid), sdf, T, (const float4 *)spheres, tidx, N, eps, h, n_oob,
                                            (cudaStream_t)stream);
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "query");
}

int pcdf_query_cost_backward(const pcdf_grid *grid, const float *sdf, int32_t T, const float *spheres,
                             const int32_t *tidx, int64_t N, float eps, const float *grad_h, float *grad_c,
                             float *grad_r, void *stream)
{
    if (int rc = check_query(grid, sdf, T, spheres, tidx, N))
        return rc;
    if (N > 0 && (!grad_h || !grad_c))
        return fail(PCDF_EINVAL, "grad_h and grad_c must be non-NULL");
    cudaError_t e = pcdf::launch_query_cost_backward(qgrid(grid), sdf, T, (const float4 *)spheres, tidx, N, eps,
                                                     grad_h, grad_c, grad_r, (cudaStream_t)stream);
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "query backward");
}

}  // extern "C"

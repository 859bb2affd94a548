// One map update on two streams (Sec. 6 composition of Sec. 8's n fields): the
// static field of the map and the T composite fields, as pcdf_build_static_sdf
// then pcdf_build_predicted_composite, with the capsules' x+y pass (it needs
// no static field) on a side stream beside the static build.  The side stream
// first waits for the work already on the stream; the stream waits for the
// capsule pass before the composite's z stage.  The static z pass also writes
// the static column maxima that the z stage reads (no separate pass over the
// static field).  Events are created per call (no timing) and released before
// returning; nothing synchronises the host.
//
// Splitting the z stage into column chunks that start behind the static z
// pass, chunk by chunk, was measured slower (0.967 ms per headline step
// whole, 1.012 ms in two chunks, 1.067 ms in four): each chunk is only a few
// waves of CTAs, and the chunks' tails cost more than the hidden static z pass.
#include <cuda_runtime.h>

#include "host.h"

using namespace pcdf::host;

namespace {

// workspace: the static build's scratch, then the composite's
size_t update_ws(const pcdf_grid *g, const CompositePlan &p, size_t *comp_off)
{
    *comp_off = align_up(full_edt_ws(g));
    return *comp_off + p.need;
}

struct Events {
    cudaEvent_t start = nullptr, done = nullptr;
    ~Events()
    {
        if (start)
            (void)cudaEventDestroy(start);
        if (done)
            (void)cudaEventDestroy(done);
    }
};

}  // namespace

extern "C" {

int pcdf_update_workspace_bytes(const pcdf_grid *grid, int32_t T, int32_t H, const int32_t *caps, size_t *bytes)
{
    if (!bytes)
        return fail(PCDF_EINVAL, "bytes is NULL");
    CompositePlan p;
    if (int rc = plan_composite(grid, T, H, caps, p))
        return rc;
    size_t off;
    *bytes = update_ws(grid, p, &off);
    return PCDF_OK;
}

int pcdf_update_fields(const pcdf_grid *grid, const uint8_t *occ, int32_t T, int32_t H, const int32_t *caps,
                       int32_t *static_sq, float *static_sdf, int32_t *comp_sq, float *comp_sdf, void *workspace,
                       size_t workspace_bytes, void *stream, void *side_stream)
{
    CompositePlan p;
    if (int rc = plan_composite(grid, T, H, caps, p))
        return rc;
    if (!occ || !static_sq || (!comp_sq && !comp_sdf) || !workspace)
        return fail(PCDF_EINVAL, "occ, static_sq, an output and workspace must be non-NULL");
    if (!aligned(workspace, kAlign))
        return fail(PCDF_EINVAL, "workspace must be %zu-byte aligned", kAlign);
    size_t coff;
    const size_t need = update_ws(grid, p, &coff);
    if (workspace_bytes < need)
        return fail(PCDF_ENOMEM, "workspace %zu bytes < %zu needed", workspace_bytes, need);
    cudaStream_t st = (cudaStream_t)stream, sd = (cudaStream_t)side_stream;
    void *wsC = (char *)workspace + coff;
    static pcdf::CapBatch none;  // unused by the occupancy-only row pass

    Events ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev.start, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&ev.done, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventRecord(ev.start, st);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(sd, ev.start, 0);
    if (e != cudaSuccess)
        return cuda_fail(e, "update stream order");
    if (p.S > 0)
        if (int rc = composite_prepare(grid, T, H, p, wsC, sd))
            return rc;
    if ((e = cudaEventRecord(ev.done, sd)) != cudaSuccess)
        return cuda_fail(e, "update stream order");
    // the static z pass also writes the column maxima that the z stage reads
    int32_t *colmax = p.S > 0 ? (int32_t *)((char *)wsC + p.colmax_off) : nullptr;
    if (int rc = run_full_edt(grid, 0, occ, &none, 0, static_sq, static_sdf, workspace, st, colmax))
        return rc;
    if ((e = cudaStreamWaitEvent(st, ev.done, 0)) != cudaSuccess)
        return cuda_fail(e, "update stream order");
    return composite_finish(grid, static_sq, static_sdf, 0, T, p, comp_sq, comp_sdf, wsC, st, colmax != nullptr);
}

}  // extern "C"

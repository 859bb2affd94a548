// The context of the C interface: a device, a stream and one device scratch
// buffer that the context owns, so that callers need not size workspaces.
// Every pcdf_ctx_* call is the workspace call of the same name with the
// workspace taken from the context; the buffer grows, stream-ordered
// (cudaMallocAsync / cudaFreeAsync on the context's stream), when a call needs
// more than it holds, and is released by pcdf_destroy.
#include <cuda_runtime.h>

#include <new>

#include "host.h"

using namespace pcdf::host;

struct pcdf_ctx {
    int device;
    cudaStream_t stream;
    void *scratch;
    size_t bytes;
};

namespace {

// makes ctx's device current for the lifetime of the guard
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev)
            err = cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            (void)cudaSetDevice(prev);
    }
};

int check_ctx(const pcdf_ctx *ctx)
{
    return ctx ? PCDF_OK : fail(PCDF_EINVAL, "ctx is NULL");
}

// the scratch holds at least `need` bytes (at least 256, so it is never NULL)
int reserve(pcdf_ctx *ctx, size_t need)
{
    need = need < kAlign ? kAlign : align_up(need);
    if (ctx->scratch && ctx->bytes >= need)
        return PCDF_OK;
    if (ctx->scratch) {
        const cudaError_t e = cudaFreeAsync(ctx->scratch, ctx->stream);
        ctx->scratch = nullptr;
        ctx->bytes = 0;
        if (e != cudaSuccess)
            return cuda_fail(e, "context scratch release");
    }
    const cudaError_t e = cudaMallocAsync(&ctx->scratch, need, ctx->stream);
    if (e != cudaSuccess) {
        ctx->scratch = nullptr;
        (void)cudaGetLastError();
        return fail(PCDF_ENOMEM, "context scratch of %zu bytes: %s", need, cudaGetErrorString(e));
    }
    ctx->bytes = need;
    return PCDF_OK;
}

}  // namespace

extern "C" {

int pcdf_create(pcdf_ctx **out, int32_t device, void *stream)
{
    if (!out)
        return fail(PCDF_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return cuda_fail(e, "device count");
    }
    if (device < 0 || device >= n)
        return fail(PCDF_EINVAL, "device %d outside [0, %d)", device, n);
    pcdf_ctx *c = new (std::nothrow) pcdf_ctx;
    if (!c)
        return fail(PCDF_ENOMEM, "context allocation");
    c->device = device;
    c->stream = (cudaStream_t)stream;
    c->scratch = nullptr;
    c->bytes = 0;
    *out = c;
    return PCDF_OK;
}

void pcdf_destroy(pcdf_ctx *ctx)
{
    if (!ctx)
        return;
    if (ctx->scratch) {
        DeviceGuard g(ctx->device);
        (void)cudaFreeAsync(ctx->scratch, ctx->stream);
    }
    delete ctx;
}

int pcdf_scratch_bytes(const pcdf_grid *grid, int32_t T, int32_t H, size_t *bytes)
{
    if (int rc = check_grid(grid))
        return rc;
    if (T < 1 || T > PCDF_MAX_T || H < 0 || H > PCDF_MAX_H)
        return fail(PCDF_EINVAL, "T or H out of range");
    if (!bytes)
        return fail(PCDF_EINVAL, "bytes is NULL");
    // the static build and the from-scratch comparator, or a composite whose
    // capsules touch every slice (the largest slab: int16 and int32
    // intermediates plus the column maxima)
    const size_t V = (size_t)nvox(grid), slab = (size_t)T * V;
    const size_t comp = align_up(slab * sizeof(int16_t)) + align_up(slab * sizeof(int32_t)) +
                        align_up((size_t)grid->nx * grid->ny * sizeof(int32_t));
    const size_t edt = full_edt_ws(grid);
    *bytes = comp > edt ? comp : edt;
    return PCDF_OK;
}

int pcdf_ctx_reserve(pcdf_ctx *ctx, size_t bytes)
{
    if (int rc = check_ctx(ctx))
        return rc;
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess)
        return cuda_fail(g.err, "context device");
    return reserve(ctx, bytes);
}

int pcdf_ctx_build_static_sdf(pcdf_ctx *ctx, const pcdf_grid *grid, const uint8_t *occ, int32_t *static_sq,
                              float *static_sdf)
{
    if (int rc = check_ctx(ctx))
        return rc;
    size_t need = 0;
    if (int rc = pcdf_static_workspace_bytes(grid, &need))
        return rc;
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess)
        return cuda_fail(g.err, "context device");
    if (int rc = reserve(ctx, need))
        return rc;
    return pcdf_build_static_sdf(grid, occ, static_sq, static_sdf, ctx->scratch, ctx->bytes, ctx->stream);
}

int pcdf_ctx_build_predicted_composite(pcdf_ctx *ctx, const pcdf_grid *grid, const int32_t *static_sq,
                                       const float *static_sdf, int32_t T, int32_t H, const int32_t *caps,
                                       int32_t *comp_sq, float *comp_sdf)
{
    if (int rc = check_ctx(ctx))
        return rc;
    size_t need = 0;
    if (int rc = pcdf_composite_workspace_bytes(grid, T, H, caps, &need))
        return rc;
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess)
        return cuda_fail(g.err, "context device");
    if (int rc = reserve(ctx, need))
        return rc;
    return pcdf_build_predicted_composite(grid, static_sq, static_sdf, T, H, caps, comp_sq, comp_sdf, ctx->scratch,
                                          ctx->bytes, ctx->stream);
}

int pcdf_ctx_build_from_scratch(pcdf_ctx *ctx, const pcdf_grid *grid, const uint8_t *occ, int32_t T, int32_t H,
                                const int32_t *caps, int32_t *sq, float *sdf)
{
    if (int rc = check_ctx(ctx))
        return rc;
    size_t need = 0;
    if (int rc = pcdf_scratch_workspace_bytes(grid, T, H, &need))
        return rc;
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess)
        return cuda_fail(g.err, "context device");
    if (int rc = reserve(ctx, need))
        return rc;
    return pcdf_build_from_scratch(grid, occ, T, H, caps, sq, sdf, ctx->scratch, ctx->bytes, ctx->stream);
}

int pcdf_ctx_query_cost(pcdf_ctx *ctx, const pcdf_grid *grid, const float *sdf, int32_t T, const float *spheres,
                        const int32_t *tidx, int64_t N, float eps, float *h, int32_t *n_oob)
{
    if (int rc = check_ctx(ctx))
        return rc;
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess)
        return cuda_fail(g.err, "context device");
    return pcdf_query_cost(grid, sdf, T, spheres, tidx, N, eps, h, n_oob, ctx->stream);
}

int pcdf_ctx_query_cost_backward(pcdf_ctx *ctx, const pcdf_grid *grid, const float *sdf, int32_t T,
                                 const float *spheres, const int32_t *tidx, int64_t N, float eps, const float *grad_h,
                                 float *grad_c, float *grad_r)
{
    if (int rc = check_ctx(ctx))
        return rc;
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess)
        return cuda_fail(g.err, "context device");
    return pcdf_query_cost_backward(grid, sdf, T, spheres, tidx, N, eps, grad_h, grad_c, grad_r, ctx->stream);
}

int pcdf_build_batched(pcdf_ctx *ctx, const pcdf_env *envs, int32_t n_env, int32_t use_graph)
{
    if (int rc = check_ctx(ctx))
        return rc;
    if (use_graph != 0 && use_graph != 1)
        return fail(PCDF_EINVAL, "use_graph must be 0 or 1");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess)
        return cuda_fail(g.err, "context device");
    pcdf_batch *b = nullptr;
    if (int rc = pcdf_batch_create(envs, n_env, nullptr, &b))
        return rc;
    size_t need = 0;
    int rc = pcdf_batch_workspace_bytes(b, &need);
    if (rc == PCDF_OK)
        rc = reserve(ctx, need);
    if (rc == PCDF_OK)
        rc = pcdf_batch_upload(b, ctx->scratch, ctx->bytes, ctx->stream);
    if (rc == PCDF_OK && !use_graph)
        rc = pcdf_batch_run(b, ctx->scratch, ctx->stream);
    if (rc == PCDF_OK && use_graph) {
        // the run (counter reset and the two persistent launches) captured as
        // one graph on a private stream (the context's stream may be the legacy
        // default stream, which cannot be captured), launched on the context's
        // stream after the upload
        cudaStream_t cs = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int run_rc = pcdf_batch_run(b, ctx->scratch, cs);
            e = cudaStreamEndCapture(cs, &graph);
            if (run_rc != PCDF_OK)
                rc = run_rc;
        }
        if (rc == PCDF_OK && e == cudaSuccess)
            e = cudaGraphInstantiate(&exec, graph, 0);
        if (rc == PCDF_OK && e == cudaSuccess)
            e = cudaGraphLaunch(exec, ctx->stream);
        if (exec)
            (void)cudaGraphExecDestroy(exec);
        if (graph)
            (void)cudaGraphDestroy(graph);
        if (cs)
            (void)cudaStreamDestroy(cs);
        if (rc == PCDF_OK && e != cudaSuccess)
            rc = cuda_fail(e, "batched run graph");
    }
    // synchronises the stream: the plan's host memory is read by the upload
    int32_t code = PCDF_OK;
    const int erc = pcdf_batch_error(b, ctx->scratch, ctx->stream, &code);
    pcdf_batch_destroy(b);
    if (rc != PCDF_OK)
        return rc;
    if (erc != PCDF_OK)
        return erc;
    return code == PCDF_OK ? PCDF_OK : fail(code, "batched run: a dependency wait timed out");
}

}  // extern "C"

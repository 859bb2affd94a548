// Hinge obstacle cost at robot body spheres and its gradient (sm_103a).
//
// The GPMP2 obstacle factor of the paper (Sec. 7, hinge form; Sec. 8, factor i
// reads composite field min(i, n)) evaluated for many spheres at once: one
// thread per sphere, eight gathered corners of the time slice's float field,
// trilinear interpolation, hinge.  The cell choice (floor of the continuous
// index) is taken in fp32 with IEEE division so that it is reproducible.
#include <cuda_runtime.h>

#include "trilinear.cuh"

namespace pcdf {
namespace {

__device__ __forceinline__ int time_index(int s, int T) { return min(max(s, 0), T - 1); }

__global__ void k_query_cost(const QueryGrid g, const float *__restrict__ sdf, int T,
                             const float4 *__restrict__ spheres, const int32_t *__restrict__ tidx, long long N,
                             float eps, float *__restrict__ h, int32_t *__restrict__ n_oob)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool oob = false;
    if (q < N) {
        const float4 s = __ldg(spheres + q);
        const int t = time_index(__ldg(tidx + q), T);
        const long long V = (long long)g.n[0] * g.n[1] * g.n[2];
        const Sample r = trilinear(g, sdf + (PCDF_IN(t, T) ? t : 0) * V, s, false);
        const float hv = (eps + s.w) - r.d;
        h[q] = hv > 0.f ? hv : 0.f;
        oob = r.oob;
    }
    if (n_oob) {
        const unsigned m = __ballot_sync(0xffffffffu, oob);
        if ((threadIdx.x & 31) == 0 && m)
            atomicAdd(n_oob, __popc(m));
    }
}

__global__ void k_query_cost_backward(const QueryGrid g, const float *__restrict__ sdf, int T,
                                      const float4 *__restrict__ spheres, const int32_t *__restrict__ tidx,
                                      long long N, float eps, const float *__restrict__ grad_h,
                                      float *__restrict__ grad_c, float *__restrict__ grad_r)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N)
        return;
    const float4 s = __ldg(spheres + q);
    const int t = time_index(__ldg(tidx + q), T);
    const long long V = (long long)g.n[0] * g.n[1] * g.n[2];
    const Sample r = trilinear(g, sdf + (PCDF_IN(t, T) ? t : 0) * V, s, true);
    const float hv = (eps + s.w) - r.d;
    const bool active = hv > 0.f && isfinite(r.d);
    const float gh = active ? __ldg(grad_h + q) : 0.f;
    const float k = -gh / g.vox;
    grad_c[3 * q + 0] = k * r.du[0];
    grad_c[3 * q + 1] = k * r.du[1];
    grad_c[3 * q + 2] = k * r.du[2];
    if (grad_r)
        grad_r[q] = gh;
}

}  // namespace

cudaError_t launch_query_cost(const QueryGrid &g, const float *sdf, int T, const float4 *spheres,
                              const int32_t *tidx, long long N, float eps, float *h, int32_t *n_oob,
                              cudaStream_t stream)
{
    if (N <= 0)
        return cudaSuccess;
    const long long nblk = (N + 255) / 256;
    k_query_cost<<<(unsigned)nblk, 256, 0, stream>>>(g, sdf, T, spheres, tidx, N, eps, h, n_oob);
    return cudaGetLastError();
}

cudaError_t launch_query_cost_backward(const QueryGrid &g, const float *sdf, int T, const float4 *spheres,
                                       const int32_t *tidx, long long N, float eps, const float *grad_h,
                                       float *grad_c, float *grad_r, cudaStream_t stream)
{
    if (N <= 0)
        return cudaSuccess;
    const long long nblk = (N + 255) / 256;
    k_query_cost_backward<<<(unsigned)nblk, 256, 0, stream>>>(g, sdf, T, spheres, tidx, N, eps, grad_h, grad_c,
                                                              grad_r);
    return cudaGetLastError();
}

}  // namespace pcdf

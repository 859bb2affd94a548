// Hinge obstacle cost at robot body spheres and its gradient (sm_103a).
//
// The GPMP2 obstacle factor of the paper (Sec. 7, hinge form; Sec. 8, factor i
// reads composite field min(i, n)) evaluated for many spheres at once: one
// thread per sphere, eight gathered corners of the time slice's float field,
// trilinear interpolation, hinge.  The cell choice (floor of the continuous
// index) is taken in fp32 with IEEE division so that it is reproducible.
#include <cuda_runtime.h>

#include "pcdf_internal.cuh"

namespace pcdf {
namespace {

struct Sample {
    float d;       // interpolated distance (may be +/-inf)
    float du[3];   // d(d)/d(u) per axis (voxel units), 0 on dead axes
    bool oob;      // some axis was clamped
};

__device__ __forceinline__ Sample trilinear(const QueryGrid &g, const float *__restrict__ field, float4 s,
                                            bool want_grad)
{
    const float p[3] = {s.x, s.y, s.z};
    int i0[3], i1[3];
    float f[3];
    bool live[3];
    bool oob = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float q = __fdiv_rn(__fsub_rn(p[a], g.origin[a]), g.vox);
        float u = __fsub_rn(q, 0.5f);
        const float hi = (float)(g.n[a] - 1);
        const bool inside = (u >= 0.0f) && (u <= hi);
        oob |= !inside;
        u = fminf(fmaxf(u, 0.0f), hi);
        int lo = (int)floorf(u);
        lo = min(lo, max(g.n[a] - 2, 0));
        i0[a] = lo;
        i1[a] = min(lo + 1, g.n[a] - 1);
        f[a] = __fsub_rn(u, (float)lo);
        live[a] = inside && g.n[a] >= 2;
    }
    const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
    float c[2][2][2];
    bool pinf = false, ninf = false;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const float v = __ldg(field + (dz ? i1[2] : i0[2]) * sz + (dy ? i1[1] : i0[1]) * sy +
                                      (dx ? i1[0] : i0[0]));
                pinf |= v == __int_as_float(0x7f800000);
                ninf |= v == __int_as_float(0xff800000);
                c[dz][dy][dx] = v;
            }
    Sample r;
    r.oob = oob;
    r.du[0] = r.du[1] = r.du[2] = 0.f;
    if (ninf || pinf) {
        r.d = ninf ? __int_as_float(0xff800000) : __int_as_float(0x7f800000);
        return r;
    }
    float cx[2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
            cx[dz][dy] = fmaf(f[0], c[dz][dy][1] - c[dz][dy][0], c[dz][dy][0]);
    const float cy0 = fmaf(f[1], cx[0][1] - cx[0][0], cx[0][0]);
    const float cy1 = fmaf(f[1], cx[1][1] - cx[1][0], cx[1][0]);
    r.d = fmaf(f[2], cy1 - cy0, cy0);
    if (want_grad) {
        float ex[2];
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
            const float e0 = c[dz][0][1] - c[dz][0][0];
            const float e1 = c[dz][1][1] - c[dz][1][0];
            ex[dz] = fmaf(f[1], e1 - e0, e0);
        }
        const float gy0 = cx[0][1] - cx[0][0], gy1 = cx[1][1] - cx[1][0];
        r.du[0] = live[0] ? fmaf(f[2], ex[1] - ex[0], ex[0]) : 0.f;
        r.du[1] = live[1] ? fmaf(f[2], gy1 - gy0, gy0) : 0.f;
        r.du[2] = live[2] ? cy1 - cy0 : 0.f;
    }
    return r;
}

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
        const Sample r = trilinear(g, sdf + t * V, s, false);
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
    const Sample r = trilinear(g, sdf + t * V, s, true);
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

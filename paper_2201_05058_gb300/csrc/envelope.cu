// Lower-envelope pass of the exact EDT along y or z (sm_103a).
//
// One thread per column; a CTA owns 64 neighbouring columns (consecutive x,
// so each global access of the CTA is one contiguous 256-byte row).  The
// thread stages its column in shared memory with independent loads, then for
// each site set
//   set O (sites: occupied voxels; output at free voxels) and
//   set F (sites: free voxels; output at occupied voxels)
// builds the lower envelope of the parabolas (x - i)^2 + g(i) in place over
// the staged column (the entry pushed while reading element e lands in a slot
// at or before e, which has already been read) and walks it forward to write
// the outputs.  Elements of the other state are zero-distance sites; inside a
// run of them only the two ends can be nearest to anything outside the run,
// so only run ends are pushed.  The staged values are reloaded before the
// second set if the first one overwrote them.  Each voxel's signed value
// carries both sets (sign = its own state, magnitude = partial distance to the
// other state), so one pass produces the signed result.
#include <cuda_runtime.h>

#include "edt_common.cuh"

namespace pcdf {
namespace {

constexpr int kColThreads = 64;

__device__ __forceinline__ int32_t widen(int16_t v)
{
    const int a = v < 0 ? -(int)v : (int)v;
    if (a == kInf16)
        return v < 0 ? -kInf32 : kInf32;
    return v < 0 ? -(a * a) : a * a;
}
__device__ __forceinline__ int32_t widen(int32_t v) { return v; }

__device__ __forceinline__ bool bit(const uint32_t *mk, int e) { return (mk[(e >> 5) * kColThreads] >> (e & 31)) & 1u; }

template <typename TIn, bool kSdf>
__global__ void __launch_bounds__(kColThreads)
    k_envelope_col(const TIn *__restrict__ in, int32_t *__restrict__ out, float *__restrict__ sdf, float vox, int n,
                   int nx, long long ncols, long long outer_stride, long long stride)
{
    extern __shared__ uint32_t smem[];
    const int tid = threadIdx.x;
    const long long c = (long long)blockIdx.x * kColThreads + tid;
    if (c >= ncols)
        return;  // no block-level synchronisation below
    const long long base = (c / nx) * outer_stride + (c % nx);
    const TIn *col = in + base;
    uint32_t *tile = smem + tid;                            // element e at tile[e * kColThreads]
    uint32_t *mk = smem + (size_t)n * kColThreads + tid;    // occupied bits, word w at mk[w * kColThreads]
    const int nw = (n + 31) >> 5;

#pragma unroll 8
    for (int e = 0; e < n; ++e)
        tile[e * kColThreads] = (uint32_t)widen(col[(long long)e * stride]);

    int fo = n, lo = -1, ff = n, lf = -1;  // first/last occupied, first/last free
    for (int w = 0; w < nw; ++w) {
        const int e0 = w << 5, cnt = min(32, n - e0);
        uint32_t occ = 0;
        for (int b = 0; b < cnt; ++b)
            occ |= (uint32_t)((int32_t)tile[(e0 + b) * kColThreads] < 0) << b;
        mk[w * kColThreads] = occ;
        const uint32_t valid = cnt == 32 ? 0xffffffffu : ((1u << cnt) - 1u);
        const uint32_t fr = ~occ & valid;
        if (occ) {
            if (fo == n)
                fo = e0 + __ffs(occ) - 1;
            lo = e0 + 31 - __clz(occ);
        }
        if (fr) {
            if (ff == n)
                ff = e0 + __ffs(fr) - 1;
            lf = e0 + 31 - __clz(fr);
        }
    }

    // set O: output at free voxels
    if (lf >= 0) {
        const int a = max(ff - 1, 0), b = min(lf + 1, n - 1);
        EnvBuilder B(tile + a * kColThreads, kColThreads);
        for (int e = a; e <= b; ++e) {
            int g;
            if (!bit(mk, e)) {
                const int32_t v = (int32_t)tile[e * kColThreads];
                if (v == kInf32)
                    continue;
                g = v;
            } else {
                // occupied: zero-distance site; only a run end can matter
                const bool nb = (e > 0 && !bit(mk, e - 1)) || (e + 1 < n && !bit(mk, e + 1));
                if (!nb)
                    continue;
                g = 0;
            }
            B.push(e, g);
        }
        EnvCursor C(tile + a * kColThreads, kColThreads, B.top);
        int32_t *o = out + base;
        float *f = kSdf ? sdf + base : nullptr;
        for (int e = ff; e <= lf; ++e) {
            if (bit(mk, e))
                continue;
            const int d = C.eval(e);
            const int32_t r = d < 0 ? kInf32 : d;
            o[(long long)e * stride] = r;
            if (kSdf)
                f[(long long)e * stride] = sq_to_sdf(r, vox);
        }
    }

    // set F: output at occupied voxels
    if (lo >= 0) {
        const int a = max(fo - 1, 0), b = min(lo + 1, n - 1);
        if (lf >= 0) {
#pragma unroll 8
            for (int e = a; e <= b; ++e)
                tile[e * kColThreads] = (uint32_t)widen(col[(long long)e * stride]);
        }
        EnvBuilder B(tile + a * kColThreads, kColThreads);
        for (int e = a; e <= b; ++e) {
            int g;
            if (bit(mk, e)) {
                const int32_t v = (int32_t)tile[e * kColThreads];
                if (v == -kInf32)
                    continue;
                g = -v;
            } else {
                const bool nb = (e > 0 && bit(mk, e - 1)) || (e + 1 < n && bit(mk, e + 1));
                if (!nb)
                    continue;
                g = 0;
            }
            B.push(e, g);
        }
        EnvCursor C(tile + a * kColThreads, kColThreads, B.top);
        int32_t *o = out + base;
        float *f = kSdf ? sdf + base : nullptr;
        for (int e = fo; e <= lo; ++e) {
            if (!bit(mk, e))
                continue;
            const int d = C.eval(e);
            const int32_t r = d < 0 ? -kInf32 : -d;
            o[(long long)e * stride] = r;
            if (kSdf)
                f[(long long)e * stride] = sq_to_sdf(r, vox);
        }
    }
}

template <typename TIn, bool kSdf>
cudaError_t launch_col(const TIn *in, int32_t *out, float *sdf, float vox, int n, int nx, long long ncols,
                       long long outer_stride, long long stride, cudaStream_t stream)
{
    if (ncols <= 0 || n <= 0)
        return cudaSuccess;
    const size_t smem = (size_t)kColThreads * (n + (n + 31) / 32) * sizeof(uint32_t);
    cudaError_t e =
        cudaFuncSetAttribute(k_envelope_col<TIn, kSdf>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long nblk = (ncols + kColThreads - 1) / kColThreads;
    k_envelope_col<TIn, kSdf><<<(unsigned)nblk, kColThreads, smem, stream>>>(in, out, sdf, vox, n, nx, ncols,
                                                                              outer_stride, stride);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_envelope_i16(const int16_t *in, int32_t *out, int n, int nx, long long ncols,
                                long long outer_stride, long long stride, cudaStream_t stream)
{
    return launch_col<int16_t, false>(in, out, nullptr, 0.f, n, nx, ncols, outer_stride, stride, stream);
}

cudaError_t launch_envelope_i32(const int32_t *in, int32_t *out, float *sdf, float vox, int n, int nx,
                                long long ncols, long long outer_stride, long long stride, cudaStream_t stream)
{
    if (sdf)
        return launch_col<int32_t, true>(in, out, sdf, vox, n, nx, ncols, outer_stride, stride, stream);
    return launch_col<int32_t, false>(in, out, nullptr, vox, n, nx, ncols, outer_stride, stride, stream);
}

}  // namespace pcdf

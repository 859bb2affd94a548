// Lower-envelope pass of the exact EDT along y or z (sm_103a): stand-alone
// kernel and launchers; the algorithm is described in envelope.cuh.
#include <cuda_runtime.h>

#include "envelope.cuh"

namespace pcdf {
namespace {

using env::kBands;
using env::kCols;

template <typename TIn, bool kSdf>
__global__ void __launch_bounds__(kCols * kBands)
    k_envelope_banded(const TIn *__restrict__ in, int32_t *__restrict__ out, float *__restrict__ sdf, float vox,
                      int n, int nx, long long ncols, long long outer_stride, int stride)
{
    extern __shared__ uint32_t smem[];
    env::envelope_tile<TIn, kSdf, false>(in, out, sdf, vox, n, nx, ncols, outer_stride, stride,
                                         (long long)blockIdx.x * kCols, smem);
}

template <typename TIn, bool kSdf>
cudaError_t launch_banded(const TIn *in, int32_t *out, float *sdf, float vox, int n, int nx, long long ncols,
                          long long outer_stride, long long stride, cudaStream_t stream)
{
    if (ncols <= 0 || n <= 0)
        return cudaSuccess;
    const size_t smem = (size_t)kCols * (n + (n + 31) / 32) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_envelope_banded<TIn, kSdf>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    // element offsets along the column stay below 2^31: n <= 512, stride <= 512 * 512
    const long long nblk = (ncols + kCols - 1) / kCols;
    k_envelope_banded<TIn, kSdf><<<(unsigned)nblk, kCols * kBands, smem, stream>>>(in, out, sdf, vox, n, nx, ncols,
                                                                                    outer_stride, (int)stride);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_envelope_i16(const int16_t *in, int32_t *out, int n, int nx, long long ncols,
                                long long outer_stride, long long stride, cudaStream_t stream)
{
    return launch_banded<int16_t, false>(in, out, nullptr, 0.f, n, nx, ncols, outer_stride, stride, stream);
}

}  // namespace pcdf

// Predicted composite fields (Sec. 6, Sec. 8) on sm_103a: stand-alone
// kernels and launchers; the algorithms are described in composite.cuh.
#include <cuda_runtime.h>

#include "composite.cuh"

namespace pcdf {
namespace {

// Columns per CTA of k_dyn_xy: a slice's columns are shared by ceil(nx / 128)
// CTAs, one column per thread.
constexpr int kDynCols = 128;

__global__ void __launch_bounds__(128)
    k_dyn_xy(const __grid_constant__ CapBatch caps, const __grid_constant__ SlabMap map, int H, int nx, int ny,
             int zlo, int S, int t0, int cap, int32_t *__restrict__ dyn_mid)
{
    const int nxb = (nx + kDynCols - 1) / kDynCols;
    const int s = (int)blockIdx.x / nxb, xb = (int)blockIdx.x % nxb;
    // a slice whose cross-sections equal an earlier slice's is read from that one
    if (map.on && map.rep[(t0 + (int)blockIdx.y) * S + s] != s)
        return;
    extern __shared__ __align__(16) int32_t sm[];
    comp::dyn_xy_slice(caps.caps + blockIdx.y * H, H, nx, ny, zlo, S, t0 + (int)blockIdx.y, s, cap, dyn_mid, sm,
                       xb * kDynCols, min((xb + 1) * kDynCols, nx));
}

// CTAs are ordered t-fastest, so the T CTAs of one column block run together
// and read the static column block from DRAM once; each of them prefetches
// every nt-th plane of that block into L2 before its own work.
template <bool kSq, bool kSdfOut, bool kStaticSdf>
__global__ void __launch_bounds__(128, 8)
    k_composite_z(const int32_t *__restrict__ static_sq, const float *__restrict__ static_sdf,
                  const int32_t *__restrict__ colmax, const int32_t *__restrict__ dyn_mid,
                  const __grid_constant__ SlabMap map, int nx, int ny, int nz, int zlo, int S, int t0, int nt,
                  int32_t *__restrict__ comp_sq, float *__restrict__ comp_sdf, float vox, int vec)
{
    extern __shared__ uint32_t smem[];
    const int t = t0 + (int)(blockIdx.x % nt);
    comp::composite_block_short<kSq, kSdfOut, kStaticSdf>(static_sq, static_sdf, colmax, dyn_mid,
                                                          map.on ? map.rep + t * S : nullptr, nx, ny, nz, zlo, S, t,
                                                          (long long)(blockIdx.x / nt) * blockDim.x, comp_sq, comp_sdf,
                                                          vox, vec != 0, smem, (int)(blockIdx.x % nt),
                                                          vec ? nt : 0);
}

__global__ void __launch_bounds__(128) k_colmax(const int32_t *__restrict__ sq, long long V2, int nz,
                                                int32_t *__restrict__ colmax)
{
    comp::colmax_block(sq, V2, nz, colmax);
}

__global__ void k_broadcast_static(const int32_t *__restrict__ static_sq, long long V, int t0, int nt,
                                   int32_t *__restrict__ comp_sq, float *__restrict__ comp_sdf, float vox)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
        const int32_t s = __ldg(static_sq + v);
        const float f = sq_to_sdf(s, vox);
        for (int t = t0; t < t0 + nt; ++t) {
            if (comp_sq)
                __stcs(comp_sq + (long long)t * V + v, s);
            if (comp_sdf)
                __stcs(comp_sdf + (long long)t * V + v, f);
        }
    }
}

constexpr int kDynThreads = 128;

size_t dyn_xy_smem(int ny, int H, int cap) { return ((size_t)ny * (H + 1) + (size_t)cap * kDynThreads) * 4; }

}  // namespace

bool dyn_xy_fits(int ny, int H, int cap) { return dyn_xy_smem(ny, H, cap) <= 200 * 1024; }

cudaError_t launch_dyn_xy(const CapBatch *caps, const SlabMap *map, int H, int nx, int ny, int zlo, int S, int t0,
                          int n_t, int cap, int32_t *dyn_mid, cudaStream_t stream)
{
    if (S <= 0 || n_t <= 0)
        return cudaSuccess;
    const size_t smem = dyn_xy_smem(ny, H, cap);
    cudaError_t e = cudaFuncSetAttribute(k_dyn_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const unsigned nxb = (unsigned)((nx + kDynCols - 1) / kDynCols);
    k_dyn_xy<<<dim3((unsigned)S * nxb, (unsigned)n_t), kDynThreads, smem, stream>>>(*caps, *map, H, nx, ny, zlo, S,
                                                                                     t0, cap, dyn_mid);
    return cudaGetLastError();
}

namespace {

template <bool kSq, bool kSdfOut, bool kStaticSdf>
cudaError_t launch_cz(int nblk, int nthr, size_t smem, const int32_t *static_sq, const float *static_sdf,
                      const int32_t *colmax, const int32_t *dyn_mid, const SlabMap *map, int nx, int ny, int nz,
                      int zlo, int S, int t0, int nt, int32_t *comp_sq, float *comp_sdf, float vox, int vec,
                      cudaStream_t stream)
{
    auto kern = k_composite_z<kSq, kSdfOut, kStaticSdf>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    kern<<<(unsigned)nblk, nthr, smem, stream>>>(static_sq, static_sdf, colmax, dyn_mid, *map, nx, ny, nz, zlo, S,
                                                 t0, nt, comp_sq, comp_sdf, vox, vec);
    return cudaGetLastError();
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

cudaError_t launch_colmax(const int32_t *sq, int nx, int ny, int nz, int32_t *colmax, cudaStream_t stream)
{
    const long long V2 = (long long)nx * ny;
    k_colmax<<<(unsigned)((V2 + 31) / 32), 128, 0, stream>>>(sq, V2, nz, colmax);
    return cudaGetLastError();
}

cudaError_t launch_composite_z(const int32_t *static_sq, const float *static_sdf, const int32_t *colmax,
                               const int32_t *dyn_mid, const SlabMap *map, int nx, int ny, int nz, int zlo, int S,
                               int t0, int nt, int32_t *comp_sq, float *comp_sdf, float vox, cudaStream_t stream)
{
    const long long V2 = (long long)nx * ny;
    const int words = S + 2 + (S + 31) / 32;
    int nthr = 128;
    while (nthr > 32 && (size_t)nthr * words * sizeof(uint32_t) > 200 * 1024)
        nthr >>= 1;
    const size_t smem = (size_t)nthr * words * sizeof(uint32_t);
    const int nblk = (int)((V2 + nthr - 1) / nthr * nt);
    const bool sq = comp_sq != nullptr, sd = comp_sdf != nullptr, st = static_sdf != nullptr && sd;
    // 16-byte copies of all-static column blocks: every plane and column
    // block starts on a 16-byte boundary
    const int vec = V2 % 4 == 0 && aligned16(static_sq) && (!st || aligned16(static_sdf)) &&
                    (!sq || aligned16(comp_sq)) && (!sd || aligned16(comp_sdf));
#define PCDF_CZ(a, b, c)                                                                                            \
    return launch_cz<a, b, c>(nblk, nthr, smem, static_sq, static_sdf, colmax, dyn_mid, map, nx, ny, nz, zlo, S, t0, \
                              nt, comp_sq, comp_sdf, vox, vec, stream)
    if (sq && sd && st)
        PCDF_CZ(true, true, true);
    if (sq && sd)
        PCDF_CZ(true, true, false);
    if (sq)
        PCDF_CZ(true, false, false);
    if (st)
        PCDF_CZ(false, true, true);
    PCDF_CZ(false, true, false);
#undef PCDF_CZ
}

cudaError_t launch_broadcast_static(const int32_t *static_sq, long long V, int t0, int nt, int32_t *comp_sq,
                                    float *comp_sdf, float vox, cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long nblk = (V + 255) / 256;
    if (nblk > (long long)sms * 8)
        nblk = (long long)sms * 8;
    k_broadcast_static<<<(unsigned)nblk, 256, 0, stream>>>(static_sq, V, t0, nt, comp_sq, comp_sdf, vox);
    return cudaGetLastError();
}

}  // namespace pcdf

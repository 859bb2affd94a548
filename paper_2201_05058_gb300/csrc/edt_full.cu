// Exact signed EDT of a whole grid (sm_103a): the static map (Sec. 6: the
// environment's exact distance field), the union of the map and the humans'
// primitives at one t (the full per-field recompute that the composite is
// compared against), and a primitive alone on its box (the template of the
// translated primitive field).
//
// Three launches:
//   k_row_bits  one warp per row (y, z): the row's occupancy as 32-bit words
//               (bit l of word w: voxel x = 32 w + l) and, per word, the
//               nearest occupied and free voxel left of it and right of it.
//   k_edt_xy    one CTA per (slice z, 32-column word w), kB threads per
//               column: the 1-D distance along x of every voxel of its 32
//               columns from the word and its carries, then the y pass by
//               the run-split banded envelope of lean.cuh.  Output: the
//               signed 2-D partial field (int32) of the slice.
//   k_edt_z     one CTA per 32 consecutive columns (x, y) of the partial
//               field, kB threads per column: the z pass by the same
//               envelope, with the float field sign(S) sqrt|S| vox.
// The 1-D row distances never reach memory, so the grid is read once as
// bytes and the 2-D partial field is written and read once.
#include <cuda_runtime.h>

#include "edt_full.cuh"

namespace pcdf {
namespace {

using lean::kCols;

constexpr int kRowsPerCta = 8;  // k_row_bits: rows (warps) per CTA
#ifndef PCDF_XY_BANDS
#define PCDF_XY_BANDS 8
#endif
#ifndef PCDF_Z_BANDS
#define PCDF_Z_BANDS 8
#endif
constexpr int kXyBands = PCDF_XY_BANDS;  // envelope threads per column, y pass
constexpr int kZBands = PCDF_Z_BANDS;    // envelope threads per column, z pass

template <int kMode>
__global__ void __launch_bounds__(32 * kRowsPerCta)
    k_row_bits(const uint8_t *__restrict__ occ, const __grid_constant__ CapBatch caps, int H, int nx, int ny,
               long long nrows, int W, uint32_t *__restrict__ bits, uint2 *__restrict__ carry, int vec4)
{
    const long long row = (long long)blockIdx.x * kRowsPerCta + (threadIdx.x >> 5);
    if (row >= nrows)
        return;  // warp-uniform
    full::row_bits_row<kMode>(occ, caps.caps, H, nx, ny, row, nrows, W, bits, carry, threadIdx.x & 31, vec4 != 0);
}

// six CTAs of 256 threads per SM: 42 registers, and the tile (33 KB at 256
// rows) with the 16-bit band table fits six times
template <int kB>
__global__ void __launch_bounds__(kCols * kB, 6)
    k_edt_xy(const uint32_t *__restrict__ bits, const uint2 *__restrict__ carry, int nx, int ny, int nz, int W,
             int32_t *__restrict__ mid)
{
    extern __shared__ uint32_t smem[];
    full::edt_xy_block<kB, false>(bits, carry, nx, ny, nz, W, blockIdx.x, blockIdx.y, mid, smem);
}

// colmax (nullable): each column's largest value of sq; five CTAs of 256
// threads per SM (51 registers: held to 42 for six, it spills and is slower)
template <int kB, bool kSdf>
__global__ void __launch_bounds__(kCols * kB, 5)
    k_edt_z(const int32_t *__restrict__ mid, int32_t *__restrict__ sq, float *__restrict__ sdf, float vox, int n,
            long long ncols, int32_t *__restrict__ colmax)
{
    extern __shared__ uint32_t smem[];
    full::edt_z_block<kB, kSdf, false>(mid, sq, sdf, vox, n, ncols, (long long)blockIdx.x * kCols, smem, colmax);
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

size_t tile_bytes(int n) { return (size_t)kCols * (n + (n + 31) / 32) * sizeof(uint32_t); }

}  // namespace

size_t full_edt_scratch(int nx, int ny, int nz, size_t *bits_off, size_t *carry_off, size_t *mid_off)
{
    const auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t nw = (size_t)nz * ny * ((nx + 31) / 32);
    *bits_off = 0;
    *carry_off = al(nw * sizeof(uint32_t));
    *mid_off = *carry_off + al(nw * sizeof(uint2));
    return *mid_off + al((size_t)nx * ny * nz * sizeof(int32_t));
}

cudaError_t launch_full_edt(int mode, const uint8_t *occ, const CapBatch *caps, int H, int nx, int ny, int nz,
                            int32_t *sq, float *sdf, float vox, void *ws, cudaStream_t st, int32_t *colmax)
{
    size_t bo, co, mo;
    full_edt_scratch(nx, ny, nz, &bo, &co, &mo);
    uint32_t *bits = (uint32_t *)((char *)ws + bo);
    uint2 *carry = (uint2 *)((char *)ws + co);
    int32_t *mid = (int32_t *)((char *)ws + mo);
    const int W = (nx + 31) / 32;
    const long long nrows = (long long)ny * nz;
    const unsigned nb = (unsigned)((nrows + kRowsPerCta - 1) / kRowsPerCta);
    // occupancy rows of whole 32-bit words: read four bytes per lane
    const int vec4 = nx % 4 == 0 && ((uintptr_t)occ & 3u) == 0;
    switch (mode) {
    case 0:
        k_row_bits<0><<<nb, 32 * kRowsPerCta, 0, st>>>(occ, *caps, H, nx, ny, nrows, W, bits, carry, vec4);
        break;
    case 1:
        k_row_bits<1><<<nb, 32 * kRowsPerCta, 0, st>>>(occ, *caps, H, nx, ny, nrows, W, bits, carry, 0);
        break;
    default:
        k_row_bits<2><<<nb, 32 * kRowsPerCta, 0, st>>>(occ, *caps, H, nx, ny, nrows, W, bits, carry, 0);
        break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;

    const size_t sxy = tile_bytes(ny);
    if ((e = set_smem(k_edt_xy<kXyBands>, sxy)) != cudaSuccess)
        return e;
    k_edt_xy<kXyBands><<<dim3((unsigned)W, (unsigned)nz), kCols * kXyBands, sxy, st>>>(bits, carry, nx, ny, nz, W, mid);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;

    const long long ncols = (long long)nx * ny;
    const unsigned nbz = (unsigned)((ncols + kCols - 1) / kCols);
    const size_t sz = tile_bytes(nz);
    if (sdf) {
        if ((e = set_smem(k_edt_z<kZBands, true>, sz)) != cudaSuccess)
            return e;
        k_edt_z<kZBands, true><<<nbz, kCols * kZBands, sz, st>>>(mid, sq, sdf, vox, nz, ncols, colmax);
    } else {
        if ((e = set_smem(k_edt_z<kZBands, false>, sz)) != cudaSuccess)
            return e;
        k_edt_z<kZBands, false><<<nbz, kCols * kZBands, sz, st>>>(mid, sq, nullptr, vox, nz, ncols, colmax);
    }
    return cudaGetLastError();
}

}  // namespace pcdf

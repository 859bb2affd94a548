// Static-map utilities of the mapping pipeline (Sec. 8) on sm_103a.
//
//  k_voxel_filter  clears every occupied voxel with fewer than a given number
//                  of occupied voxels among its 26 in-grid neighbours (the
//                  paper clears voxels with fewer than five connected voxels).
//                  A CTA owns a 32 x 8 tile of columns and 32 slices, staged
//                  with their one-voxel halo in shared memory at once; each
//                  thread then sweeps its column with the 3 x 3 sums of the
//                  previous, current and next slice in registers.
//  k_collapse      the 2-D map for the prediction module: a column is
//                  occupied if any of its voxels in a slice range is.  Its EDT
//                  is the static EDT of a grid one slice thick.
#include <cuda_runtime.h>

#include "host.h"

using namespace pcdf::host;

namespace pcdf {
namespace {

constexpr int kFX = 32, kFY = 8, kFZ = 32;  // tile of a CTA: columns x, y; slices per CTA
constexpr int kHX = kFX + 2, kHY = kFY + 2;

// The CTA stages its slices and their one-voxel halo (kFZ + 2 slices of
// kHY x kHX bytes) with every load in flight at once, then each thread sweeps
// its column keeping the 3 x 3 sums of three consecutive slices.
__global__ void __launch_bounds__(kFX *kFY)
    k_voxel_filter(const uint8_t *__restrict__ occ, int nx, int ny, int nz, int min_n, uint8_t *__restrict__ out)
{
    __shared__ uint8_t tile[kFZ + 2][kHY][kHX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kFX + tx;
    const int x = blockIdx.x * kFX + tx, y = blockIdx.y * kFY + ty;
    const int z0 = blockIdx.z * kFZ, z1 = min(z0 + kFZ, nz);
    const long long V2 = (long long)nx * ny;
    const int x0 = blockIdx.x * kFX - 1, y0 = blockIdx.y * kFY - 1;
    const int n = (z1 - z0 + 2) * kHY * kHX;
    for (int v = tid; v < n; v += kFX * kFY) {
        const int zz = v / (kHY * kHX), rem = v - zz * (kHY * kHX);
        const int hy = rem / kHX, hx = rem - hy * kHX;
        const int gx = x0 + hx, gy = y0 + hy, gz = z0 - 1 + zz;
        uint8_t o = 0;
        if (gz >= 0 && gz < nz && gx >= 0 && gx < nx && gy >= 0 && gy < ny)
            o = __ldg(occ + gz * V2 + (long long)gy * nx + gx) != 0;
        tile[zz][hy][hx] = o;
    }
    __syncthreads();
    auto sum3 = [&](int zz) {
        int s = 0;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
                s += tile[zz][ty + dy][tx + dx];
        return s;
    };
    if (x >= nx || y >= ny)
        return;  // no block-level synchronisation below
    int s_prev = sum3(0), s_cur = sum3(1);
    for (int z = z0; z < z1; ++z) {
        const int zz = z - z0 + 1;
        const int s_next = sum3(zz + 1);
        const int o = tile[zz][ty + 1][tx + 1];
        out[z * V2 + (long long)y * nx + x] = (uint8_t)(o && s_prev + s_cur + s_next - 1 >= min_n);
        s_prev = s_cur;
        s_cur = s_next;
    }
}

__global__ void k_collapse(const uint8_t *__restrict__ occ, int nx, int ny, int z0, int z1,
                           uint8_t *__restrict__ out2d)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long V2 = (long long)nx * ny;
    if (c >= V2)
        return;
    uint8_t o = 0;
    for (int z = z0; z < z1; ++z)
        o |= __ldg(occ + z * V2 + c);
    out2d[c] = o != 0;
}

}  // namespace
}  // namespace pcdf

extern "C" {

int pcdf_filter_voxels(const pcdf_grid *grid, const uint8_t *occ, int32_t min_neighbours, uint8_t *out, void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (!occ || !out || occ == out)
        return fail(PCDF_EINVAL, "occ and out must be non-NULL and distinct");
    if (min_neighbours < 0 || min_neighbours > 27)
        return fail(PCDF_EINVAL, "min_neighbours %d outside [0, 27]", min_neighbours);
    const dim3 blk(pcdf::kFX, pcdf::kFY);
    const dim3 grd((grid->nx + pcdf::kFX - 1) / pcdf::kFX, (grid->ny + pcdf::kFY - 1) / pcdf::kFY,
                   (grid->nz + pcdf::kFZ - 1) / pcdf::kFZ);
    pcdf::k_voxel_filter<<<grd, blk, 0, (cudaStream_t)stream>>>(occ, grid->nx, grid->ny, grid->nz, min_neighbours,
                                                                out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "voxel filter");
}

int pcdf_collapse_2d(const pcdf_grid *grid, const uint8_t *occ, int32_t z0, int32_t z1, uint8_t *out2d, void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (!occ || !out2d)
        return fail(PCDF_EINVAL, "occ and out2d must be non-NULL");
    const int a = z0 < 0 ? 0 : z0, b = z1 > grid->nz ? grid->nz : z1;
    const long long V2 = (long long)grid->nx * grid->ny;
    pcdf::k_collapse<<<(unsigned)((V2 + 255) / 256), 256, 0, (cudaStream_t)stream>>>(occ, grid->nx, grid->ny, a,
                                                                                     b < a ? a : b, out2d);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "collapse");
}

}  // extern "C"

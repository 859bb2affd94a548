// Row pass of the exact EDT along x (sm_103a).
//
// For every voxel, the distance along its row to the nearest voxel of the
// other state, stored as int16 with the sign of the voxel's own state (+ free,
// - occupied) and kInf16 when the row holds no voxel of the other state.  The
// occupancy comes from the static map, from capsules (the predicted human
// primitives of Sec. 6), or from their union (the from-scratch comparator).
#include <cuda_runtime.h>

#include "rows.cuh"

namespace pcdf {
namespace {

constexpr int kRowWarps = 8;   // rows (one warp each) per CTA

template <int C, int kMode>
__global__ void __launch_bounds__(32 * kRowWarps)
    k_pass_x(const uint8_t *__restrict__ occ, const __grid_constant__ CapBatch caps, int H, int nx, int ny, int z0,
             int nslices, int16_t *__restrict__ g16)
{
    const int lane = threadIdx.x & 31;
    const long long nrows = (long long)nslices * ny;
    const long long row = (long long)blockIdx.x * kRowWarps + (threadIdx.x >> 5);
    if (row >= nrows)
        return;  // warp-uniform
    const int s = (int)(row / ny), y = (int)(row % ny);
    const int t = blockIdx.y;
    row_pass_row<C, kMode>(occ, caps.caps + t * H, H, nx, ny, y, z0 + s, g16 + ((long long)t * nrows + row) * nx,
                           lane);
}

template <int C>
cudaError_t launch_pass_x_c(int mode, const uint8_t *occ, const CapBatch *caps, int H, int nx, int ny, int z0,
                            int nslices, int n_t, int16_t *g16, cudaStream_t stream)
{
    const long long nrows = (long long)nslices * ny;
    const dim3 grid((unsigned)((nrows + kRowWarps - 1) / kRowWarps), (unsigned)n_t);
    const dim3 block(32 * kRowWarps);
    switch (mode) {
    case 0: k_pass_x<C, 0><<<grid, block, 0, stream>>>(occ, *caps, H, nx, ny, z0, nslices, g16); break;
    case 1: k_pass_x<C, 1><<<grid, block, 0, stream>>>(occ, *caps, H, nx, ny, z0, nslices, g16); break;
    default: k_pass_x<C, 2><<<grid, block, 0, stream>>>(occ, *caps, H, nx, ny, z0, nslices, g16); break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pass_x(int mode, const uint8_t *occ, const CapBatch *caps, int H, int nx, int ny, int z0,
                          int nslices, int n_t, int16_t *g16, cudaStream_t stream)
{
    if (nslices <= 0 || n_t <= 0)
        return cudaSuccess;
    const int c = (nx + 31) / 32;
    if (c <= 1) return launch_pass_x_c<1>(mode, occ, caps, H, nx, ny, z0, nslices, n_t, g16, stream);
    if (c <= 2) return launch_pass_x_c<2>(mode, occ, caps, H, nx, ny, z0, nslices, n_t, g16, stream);
    if (c <= 4) return launch_pass_x_c<4>(mode, occ, caps, H, nx, ny, z0, nslices, n_t, g16, stream);
    if (c <= 8) return launch_pass_x_c<8>(mode, occ, caps, H, nx, ny, z0, nslices, n_t, g16, stream);
    if (c <= 12) return launch_pass_x_c<12>(mode, occ, caps, H, nx, ny, z0, nslices, n_t, g16, stream);
    return launch_pass_x_c<16>(mode, occ, caps, H, nx, ny, z0, nslices, n_t, g16, stream);
}

}  // namespace pcdf

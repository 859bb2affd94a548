// Static-map utilities of the mapping pipeline (Sec. 8) on sm_103a.
//
//  k_voxel_filter  clears every occupied voxel with fewer than a given number
//                  of occupied voxels among its 26 in-grid neighbours (the
//                  paper clears voxels with fewer than five connected voxels).
//                  A CTA owns a 32 x 8 tile of columns and 32 slices, staged
//                  with their one-voxel halo in shared memory at once; each
//                  thread then sweeps its column with the 3 x 3 sums of the
//                  previous, current and next slice in registers.
//  k_voxel_filter4 the same filter on four voxels per thread when rows are
//                  whole 32-bit words (nx % 4 == 0, 4-byte aligned maps): a
//                  word holds the four voxels' bytes, the 3 x 3 x 3 count is
//                  taken byte-wise in the word (x by shifts with the
//                  neighbouring words' end bytes, from the lanes beside it,
//                  then y and z by word additions: a count is at most 27, so
//                  no byte carries into the next), and the four results are
//                  stored as one word.  A CTA stages a tile of words with
//                  its halo in shared memory (all loads in flight at once)
//                  and forms the x, then y, then z sums there, each once.
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

// k_voxel_filter4 tile: 32 words (lanes; words 1..30 are outputs, 0 and 31
// the x halo) x 8 rows x 8 slices of outputs, staged with a one-row and
// one-slice halo
constexpr int kF4Out = 30, kF4Y = 8, kF4Z = 8;
constexpr int kF4HY = kF4Y + 2, kF4HZ = kF4Z + 2;

// 0x01 in every byte of w that is non-zero, 0x00 elsewhere
__device__ __forceinline__ uint32_t bytes_nonzero(uint32_t w)
{
    uint32_t t = w | (w >> 4);
    t |= t >> 2;
    t |= t >> 1;
    return t & 0x01010101u;
}

// Lane l holds word wi = blockIdx.x * kF4Out + l - 1 of every staged row (0
// outside the grid), so the lanes 1..30 find both x neighbours of their four
// voxels in the lanes beside them.  Warp w (of 8) works on staged rows
// w, w + 8, ... in each pass:
//  0. stage the kF4HZ x kF4HY rows of words (slices z0 - 1 .., rows y0 - 1 ..),
//     every load in flight at once;
//  1. per staged row: bytes normalised to 0/1 and summed over x, the
//     normalised words of the output rows kept aside;
//  2. per slice and output row: the x sums of the row and its two y
//     neighbours added;
//  3. per output slice and row: the x+y sums of the slice and its two z
//     neighbours added, compared with min_neighbours + 1 (the count includes
//     the voxel) and masked by the voxel's own occupancy.
__global__ void __launch_bounds__(32 * kF4Y)
    k_voxel_filter4(const uint32_t *__restrict__ occ4, int nw, int ny, int nz, uint32_t thresh4,
                    uint32_t *__restrict__ out4)
{
    __shared__ uint32_t sx[kF4HZ][kF4HY][32];   // x sums of the staged rows
    __shared__ uint32_t sxy[kF4HZ][kF4Y][32];   // x+y sums of the output rows
    __shared__ uint32_t cen[kF4Z][kF4Y][32];    // normalised words of the outputs
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wi = blockIdx.x * kF4Out + lane - 1;
    const int y0 = blockIdx.y * kF4Y, z0 = blockIdx.z * kF4Z;
    const bool xin = wi >= 0 && wi < nw;
    const long long nwords = (long long)nz * ny * nw;
    constexpr int kRows = kF4HZ * kF4HY;
    constexpr int kPer = (kRows + kF4Y - 1) / kF4Y;
    uint32_t v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int r = warp + k * kF4Y;
        const int zz = r / kF4HY, yy = r - zz * kF4HY;
        const int z = z0 - 1 + zz, y = y0 - 1 + yy;
        const bool in = r < kRows && xin && z >= 0 && z < nz && y >= 0 && y < ny;
        const long long o = ((long long)(in ? z : 0) * ny + (in ? y : 0)) * nw + (in ? wi : 0);
        v[k] = in && PCDF_IN(o, nwords) ? __ldg(occ4 + o) : 0u;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int r = warp + k * kF4Y;
        if (r >= kRows)
            break;  // warp-uniform
        const int zz = r / kF4HY, yy = r - zz * kF4HY;
        const uint32_t n = bytes_nonzero(v[k]);
        const uint32_t l = __shfl_up_sync(0xffffffffu, n, 1), rr = __shfl_down_sync(0xffffffffu, n, 1);
        sx[zz][yy][lane] = n + ((n << 8) | (l >> 24)) + ((n >> 8) | (rr << 24));
        if (zz >= 1 && zz <= kF4Z && yy >= 1 && yy <= kF4Y)
            cen[zz - 1][yy - 1][lane] = n;
    }
    __syncthreads();
    for (int r = warp; r < kF4HZ * kF4Y; r += kF4Y) {
        const int zz = r / kF4Y, yy = r - zz * kF4Y;
        sxy[zz][yy][lane] = sx[zz][yy][lane] + sx[zz][yy + 1][lane] + sx[zz][yy + 2][lane];
    }
    __syncthreads();
    if (!xin || lane == 0 || lane == 31)
        return;  // no block-level synchronisation below
    for (int r = warp; r < kF4Z * kF4Y; r += kF4Y) {
        const int zz = r / kF4Y, yy = r - zz * kF4Y;
        const int z = z0 + zz, y = y0 + yy;
        if (z >= nz || y >= ny)
            continue;
        const uint32_t total = sxy[zz][yy][lane] + sxy[zz + 1][yy][lane] + sxy[zz + 2][yy][lane];
        const uint32_t keep = __vcmpgeu4(total, thresh4) & (cen[zz][yy][lane] * 0xFFu);
        const long long o = ((long long)z * ny + y) * nw + wi;
        if (PCDF_IN(o, nwords))
            out4[o] = keep & 0x01010101u;
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
    if (grid->nx % 4 == 0 && ((uintptr_t)occ & 3u) == 0 && ((uintptr_t)out & 3u) == 0) {
        const int nw = grid->nx / 4;
        const dim3 grd((unsigned)((nw + pcdf::kF4Out - 1) / pcdf::kF4Out),
                       (unsigned)((grid->ny + pcdf::kF4Y - 1) / pcdf::kF4Y),
                       (unsigned)((grid->nz + pcdf::kF4Z - 1) / pcdf::kF4Z));
        const uint32_t thresh4 = (uint32_t)(min_neighbours + 1) * 0x01010101u;  // <= 28 per byte
        pcdf::k_voxel_filter4<<<grd, 32 * pcdf::kF4Y, 0, (cudaStream_t)stream>>>(
            (const uint32_t *)occ, nw, grid->ny, grid->nz, thresh4, (uint32_t *)out);
    } else {
        const dim3 blk(pcdf::kFX, pcdf::kFY);
        const dim3 grd((grid->nx + pcdf::kFX - 1) / pcdf::kFX, (grid->ny + pcdf::kFY - 1) / pcdf::kFY,
                       (grid->nz + pcdf::kFZ - 1) / pcdf::kFZ);
        pcdf::k_voxel_filter<<<grd, blk, 0, (cudaStream_t)stream>>>(occ, grid->nx, grid->ny, grid->nz,
                                                                    min_neighbours, out);
    }
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

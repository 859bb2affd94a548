// Row pass of the exact EDT along x (sm_103a).
//
// For every voxel, the distance along its row to the nearest voxel of the
// other state, stored as int16 with the sign of the voxel's own state (+ free,
// - occupied) and kInf16 when the row holds no voxel of the other state.  The
// occupancy comes from the static map, from capsules (the predicted human
// primitives of Sec. 6), or from their union (the from-scratch comparator).
#include <cuda_runtime.h>

#include "edt_common.cuh"

namespace pcdf {
namespace {

constexpr int kBig = 1 << 20;  // "none" offset, beyond any grid coordinate
constexpr int kRowWarps = 8;   // rows (one warp each) per CTA

// ---------------------------------------------------------------------------
// row pass along x
// ---------------------------------------------------------------------------
// One warp per row.  Lane l owns x = 32*j + l for segments j = 0..C-1, so
// loads and stores are coalesced.  Ballots give, per segment, the bit masks
// of occupied and free voxels; the nearest voxel of each state at or left of
// x (and at or right of x) comes from the highest (lowest) set bit of the
// masked ballot, carried across segments as a warp-uniform position.
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
    const int z = z0 + s;
    const int t = blockIdx.y;
    int16_t *grow = g16 + ((long long)t * nrows + row) * nx;

    // capsules whose bounding box crosses this row (H <= 64)
    unsigned long long active = 0;
    if (kMode != 0) {
        for (int h = 0; h < H; ++h) {
            const CapInfo &c = caps.caps[t * H + h];
            if (c.lo[0] <= c.hi[0] && y >= c.lo[1] && y <= c.hi[1] && z >= c.lo[2] && z <= c.hi[2])
                active |= 1ull << h;
        }
    }

    uint32_t mo[C], mf[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int x = 32 * j + lane;
        const bool valid = x < nx;
        bool o = false;
        if (valid) {
            if (kMode != 2)
                o = occ[((long long)z * ny + y) * nx + x] != 0;
            if (kMode != 0 && !o) {
                for (unsigned long long m = active; m; m &= m - 1) {
                    const CapInfo &c = caps.caps[t * H + (__ffsll((long long)m) - 1)];
                    if (x >= c.lo[0] && x <= c.hi[0] && capsule_contains(c, x, y, z)) {
                        o = true;
                        break;
                    }
                }
            }
        }
        mo[j] = __ballot_sync(0xffffffffu, valid && o);
        mf[j] = __ballot_sync(0xffffffffu, valid && !o);
    }

    const uint32_t incl = (2u << lane) - 1u;    // lanes <= lane (lane 31: all)
    const uint32_t from = ~((1u << lane) - 1u);  // lanes >= lane
    int leftO[C], leftF[C];
    int lastO = -kBig, lastF = -kBig;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        uint32_t m = mo[j] & incl;
        leftO[j] = m ? 32 * j + 31 - __clz(m) : lastO;
        m = mf[j] & incl;
        leftF[j] = m ? 32 * j + 31 - __clz(m) : lastF;
        if (mo[j])
            lastO = 32 * j + 31 - __clz(mo[j]);
        if (mf[j])
            lastF = 32 * j + 31 - __clz(mf[j]);
    }
    int nextO = kBig, nextF = kBig;
#pragma unroll
    for (int j = C - 1; j >= 0; --j) {
        uint32_t m = mo[j] & from;
        const int rO = m ? 32 * j + __ffs(m) - 1 : nextO;
        m = mf[j] & from;
        const int rF = m ? 32 * j + __ffs(m) - 1 : nextF;
        if (mo[j])
            nextO = 32 * j + __ffs(mo[j]) - 1;
        if (mf[j])
            nextF = 32 * j + __ffs(mf[j]) - 1;
        const int x = 32 * j + lane;
        if (x < nx) {
            const bool o = (mo[j] >> lane) & 1u;
            const int d = o ? min(x - leftF[j], rF - x) : min(x - leftO[j], rO - x);
            const int16_t v = d >= nx ? kInf16 : (int16_t)d;
            grow[x] = o ? (int16_t)-v : v;
        }
    }
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

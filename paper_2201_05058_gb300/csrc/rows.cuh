// Row pass of the exact EDT along x: device code shared by the stand-alone
// kernel and the batched persistent kernel.
//
// For every voxel, the distance along its row to the nearest voxel of the
// other state, stored as int16 with the sign of the voxel's own state (+ free,
// - occupied) and kInf16 when the row holds no voxel of the other state.  The
// occupancy comes from the static map (mode 0), from the map OR capsules
// (mode 1, the from-scratch comparator) or from capsules only (mode 2; the
// predicted human primitives of Sec. 6).
#pragma once

#include "edt_common.cuh"

namespace pcdf {

constexpr int kRowBig = 1 << 20;  // "none" offset, beyond any grid coordinate

// One warp computes row (y, z).  Lane l owns x = 32*j + l for segments
// j = 0..C-1, so loads and stores are coalesced.  Ballots give, per segment,
// the bit masks of occupied and free voxels; the nearest voxel of each state
// at or left of x (and at or right of x) comes from the highest (lowest) set
// bit of the masked ballot, carried across segments as a warp-uniform
// position.  caps: the H capsules of this time step (modes 1 and 2).
template <int C, int kMode>
__device__ __forceinline__ void row_pass_row(const uint8_t *__restrict__ occ, const CapInfo *caps, int H, int nx,
                                             int ny, int y, int z, int16_t *__restrict__ grow, int lane)
{
    // capsules whose bounding box crosses this row (H <= 64)
    unsigned long long active = 0;
    if (kMode != 0) {
        for (int h = 0; h < H; ++h) {
            const CapInfo &c = caps[h];
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
                    const CapInfo &c = caps[__ffsll((long long)m) - 1];
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
    int lastO = -kRowBig, lastF = -kRowBig;
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
    int nextO = kRowBig, nextF = kRowBig;
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



// C (segments of 32 voxels per row) for a row of nx voxels; one of 1, 2, 4, 8, 12, 16
inline int row_segments(int nx)
{
    const int c = (nx + 31) / 32;
    return c <= 1 ? 1 : c <= 2 ? 2 : c <= 4 ? 4 : c <= 8 ? 8 : c <= 12 ? 12 : 16;
}

}  // namespace pcdf

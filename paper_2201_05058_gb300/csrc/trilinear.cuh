// Trilinear sampling of a float distance field at a world point, shared by
// the cost query and the surrogate (sm_103a).  The cell choice (floor of the
// continuous index) is taken in fp32 with IEEE division so that it is
// reproducible; see the hinge-cost conventions in include/pcdf.h.
#pragma once

#include "pcdf_internal.cuh"

namespace pcdf {

struct Sample {
    float d;       // interpolated distance (may be +/-inf)
    float du[3];   // d(d)/d(u) per axis (voxel units), 0 on dead axes
    bool oob;      // some axis was clamped
};

// The cell of a point: lower and upper corner indices per axis, the fp32
// fractions, the axes along which d varies, and whether any axis was clamped.
struct Cell {
    int i0[3], i1[3];
    float f[3];
    bool live[3];
    bool oob;
};

__device__ __forceinline__ Cell locate(const QueryGrid &g, float4 s)
{
    const float p[3] = {s.x, s.y, s.z};
    Cell c;
    c.oob = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float q = __fdiv_rn(__fsub_rn(p[a], g.origin[a]), g.vox);
        float u = __fsub_rn(q, 0.5f);
        const float hi = (float)(g.n[a] - 1);
        const bool inside = (u >= 0.0f) && (u <= hi);
        c.oob |= !inside;
        u = fminf(fmaxf(u, 0.0f), hi);
        int lo = (int)floorf(u);
        lo = min(lo, max(g.n[a] - 2, 0));
        c.i0[a] = lo;
        c.i1[a] = min(lo + 1, g.n[a] - 1);
        c.f[a] = __fsub_rn(u, (float)lo);
        c.live[a] = inside && g.n[a] >= 2;
    }
    return c;
}

// Interpolate corner values v[dz][dy][dx] of a cell: along x, then y, then z.
// Any -inf corner gives -inf, else any +inf corner gives +inf.
__device__ __forceinline__ Sample interpolate(const Cell &cl, const float (&c)[2][2][2], bool want_grad)
{
    bool pinf = false, ninf = false;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                pinf |= c[dz][dy][dx] == __int_as_float(0x7f800000);
                ninf |= c[dz][dy][dx] == __int_as_float(0xff800000);
            }
    Sample r;
    r.oob = cl.oob;
    r.du[0] = r.du[1] = r.du[2] = 0.f;
    if (ninf || pinf) {
        r.d = ninf ? __int_as_float(0xff800000) : __int_as_float(0x7f800000);
        return r;
    }
    const float *f = cl.f;
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
        r.du[0] = cl.live[0] ? fmaf(f[2], ex[1] - ex[0], ex[0]) : 0.f;
        r.du[1] = cl.live[1] ? fmaf(f[2], gy1 - gy0, gy0) : 0.f;
        r.du[2] = cl.live[2] ? cy1 - cy0 : 0.f;
    }
    return r;
}

__device__ __forceinline__ Sample trilinear(const QueryGrid &g, const float *__restrict__ field, float4 s,
                                            bool want_grad)
{
    const Cell cl = locate(g, s);
    const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
    float c[2][2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const long long o = (dz ? cl.i1[2] : cl.i0[2]) * sz + (dy ? cl.i1[1] : cl.i0[1]) * sy +
                                    (dx ? cl.i1[0] : cl.i0[0]);
                c[dz][dy][dx] = PCDF_IN(o, sz * g.n[2]) ? __ldg(field + o) : 0.f;
            }
    return interpolate(cl, c, want_grad);
}

}  // namespace pcdf

// Device helpers shared by the distance-transform kernels.
//
// Lower envelopes: the squared distance along one axis to a set of sites i
// with partial squared distances g(i) is min_i (x - i)^2 + g(i), the lower
// envelope of equal-curvature parabolas.  Envelopes are kept as stacks of
// packed words (site << 22 | g): sites are below 512 and g below 2^22 for
// every grid this library accepts, and all products below stay under 2^31.
#pragma once

#include "pcdf_internal.cuh"

namespace pcdf {

constexpr uint32_t kG22 = (1u << 22) - 1;

// Also callable from host code, so that the envelope code can be exercised on
// the CPU.
#define PCDF_HD __host__ __device__ __forceinline__

PCDF_HD uint32_t pack_site(int s, int g) { return ((uint32_t)s << 22) | (uint32_t)g; }
PCDF_HD int site_of(uint32_t w) { return (int)(w >> 22); }
PCDF_HD int gval_of(uint32_t w) { return (int)(w & kG22); }
PCDF_HD int parab(int x, int s, int g) { return (x - s) * (x - s) + g; }

// With sites s0 < s1 < s2, s1 is nowhere strictly below both neighbours iff
// the parabola of s2 overtakes s1 no later than s1 overtakes s0.  The two
// abscissae are the fractions (f1 - f0) / 2(s1 - s0) and (f2 - f1) / 2(s2 - s1)
// with f = s^2 + g; they are compared by cross-multiplication (positive
// denominators), so the test is exact.
PCDF_HD bool dominated(int s0, int g0, int s1, int g1, int s2, int g2)
{
    const int f0 = s0 * s0 + g0, f1 = s1 * s1 + g1, f2 = s2 * s2 + g2;
    return (f2 - f1) * (s1 - s0) <= (f1 - f0) * (s2 - s1);
}

// Forward cursor over an envelope stack in shared memory whose entry q lives
// at stk[q * stride]; the current and next site are kept in registers.
// eval(z) requires z to be non-decreasing between calls.
struct EnvCursor {
    const uint32_t *stk;
    int stride, top, q;
    int s, g, sn, gn;
    __device__ __forceinline__ EnvCursor(const uint32_t *stk_, int stride_, int top_)
        : stk(stk_), stride(stride_), top(top_), q(0), s(0), g(0), sn(0), gn(0)
    {
        if (top >= 0) {
            s = site_of(stk[0]);
            g = gval_of(stk[0]);
        }
        if (top >= 1) {
            sn = site_of(stk[stride]);
            gn = gval_of(stk[stride]);
        }
    }
    // min over the envelope at z; -1 if the envelope is empty
    __device__ __forceinline__ int eval(int z)
    {
        if (top < 0)
            return -1;
        int fc = parab(z, s, g);
        while (q < top) {
            const int fn = parab(z, sn, gn);
            if (fn > fc)
                break;
            ++q;
            s = sn;
            g = gn;
            fc = fn;
            if (q < top) {
                const uint32_t w = stk[(q + 1) * stride];
                sn = site_of(w);
                gn = gval_of(w);
            }
        }
        return fc;
    }
    __device__ __forceinline__ bool next_wins(int z) const { return q < top && parab(z, sn, gn) <= parab(z, s, g); }
    __device__ __forceinline__ void advance()
    {
        ++q;
        s = sn;
        g = gn;
        if (q < top) {
            const uint32_t w = stk[(q + 1) * stride];
            sn = site_of(w);
            gn = gval_of(w);
        }
    }
    // out[z * ostride] = eval(z) for z = z0 .. z1 - 1 (the envelope non-empty),
    // taking the same choices as eval without re-evaluating both parabolas
    // at every z: with f the current and f' the next parabola, f'(z) - f(z)
    // falls by 2 (sn - s) per step, so the next site takes over when that
    // running difference is no longer positive; f itself advances by
    // 2 (z - s) + 1.
    __device__ __forceinline__ void fill(int z0, int z1, int32_t *out, long long ostride)
    {
        if (z0 >= z1)
            return;
        int z = z0;
        while (next_wins(z))
            advance();
        int fc = parab(z, s, g), inc = 2 * (z - s) + 1;
        int delta = q < top ? parab(z, sn, gn) - fc : INT32_MAX, dd = q < top ? 2 * (sn - s) : 0;
        int32_t *p = out + (long long)z * ostride;
        for (; z < z1; ++z) {
            if (delta <= 0) {
                advance();
                while (next_wins(z))
                    advance();
                fc = parab(z, s, g);
                inc = 2 * (z - s) + 1;
                delta = q < top ? parab(z, sn, gn) - fc : INT32_MAX;
                dd = q < top ? 2 * (sn - s) : 0;
            }
            *p = fc;
            p += ostride;
            fc += inc;
            inc += 2;
            delta -= dd;
        }
    }
};

// Push site (e, g) onto a stack kept in shared memory (entry q at
// stk[q * stride]) with the top two entries cached in registers, popping the
// entries that the new site makes useless.
struct EnvBuilder {
    uint32_t *stk;
    int stride, top;
    int s0, g0, s1, g1;
    int lim;  // entries the stack may hold (bounds checks)
    __device__ __forceinline__ EnvBuilder(uint32_t *stk_, int stride_, int lim_ = 1 << 30)
        : stk(stk_), stride(stride_), top(-1), s0(0), g0(0), s1(0), g1(0), lim(lim_) {}
    __device__ __forceinline__ void push(int e, int g)
    {
        while (top >= 1 && dominated(s0, g0, s1, g1, e, g)) {
            --top;
            s1 = s0;
            g1 = g0;
            if (top >= 1) {
                const uint32_t w = PCDF_IN(top - 1, lim) ? stk[(top - 1) * stride] : 0u;
                s0 = site_of(w);
                g0 = gval_of(w);
            }
        }
        ++top;
        if (PCDF_IN(top, lim))
            stk[top * stride] = pack_site(e, g);
        s0 = s1;
        g0 = g1;
        s1 = e;
        g1 = g;
    }
};

// Is the centre of voxel (i, j, k), 16 * (i, j, k) + 8 in fixed point, inside
// the closed capsule?  Squared distance to the segment against r^2 without
// rounding: with s = (p-a).(b-a) and L = |b-a|^2 the nearest point is a
// (s <= 0), b (s >= L) or interior, where |p-a|^2 L - s^2 <= r^2 L.
__device__ __forceinline__ bool capsule_contains(const CapInfo &c, int i, int j, int k)
{
    const long long px = 16LL * i + 8, py = 16LL * j + 8, pz = 16LL * k + 8;
    const long long wx = px - c.a[0], wy = py - c.a[1], wz = pz - c.a[2];
    const long long dx = (long long)c.b[0] - c.a[0], dy = (long long)c.b[1] - c.a[1],
                    dz = (long long)c.b[2] - c.a[2];
    const long long L = dx * dx + dy * dy + dz * dz;
    const long long s = wx * dx + wy * dy + wz * dz;
    const long long r2 = (long long)c.r * c.r;
    if (c.cyl)  // projection on the segment, distance to the line at most r (L > 0)
        return s >= 0 && s <= L && (wx * wx + wy * wy + wz * wz) * L - s * s <= r2 * L;
    if (L == 0 || s <= 0)
        return wx * wx + wy * wy + wz * wz <= r2;
    if (s >= L) {
        const long long ex = px - c.b[0], ey = py - c.b[1], ez = pz - c.b[2];
        return ex * ex + ey * ey + ez * ez <= r2;
    }
    return (wx * wx + wy * wy + wz * wz) * L - s * s <= r2 * L;
}

// sign(S) * sqrt(|S|) * vox, IEEE round-to-nearest square root and product;
// +/-kInf32 -> +/-inf.  |S| < 2^24, so the int -> float conversion is exact.
__device__ __forceinline__ float sq_to_sdf(int32_t s, float vox)
{
    if (s == kInf32)
        return __int_as_float(0x7f800000);
    if (s == -kInf32)
        return __int_as_float(0xff800000);
    const int32_t a = s < 0 ? -s : s;
    const float m = __fmul_rn(__fsqrt_rn(__int2float_rn(a)), vox);
    return s < 0 ? -m : m;
}

// The same value as sq_to_sdf with a select instead of branches.
__device__ __forceinline__ float sq_to_sdf_fast(int32_t v, float vox)
{
    const int32_t a = v < 0 ? -v : v;
    float m = __fmul_rn(__fsqrt_rn(__int2float_rn(a)), vox);
    m = a == kInf32 ? __int_as_float(0x7f800000) : m;
    return __int_as_float(__float_as_int(m) | (v & (int32_t)0x80000000));
}

}  // namespace pcdf

// Surrogate distance queries with an exact fallback (sm_103a).
//
// The learned part predicts, per human capsule, the dynamic field value at a
// point; a query's distance is the min over the humans and the trilinear
// static field.  Where that prediction lies within `band` of the hinge
// threshold eps + r the prediction could flip the collision decision, so the
// query is answered exactly instead: the eight corner voxels of its cell get
// their exact composite values (static squared EDT from the static field; the
// dynamic squared EDT by a local search over the capsules' voxels, bounded as
// described at exact_dyn_sq) and are interpolated by the same code as the
// exact cost query, giving bit-identical results on those queries.
//
// Kernels:
//   k_sur_samples   training samples (features, target) drawn from exact
//                   dynamic fields with a counter-hash generator;
//   k_sur_features  query features, one row per (sphere, human);
//   k_sur_combine   min over humans and static field, hinge, fallback list;
//   k_sur_fallback  exact answers for the listed queries (warp per query).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "edt_common.cuh"
#include "host.h"
#include "trilinear.cuh"

using namespace pcdf::host;

namespace pcdf {
namespace sur {

using bf16 = __nv_bfloat16;
constexpr float kLen = 2.0f;  // metres: scale of the point-to-endpoint features

struct FeatGrid {
    QueryGrid g;
};

__device__ __forceinline__ float fixed_to_m(int32_t v, float origin, float vox)
{
    return __fadd_rn(origin, __fmul_rn((float)v, __fdiv_rn(vox, 16.f)));
}

// Continuous geometry of one capsule seen from point p (metres): the signed
// distance |p - n| - r to its surface (n the nearest axis point), the axis
// parameter of n in [0, 1] and the unit vector from n to p (zero on the axis).
struct CapGeo {
    float dist, s, u[3];
};

__device__ __forceinline__ CapGeo capsule_geo(const QueryGrid &g, const float (&p)[3], const int32_t *cap)
{
    float w[3], ab[3], L = 0.f, sd = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float am = fixed_to_m(cap[a], g.origin[a], g.vox);
        const float bm = fixed_to_m(cap[3 + a], g.origin[a], g.vox);
        w[a] = p[a] - am;
        ab[a] = bm - am;
        L += ab[a] * ab[a];
        sd += w[a] * ab[a];
    }
    CapGeo r;
    r.s = L > 0.f ? fminf(fmaxf(sd / L, 0.f), 1.f) : 0.f;
    float nn = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r.u[a] = w[a] - r.s * ab[a];
        nn += r.u[a] * r.u[a];
    }
    const float len = sqrtf(nn);
    const float inv = len > 1e-6f ? 1.f / len : 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        r.u[a] *= inv;
    r.dist = len - (float)cap[6] * (g.vox / 16.f);
    return r;
}

// Features of point p at time index t (horizon T) for one capsule: two
// zeros, the height of p above the grid floor in units of kLen, t scaled to
// [-1, 1], p - a and p - b in units of kLen, the radius in units of kLen, the
// continuous signed distance to the capsule in units of kLen and the axis
// parameter of its nearest point scaled to [-1, 1], then zeros.  Nothing but
// the floor fixes a position, so a network trained in one grid applies to
// any grid of the same voxel size.  The network's output is the exact
// field's departure from the continuous distance (its target in training).
__device__ __forceinline__ void features(const FeatGrid &G, const float (&p)[3], int t, int T, const int32_t *cap,
                                         const CapGeo &geo, bf16 *out)
{
    float f[16];
    f[0] = 0.f;
    f[1] = 0.f;
    f[2] = (p[2] - G.g.origin[2]) * (1.f / kLen);
    f[3] = T > 1 ? 2.f * (float)t / (float)(T - 1) - 1.f : 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f[4 + a] = (p[a] - fixed_to_m(cap[a], G.g.origin[a], G.g.vox)) * (1.f / kLen);
        f[7 + a] = (p[a] - fixed_to_m(cap[3 + a], G.g.origin[a], G.g.vox)) * (1.f / kLen);
    }
    f[10] = (float)cap[6] * (G.g.vox / 16.f) * (1.f / kLen);
    f[11] = geo.dist * (1.f / kLen);
    f[12] = 2.f * geo.s - 1.f;
#pragma unroll
    for (int a = 13; a < 16; ++a)
        f[a] = 0.f;
    bf16 h[16];
#pragma unroll
    for (int a = 0; a < 16; ++a)
        h[a] = __float2bfloat16_rn(f[a]);
    reinterpret_cast<uint4 *>(out)[0] = reinterpret_cast<const uint4 *>(h)[0];
    reinterpret_cast<uint4 *>(out)[1] = reinterpret_cast<const uint4 *>(h)[1];
}

__device__ __forceinline__ uint32_t hash32(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (uint32_t)(x >> 32);
}
__device__ __forceinline__ float uni(uint64_t seed, long long i, int k)
{
    return (hash32(seed ^ ((uint64_t)i * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)k << 56)) + 0.5f) *
           (1.f / 4294967296.f);
}

// Sample i: a field j (exact dynamic field of one capsule at time index tf[j]),
// a point uniform in the grid (probability 1 - near) or within 1 m of the
// capsule axis, the field's trilinear value there as the target.
__global__ void k_sur_samples(FeatGrid G, const float *__restrict__ fields, const int32_t *__restrict__ caps,
                              const int32_t *__restrict__ tf, int n_fields, int T, long long M,
                              unsigned long long seed, float near, bf16 *__restrict__ x, float *__restrict__ target)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M)
        return;
    const int j = min((int)(uni(seed, i, 0) * n_fields), n_fields - 1);
    const int32_t *cap = caps + 7 * j;
    const float ext[3] = {G.g.n[0] * G.g.vox, G.g.n[1] * G.g.vox, G.g.n[2] * G.g.vox};
    float p[3];
    if (uni(seed, i, 1) >= near) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            p[a] = G.g.origin[a] + uni(seed, i, 2 + a) * ext[a];
    } else {
        const float s = uni(seed, i, 2);
        const float u = 2.f * uni(seed, i, 3) - 1.f, phi = 6.2831853f * uni(seed, i, 4);
        const float rad = uni(seed, i, 5) * 1.0f;
        const float w = sqrtf(fmaxf(0.f, 1.f - u * u));
        const float dir[3] = {w * cosf(phi), w * sinf(phi), u};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float am = fixed_to_m(cap[a], G.g.origin[a], G.g.vox);
            const float bm = fixed_to_m(cap[3 + a], G.g.origin[a], G.g.vox);
            p[a] = am + s * (bm - am) + rad * dir[a];
            p[a] = fminf(fmaxf(p[a], G.g.origin[a]), G.g.origin[a] + ext[a]);
        }
    }
    const long long V = (long long)G.g.n[0] * G.g.n[1] * G.g.n[2];
    const Sample r = trilinear(G.g, fields + (long long)j * V, make_float4(p[0], p[1], p[2], 0.f), false);
    const CapGeo geo = capsule_geo(G.g, p, cap);
    target[i] = r.d - geo.dist;
    features(G, p, tf[j], T, cap, geo, x + i * 16);
}

__global__ void k_sur_features(FeatGrid G, const float4 *__restrict__ spheres, const int32_t *__restrict__ tidx,
                               long long N, int T, int H, const int32_t *__restrict__ caps, bf16 *__restrict__ x)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * H)
        return;
    const long long q = i / H;
    const int h = (int)(i % H);
    const float4 s = spheres[q];
    const int t = min(max(tidx[q], 0), T - 1);
    const float p[3] = {s.x, s.y, s.z};
    const int32_t *cap = caps + 7 * ((long long)t * H + h);
    features(G, p, t, T, cap, capsule_geo(G.g, p, cap), x + i * 16);
}

// Continuous signed distance |p - n| - r from point p (metres) to a capsule.
__device__ __forceinline__ float capsule_dist(const QueryGrid &g, const float (&p)[3], const int32_t *cap)
{
    float w[3], ab[3], L = 0.f, sd = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float am = fixed_to_m(cap[a], g.origin[a], g.vox);
        w[a] = p[a] - am;
        ab[a] = fixed_to_m(cap[3 + a], g.origin[a], g.vox) - am;
        L += ab[a] * ab[a];
        sd += w[a] * ab[a];
    }
    const float sp = L > 0.f ? fminf(fmaxf(sd / L, 0.f), 1.f) : 0.f;
    float nn = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = w[a] - sp * ab[a];
        nn += u * u;
    }
    return sqrtf(nn) - (float)cap[6] * (g.vox / 16.f);
}

constexpr float kCertMargin = 1e-4f;  // metres: covers the FP32 rounding of distances and interpolation
constexpr float kSqrt3 = 1.7320508f;

// Can the exact field of capsule cap (fixed point, 1/16 voxel from the grid
// corner) exceed the continuous distance at an exterior voxel centre by more
// than sqrt(3) voxels?  Not when the radius is at least sqrt(3)/2 voxels
// (some voxel centre lies within sqrt(3)/2 voxels of any point at that depth
// inside it) and the capsule lies inside the grid (that centre is a voxel of
// the grid).
__device__ __forceinline__ bool capsule_regular(const QueryGrid &g, const int32_t *cap)
{
    if (cap[6] < 14)  // 14/16 voxel > sqrt(3)/2 voxel
        return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long mn = (long long)min(cap[a], cap[3 + a]) - cap[6];
        const long long mx = (long long)max(cap[a], cap[3 + a]) + cap[6];
        if (mn < 0 || mx > 16LL * g.n[a])
            return false;
    }
    return true;
}

// The certificate of a query: exact bounds [d_lo, d_hi] on the exact path's
// distance d, from the exact static corners and bounds on the humans' exact
// field at the corners, plus which humans can lower the field at some corner.
//  * At a voxel centre c outside capsule k (continuous distance D > 0) the
//    exact field of the capsule's voxels is at least D (the nearest voxel
//    centre inside lies in the solid) and, for a regular capsule, at most
//    D + sqrt(3) vox (from the nearest surface point go sqrt(3)/2 vox inward:
//    the voxel holding that point has its centre inside the capsule).  The
//    humans' field outside them is the min over the capsules.
//  * At a centre inside (D <= 0) it is at most D (every free voxel centre lies
//    outside the solid, at least |D| away); no lower bound is used.
//  * The composite corner is min(static, humans) and the trilinear weights
//    are non-negative, so interpolating the corner bounds bounds d.
// A margin of kCertMargin on each side covers FP32 rounding.
struct Cert {
    float dlo, dhi;
    unsigned long long matters;  // bit k: capsule k can be below the static field at some corner
};

__device__ __forceinline__ Cert certify(const QueryGrid &g, const float *__restrict__ static_sdf, const Cell &cl,
                                        const float (&p)[3], const int32_t *caps_t, int H)
{
    const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
    float sc[2][2][2], lo[2][2][2], hi[2][2][2], smax = __int_as_float(0xff800000);
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                sc[dz][dy][dx] = __ldg(static_sdf + (dz ? cl.i1[2] : cl.i0[2]) * sz + (dy ? cl.i1[1] : cl.i0[1]) * sy +
                                       (dx ? cl.i1[0] : cl.i0[0]));
                smax = fmaxf(smax, sc[dz][dy][dx]);
                lo[dz][dy][dx] = hi[dz][dy][dx] = __int_as_float(0x7f800000);
            }
    // the largest distance from p to a corner of its cell
    float md2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float c0 = g.origin[a] + ((float)cl.i0[a] + 0.5f) * g.vox;
        const float c1 = g.origin[a] + ((float)cl.i1[a] + 0.5f) * g.vox;
        const float m = fmaxf(fabsf(p[a] - c0), fabsf(p[a] - c1));
        md2 += m * m;
    }
    const float reach = sqrtf(md2) + 2.f * kCertMargin;
    Cert r;
    r.matters = 0;
    const float ninf = __int_as_float(0xff800000), pinf = __int_as_float(0x7f800000);
    for (int k = 0; k < H; ++k) {
        const int32_t *cap = caps_t + 7 * k;
        // the continuous distance is 1-Lipschitz: if at p it exceeds zero and
        // every static corner value by the reach, every corner lies outside
        // the capsule with its lower end above the static value there, and
        // the capsule changes neither bound
        if (capsule_dist(g, p, cap) - reach > fmaxf(smax, 2.f * kCertMargin))
            continue;
        const bool reg = capsule_regular(g, cap);
        bool m = false;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const float c[3] = {g.origin[0] + ((float)(dx ? cl.i1[0] : cl.i0[0]) + 0.5f) * g.vox,
                                        g.origin[1] + ((float)(dy ? cl.i1[1] : cl.i0[1]) + 0.5f) * g.vox,
                                        g.origin[2] + ((float)(dz ? cl.i1[2] : cl.i0[2]) + 0.5f) * g.vox};
                    const float D = capsule_dist(g, c, cap);
                    const float l = D > kCertMargin ? D - kCertMargin : ninf;
                    const float u = reg ? D + kSqrt3 * g.vox + kCertMargin : (D < -kCertMargin ? D + kCertMargin : pinf);
                    lo[dz][dy][dx] = fminf(lo[dz][dy][dx], l);
                    hi[dz][dy][dx] = fminf(hi[dz][dy][dx], u);
                    m |= l < sc[dz][dy][dx];
                }
        if (m)
            r.matters |= 1ull << k;
    }
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                lo[dz][dy][dx] = fminf(sc[dz][dy][dx], lo[dz][dy][dx]);
                hi[dz][dy][dx] = fminf(sc[dz][dy][dx], hi[dz][dy][dx]);
            }
    r.dlo = interpolate(cl, lo, false).d - kCertMargin;
    r.dhi = interpolate(cl, hi, false).d + kCertMargin;
    return r;
}

// Rows (sphere q, capsule k) that need the network, from the certificate of
// query q: capsules that cannot be below the static field at any corner of
// the cell never need it (the row is skipped, y_index -1, and the capsule
// counts as +INF).  mode 0 (the certified query): rows only of queries whose
// decision is certainly active (d_hi < eps + r), the only ones whose cost uses
// the network's value; mode 1: every row where the capsule can matter (to
// measure the network).  Rows get their features at slots taken in warp
// order; bounds[q] = (d_lo, d_hi).
__global__ void k_sur_select(FeatGrid G, const float *__restrict__ static_sdf, const float4 *__restrict__ spheres,
                             const int32_t *__restrict__ tidx, long long N, int T, int H,
                             const int32_t *__restrict__ caps, float eps, int mode, bf16 *__restrict__ x,
                             int32_t *__restrict__ y_index, int *__restrict__ count, float2 *__restrict__ bounds)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long need = 0;
    float p[3] = {0.f, 0.f, 0.f};
    int t = 0;
    if (q < N) {
        const float4 s = spheres[q];
        t = min(max(tidx[q], 0), T - 1);
        p[0] = s.x;
        p[1] = s.y;
        p[2] = s.z;
        const Cell cl = locate(G.g, s);
        const Cert c = certify(G.g, static_sdf, cl, p, caps + 7LL * t * H, H);
        bounds[q] = make_float2(c.dlo, c.dhi);
        need = c.matters;
        if (mode == 0 && !(c.dhi < eps + s.w))
            need = 0;
    }
    // slots: one atomic per warp, rows in lane order
    const int lane = threadIdx.x & 31;
    const int cnt = __popcll(need);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int base = 0;
    if (total) {
        if (lane == 31)
            base = atomicAdd(count, total);
        base = __shfl_sync(0xffffffffu, base, 31);
    }
    if (q < N) {
        int slot = base + incl - cnt;
        for (int k = 0; k < H; ++k) {
            const int32_t *cap = caps + 7 * ((long long)t * H + k);
            if ((need >> k) & 1ull) {
                y_index[q * H + k] = slot;
                features(G, p, t, T, cap, capsule_geo(G.g, p, cap), x + (long long)slot * 16);
                ++slot;
            } else {
                y_index[q * H + k] = -1;
            }
        }
    }
}

// The prediction is made like the exact distance: the eight corners of the
// query's cell get min(static corner value, predicted dynamic value there) and
// are interpolated.  The dynamic value of a capsule at the point is its
// continuous distance plus the network's output (the learned departure of the
// exact voxel field from it); at a corner it is extrapolated along the
// capsule's distance gradient (the unit vector from the nearest axis point),
// then the min over humans.  Capsules without a row count as +INF.
//
// With the certificate (bounds, from k_sur_select): the prediction is clamped
// to [d_lo, d_hi]; a query whose threshold eps + r lies inside the interval
// (the decision is not certain) is answered exactly, and so is a certainly
// active query whose prediction lies within `band` of the threshold.  Every
// other decision is the exact one by construction.  Without it (bounds NULL,
// to measure the network): a query with some row is answered exactly when
// the prediction lies within `band` of the threshold; a query without rows
// has the static field as its exact distance.
__global__ void k_sur_combine(QueryGrid g, const float *__restrict__ static_sdf, const float4 *__restrict__ spheres,
                              const int32_t *__restrict__ tidx, int T, const CapInfo *__restrict__ caps, long long N,
                              int H, const float *__restrict__ y, const int32_t *__restrict__ y_index,
                              const float2 *__restrict__ bounds, float eps, float band,
                              float *__restrict__ h, float *__restrict__ d_out, int *__restrict__ list,
                              int *__restrict__ count)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool fb = false;
    if (q < N) {
        const float4 s = spheres[q];
        const int t = min(max(tidx[q], 0), T - 1);
        const Cell cl = locate(g, s);
        const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
        float c[2][2][2], dync[2][2][2];
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    c[dz][dy][dx] = __ldg(static_sdf + (dz ? cl.i1[2] : cl.i0[2]) * sz + (dy ? cl.i1[1] : cl.i0[1]) * sy +
                                          (dx ? cl.i1[0] : cl.i0[0]));
                    dync[dz][dy][dx] = __int_as_float(0x7f800000);
                }
        const float p[3] = {s.x, s.y, s.z};
        bool rows = false;
        for (int k = 0; k < H; ++k) {
            const long long yi = y_index ? (long long)y_index[q * H + k] : q * H + k;
            if (yi < 0)
                continue;  // the static field wins in the cell whatever this capsule
            rows = true;
            const CapInfo &C = caps[(long long)t * H + k];
            const int32_t cp[7] = {C.a[0], C.a[1], C.a[2], C.b[0], C.b[1], C.b[2], C.r};
            const CapGeo geo = capsule_geo(g, p, cp);
            const float yk = y[yi] + geo.dist;  // residual + continuous distance
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        const int iv[3] = {dx ? cl.i1[0] : cl.i0[0], dy ? cl.i1[1] : cl.i0[1], dz ? cl.i1[2] : cl.i0[2]};
                        float proj = 0.f;
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            proj += geo.u[a] * (g.origin[a] + ((float)iv[a] + 0.5f) * g.vox - p[a]);
                        dync[dz][dy][dx] = fminf(dync[dz][dy][dx], yk + proj);
                    }
        }
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx)
                    c[dz][dy][dx] = fminf(c[dz][dy][dx], dync[dz][dy][dx]);
        float d = interpolate(cl, c, false).d;
        const float thr = eps + s.w;
        if (bounds) {
            const float2 b = bounds[q];
            d = fminf(fmaxf(d, b.x), b.y);
            const bool inactive = thr <= b.x, active = b.y < thr;
            fb = !(inactive || active) || (active && rows && fabsf(d - thr) < band);
        } else {
            fb = rows && fabsf(d - thr) < band;
        }
        const float hv = thr - d;
        h[q] = hv > 0.f ? hv : 0.f;
        if (d_out)
            d_out[q] = d;
    }
    // warp-aggregated append to the fallback list
    const unsigned m = __ballot_sync(0xffffffffu, fb);
    if (m) {
        const int lane = threadIdx.x & 31;
        int base = 0;
        if (lane == __ffs(m) - 1)
            base = atomicAdd(count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (fb)
            list[base + __popc(m & ((1u << lane) - 1u))] = (int)q;
    }
}

// --- exact dynamic squared distances at the corners of a cell -----------

__device__ __forceinline__ int warp_min(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ bool inside_any(const CapInfo *caps, int H, int i, int j, int k)
{
    for (int c = 0; c < H; ++c)
        if (caps[c].lo[0] <= caps[c].hi[0] && capsule_contains(caps[c], i, j, k))
            return true;
    return false;
}

// For every voxel u of the box [lo, hi] with pred(u), lower best[c] to
// |v_c - u|^2 for the corners c in `mask`.  Lanes take the x positions of a
// row; rows are walked in order; the minima are reduced over the warp.
template <class Pred>
__device__ __forceinline__ void scan_box(const int (&v)[8][3], unsigned mask, const int (&lo)[3], const int (&hi)[3],
                                         int (&best)[8], Pred pred)
{
    const int lane = threadIdx.x & 31;
    for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0] + lane; i <= hi[0]; i += 32) {
                if (!pred(i, j, k))
                    continue;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (!((mask >> c) & 1u))
                        continue;
                    const int d = (i - v[c][0]) * (i - v[c][0]) + (j - v[c][1]) * (j - v[c][1]) +
                                  (k - v[c][2]) * (k - v[c][2]);
                    best[c] = min(best[c], d);
                }
            }
#pragma unroll
    for (int c = 0; c < 8; ++c)
        best[c] = warp_min(best[c]);
}

// Exact dynamic squared EDT (signed, as the composite kernels) at the eight
// corners v_c of a cell.
//
// A corner outside every capsule: min over the capsules C of the squared
// distance to C's voxels.  If q is the point of C nearest to v's centre at
// continuous distance d (voxel units), every point u of the convex capsule
// satisfies |v - u|^2 >= d^2 + |u - q|^2, and some voxel of C lies within
// d + sqrt(3) of v (a ball of radius sqrt(3)/2 around the point sqrt(3)/2
// inside q holds a lattice point when r >= sqrt(3)/2), so the nearest voxel
// lies within sqrt((d + sqrt(3))^2 - d^2) of q.  One box covers those balls
// for all eight corners with a margin; capsules that are thin, cut by the grid
// boundary, or whose result breaks the d + sqrt(3) bound at some corner are
// searched over their whole in-grid bounding box instead.
// A corner inside some capsule: minus the squared distance to the nearest
// voxel outside all capsules, searched in growing cube shells.
__device__ void exact_cell_dyn(const QueryGrid &g, const CapInfo *caps, int H, const int (&v)[8][3], int (&out)[8])
{
    const int n[3] = {g.n[0], g.n[1], g.n[2]};
    unsigned ext = 0;
    for (int c = 0; c < 8; ++c) {
        out[c] = kInf32;
        if (!inside_any(caps, H, v[c][0], v[c][1], v[c][2]))
            ext |= 1u << c;
    }
    // interior corners (rare: corners within the humans)
    for (int c = 0; c < 8; ++c) {
        if ((ext >> c) & 1u)
            continue;
        int best[8];
        for (int q = 0; q < 8; ++q)
            best[q] = kInf32;
        for (int rad = 1; rad <= max(n[0], max(n[1], n[2])); ++rad) {
            if (best[c] != kInf32 && (long long)rad * rad >= best[c])
                break;
            for (int face = 0; face < 6; ++face) {
                const int ax = face >> 1, sg = (face & 1) ? 1 : -1;
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    lo[a] = max(v[c][a] - rad, 0);
                    hi[a] = min(v[c][a] + rad, n[a] - 1);
                }
                const int f = v[c][ax] + sg * rad;
                if (f < 0 || f > n[ax] - 1)
                    continue;
                lo[ax] = hi[ax] = f;
                scan_box(v, 1u << c, lo, hi, best, [&](int i, int j, int k) { return !inside_any(caps, H, i, j, k); });
            }
        }
        out[c] = best[c] == kInf32 ? -kInf32 : -best[c];
    }
    if (!ext)
        return;
    for (int cc = 0; cc < H; ++cc) {
        const CapInfo &C = caps[cc];
        if (C.lo[0] > C.hi[0])
            continue;
        bool full = C.r < 14;  // r < sqrt(3)/2 voxel, in 16ths
        for (int a = 0; a < 3; ++a) {
            const int mn = min(C.a[a], C.b[a]) - C.r, mx = max(C.a[a], C.b[a]) + C.r;
            const int ulo = (mn - 8 + 15 + 16 * 4096) / 16 - 4096, uhi = (mx - 8 + 16 * 4096) / 16 - 4096;
            full |= ulo < 0 || uhi > n[a] - 1;  // cut by the grid boundary
        }
        int best[8];
        for (int c = 0; c < 8; ++c)
            best[c] = kInf32;
        float bound[8];
        if (!full) {
            int lo[3] = {1 << 20, 1 << 20, 1 << 20}, hi[3] = {-(1 << 20), -(1 << 20), -(1 << 20)};
            const float ab[3] = {(float)(C.b[0] - C.a[0]), (float)(C.b[1] - C.a[1]), (float)(C.b[2] - C.a[2])};
            const float L = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
            for (int c = 0; c < 8; ++c) {
                bound[c] = 0.f;
                if (!((ext >> c) & 1u))
                    continue;
                const float pv[3] = {16.f * v[c][0] + 8.f, 16.f * v[c][1] + 8.f, 16.f * v[c][2] + 8.f};
                float w[3], s = 0.f;
                for (int a = 0; a < 3; ++a) {
                    w[a] = pv[a] - (float)C.a[a];
                    s += w[a] * ab[a];
                }
                const float tpar = L > 0.f ? fminf(fmaxf(s / L, 0.f), 1.f) : 0.f;
                float q[3], dd = 0.f;
                for (int a = 0; a < 3; ++a) {
                    q[a] = (float)C.a[a] + tpar * ab[a];
                    dd += (pv[a] - q[a]) * (pv[a] - q[a]);
                }
                const float dist = sqrtf(dd);
                const float dv = fmaxf(dist - (float)C.r, 0.f) / 16.f;  // voxel units
                bound[c] = dv + 1.7320508f + 0.01f;
                const float R = sqrtf(2.f * 1.7320508f * dv + 3.f) + 2.f;
                for (int a = 0; a < 3; ++a) {
                    const float qs = dist > 0.f ? q[a] + (pv[a] - q[a]) * ((float)C.r / dist) : q[a];
                    const float qv = (qs - 8.f) / 16.f;
                    lo[a] = min(lo[a], (int)floorf(qv - R));
                    hi[a] = max(hi[a], (int)ceilf(qv + R));
                }
            }
            for (int a = 0; a < 3; ++a) {
                lo[a] = max(lo[a], C.lo[a]);
                hi[a] = min(hi[a], C.hi[a]);
            }
            scan_box(v, ext, lo, hi, best, [&](int i, int j, int k) { return capsule_contains(C, i, j, k); });
            for (int c = 0; c < 8; ++c)
                if (((ext >> c) & 1u) && (best[c] == kInf32 || (float)best[c] > bound[c] * bound[c]))
                    full = true;
        }
        if (full) {
            for (int c = 0; c < 8; ++c)
                best[c] = kInf32;
            const int lo[3] = {C.lo[0], C.lo[1], C.lo[2]}, hi[3] = {C.hi[0], C.hi[1], C.hi[2]};
            scan_box(v, ext, lo, hi, best, [&](int i, int j, int k) { return capsule_contains(C, i, j, k); });
        }
        for (int c = 0; c < 8; ++c)
            if ((ext >> c) & 1u)
                out[c] = min(out[c], best[c]);
    }
}

__global__ void k_sur_fallback(QueryGrid g, const int32_t *__restrict__ static_sq,
                               const float *__restrict__ static_sdf, const float4 *__restrict__ spheres,
                               const int32_t *__restrict__ tidx, int T, int H, const CapInfo *__restrict__ caps,
                               float eps, const int *__restrict__ list, const int *__restrict__ count,
                               float *__restrict__ h, float *__restrict__ d_out)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int n = *count;
    for (long long w = warp; w < n; w += nwarps) {
        const long long q = list[w];
        const float4 s = spheres[q];
        const int t = min(max(tidx[q], 0), T - 1);
        const Cell cl = locate(g, s);
        int v[8][3];
        for (int c = 0; c < 8; ++c) {
            v[c][0] = (c & 1) ? cl.i1[0] : cl.i0[0];
            v[c][1] = (c & 2) ? cl.i1[1] : cl.i0[1];
            v[c][2] = (c & 4) ? cl.i1[2] : cl.i0[2];
        }
        int dyn[8];
        exact_cell_dyn(g, caps + (long long)t * H, H, v, dyn);
        if (lane == 0) {
            float c[2][2][2];
            for (int k = 0; k < 8; ++k) {
                const long long o = ((long long)v[k][2] * g.n[1] + v[k][1]) * g.n[0] + v[k][0];
                const int32_t sv = static_sq[o];
                c[(k >> 2) & 1][(k >> 1) & 1][k & 1] = sv <= dyn[k] ? static_sdf[o] : sq_to_sdf_fast(min(sv, dyn[k]), g.vox);
            }
            const Sample r = interpolate(cl, c, false);
            const float hv = (eps + s.w) - r.d;
            h[q] = hv > 0.f ? hv : 0.f;
            if (d_out)
                d_out[q] = r.d;
        }
    }
}

// The same exact answers from the 2-D partial field of the capsule slab that
// pcdf_composite_prepare leaves in its workspace (dyn_mid[t][e][y][x] for the
// slab slices zlo + e, e < S).  The dynamic value at a corner voxel is the
// lower envelope of its column evaluated directly: outside the humans min
// over slab slices z' of (z - z')^2 + g(z') (g the partial at a free voxel,
// 0 at an occupied one); inside, minus min over the column of (z - z')^2 +
// g(z') with g = 0 at free voxels (the slab's and the first ones beyond it)
// and minus the partial at occupied ones.  The minima are the ones the
// composite z pass takes, so the values are the same integers.
// Four lanes per query, one per column of the cell (x bit 0, y bit 1), both
// corner heights z0 and z1 = z0 (+ 1) at once.  Every term is at least
// (z - z')^2, so each lane visits the slices in order of distance from the
// corner pair (z0 - k below, z0 + 1 + k above) and stops once (k + 1)^2
// reaches both minima; the quad's eight corner values meet in its first lane
// for the interpolation.
__global__ void k_sur_fallback_slab(QueryGrid g, const int32_t *__restrict__ static_sq,
                                    const float *__restrict__ static_sdf, const float4 *__restrict__ spheres,
                                    const int32_t *__restrict__ tidx, int T, const int32_t *__restrict__ dyn_mid,
                                    const __grid_constant__ pcdf::SlabMap map, int zlo, int S, float eps,
                                    const int *__restrict__ list, const int *__restrict__ count,
                                    float *__restrict__ h, float *__restrict__ d_out)
{
    const int lane = threadIdx.x & 31, col = lane & 3;
    const long long gq = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 2;  // this quad's first query
    const long long nq = ((long long)gridDim.x * blockDim.x) >> 2;
    const long long V2 = (long long)g.n[0] * g.n[1];
    const int nz = g.n[2];
    const int n = *count;
    for (long long w = gq;; w += nq) {
        // the loop ends for the whole warp at once (shuffles below)
        if (w - (lane >> 2) >= n)
            break;
        const bool valid = w < n;
        const long long q = list[valid ? w : w - (lane >> 2)];
        const float4 s = spheres[q];
        const int t = min(max(tidx[q], 0), T - 1);
        const Cell cl = locate(g, s);
        const int x = (col & 1) ? cl.i1[0] : cl.i0[0], y = (col & 2) ? cl.i1[1] : cl.i0[1];
        const int32_t *pc = dyn_mid + (long long)t * S * V2 + (long long)y * g.n[0] + x;  // slice e at pc[e * V2]
        const uint8_t *rp = map.on ? map.rep + t * S : nullptr;  // slab element e is stored in slice rp[e]
        auto slab = [&](int e) { return __ldg(pc + (long long)(rp ? rp[e] : e) * V2); };
        const int zc[2] = {cl.i0[2], cl.i1[2]};
        bool inside[2];
        int best[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = zc[u] - zlo;
            inside[u] = e >= 0 && e < S && slab(e) < 0;
            best[u] = kInf32;
            if (inside[u]) {
                // the free voxels next to the slab
                if (zlo - 1 >= 0)
                    best[u] = min(best[u], (zc[u] - (zlo - 1)) * (zc[u] - (zlo - 1)));
                if (zlo + S < nz)
                    best[u] = min(best[u], (zlo + S - zc[u]) * (zlo + S - zc[u]));
            }
        }
        auto visit = [&](int e, int32_t P) {
            const int zz = zlo + e;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int dz2 = (zc[u] - zz) * (zc[u] - zz);
                if (inside[u]) {
                    if (P >= 0)
                        best[u] = min(best[u], dz2);  // a free voxel
                    else if (P != -kInf32)
                        best[u] = min(best[u], dz2 - P);
                } else {
                    if (P < 0)
                        best[u] = min(best[u], dz2);  // an occupied voxel
                    else if (P != kInf32)
                        best[u] = min(best[u], dz2 + P);
                }
            }
        };
        const int ec = zc[0] - zlo;
        // k runs until both sides have left the slab; four steps (eight
        // slices) are loaded before they are folded in
        const int kmax = max(ec + 1, S - ec);
        for (int k0 = 0; k0 < kmax; k0 += 4) {
            const long long bound = (long long)k0 * k0;  // every slice not yet visited is >= k0 away
            if (bound >= (long long)max(best[0], best[1]))
                break;
            int32_t P[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int ea = ec - k0 - i, eb = ec + 1 + k0 + i;
                P[2 * i] = (ea >= 0 && ea < S) ? slab(ea) : kInf32;
                P[2 * i + 1] = (eb >= 0 && eb < S) ? slab(eb) : kInf32;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int ea = ec - k0 - i, eb = ec + 1 + k0 + i;
                if (ea >= 0 && ea < S)
                    visit(ea, P[2 * i]);
                if (eb >= 0 && eb < S)
                    visit(eb, P[2 * i + 1]);
            }
        }
        // this lane's two corners (x, y of its column; z0 and z1)
        float cv[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            int b = best[u];
            if (inside[u])
                b = b == kInf32 ? -kInf32 : -b;
            const long long o = ((long long)zc[u] * g.n[1] + y) * g.n[0] + x;
            const int32_t sv = __ldg(static_sq + o);
            cv[u] = sv <= b ? __ldg(static_sdf + o) : sq_to_sdf_fast(min(sv, b), g.vox);
        }
        float c[2][2][2];
        const int base = lane & ~3;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            c[0][k >> 1][k & 1] = __shfl_sync(0xffffffffu, cv[0], base + k);
            c[1][k >> 1][k & 1] = __shfl_sync(0xffffffffu, cv[1], base + k);
        }
        if (valid && col == 0) {
            const Sample r = interpolate(cl, c, false);
            const float hv = (eps + s.w) - r.d;
            h[q] = hv > 0.f ? hv : 0.f;
            if (d_out)
                d_out[q] = r.d;
        }
    }
}

FeatGrid feat_grid(const pcdf_grid *grid)
{
    FeatGrid G;
    G.g.n[0] = grid->nx;
    G.g.n[1] = grid->ny;
    G.g.n[2] = grid->nz;
    for (int a = 0; a < 3; ++a)
        G.g.origin[a] = grid->origin[a];
    G.g.vox = grid->vox;
    return G;
}

}  // namespace sur
}  // namespace pcdf

using namespace pcdf::sur;

extern "C" {

int pcdf_surrogate_samples(const pcdf_grid *grid, const float *fields, const int32_t *caps, const int32_t *tf,
                           int32_t n_fields, int32_t T, int64_t M, uint64_t seed, float near, uint16_t *x,
                           float *target, void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (!fields || !caps || !tf || !x || !target || n_fields < 1 || T < 1 || M < 0)
        return fail(PCDF_EINVAL, "bad surrogate sample arguments");
    if (!aligned(x, 16))
        return fail(PCDF_EINVAL, "x must be 16-byte aligned");
    if (M == 0)
        return PCDF_OK;
    k_sur_samples<<<(unsigned)((M + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        feat_grid(grid), fields, caps, tf, n_fields, T, M, (unsigned long long)seed, near, (bf16 *)x, target);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "surrogate samples");
}

int pcdf_surrogate_features(const pcdf_grid *grid, const float *spheres, const int32_t *tidx, int64_t N, int32_t T,
                            int32_t H, const int32_t *caps, uint16_t *x, void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (N < 0 || T < 1 || H < 1 || (N > 0 && (!spheres || !tidx || !caps || !x)))
        return fail(PCDF_EINVAL, "bad surrogate feature arguments");
    if (!aligned(spheres, 16) || !aligned(x, 16))
        return fail(PCDF_EINVAL, "spheres and x must be 16-byte aligned");
    const long long R = N * H;
    if (R == 0)
        return PCDF_OK;
    k_sur_features<<<(unsigned)((R + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        feat_grid(grid), (const float4 *)spheres, tidx, N, T, H, caps, (bf16 *)x);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "surrogate features");
}

int pcdf_surrogate_select(const pcdf_grid *grid, const float *static_sdf, const float *spheres, const int32_t *tidx,
                          int64_t N, int32_t T, int32_t H, const int32_t *caps, float eps, int32_t mode, uint16_t *x,
                          int32_t *y_index, int32_t *count, float *bounds, void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (N < 0 || T < 1 || H < 1 || H > 64 || !count || (mode != 0 && mode != 1) ||
        (N > 0 && (!static_sdf || !spheres || !tidx || !caps || !x || !y_index || !bounds)))
        return fail(PCDF_EINVAL, "bad surrogate selection arguments");
    if (!std::isfinite(eps))
        return fail(PCDF_EINVAL, "eps must be finite");
    if (N > 0 && !aligned(bounds, 8))
        return fail(PCDF_EINVAL, "bounds must be 8-byte aligned");
    if (!aligned(spheres, 16) || !aligned(x, 16))
        return fail(PCDF_EINVAL, "spheres and x must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t), st);
    if (e != cudaSuccess)
        return cuda_fail(e, "surrogate selection");
    if (N == 0)
        return PCDF_OK;
    k_sur_select<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(feat_grid(grid), static_sdf, (const float4 *)spheres, tidx,
                                                             N, T, H, caps, eps, mode, (bf16 *)x, y_index, count,
                                                             (float2 *)bounds);
    e = cudaGetLastError();
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "surrogate selection");
}

int pcdf_surrogate_finish_workspace_bytes(int32_t T, int32_t H, int64_t N, size_t *bytes)
{
    if (!bytes || T < 1 || H < 1 || N < 0)
        return fail(PCDF_EINVAL, "bad arguments");
    *bytes = align_up(sizeof(int)) + align_up((size_t)N * sizeof(int)) + align_up((size_t)T * H * sizeof(pcdf::CapInfo));
    return PCDF_OK;
}

}  // extern "C"

namespace {

// capsules into the workspace from a kernel parameter: the values are copied
// at launch (and captured by value in a CUDA graph), so the host array may go
// as soon as the call returns
__global__ void k_put_caps(const __grid_constant__ pcdf::CapBatch b, pcdf::CapInfo *__restrict__ dst)
{
    for (int i = threadIdx.x; i < b.count; i += blockDim.x)
        dst[i] = b.caps[i];
}

// combine, then the exact answers: from the capsule slab's 2-D partials when
// dyn_mid is given, else by local search over the capsules' voxels
int surrogate_finish(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf, const float *spheres,
                     const int32_t *tidx, int64_t N, int32_t T, int32_t H, const int32_t *caps_host,
                     const int32_t *dyn_mid, const pcdf::SlabMap *map, int zlo_slab, int S_slab, const float *y,
                     const int32_t *y_index, const float *bounds, float eps, float band, float *h, float *d_out,
                     int32_t *n_fallback, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!static_sq || !static_sdf || !spheres || !tidx || !y || !h || !workspace)
        return fail(PCDF_EINVAL, "required pointer is NULL");
    if (bounds && !aligned(bounds, 8))
        return fail(PCDF_EINVAL, "bounds must be 8-byte aligned");
    if (!aligned(spheres, 16) || !aligned(workspace, kAlign))
        return fail(PCDF_EINVAL, "spheres must be 16-byte aligned, workspace %zu-byte aligned", kAlign);
    size_t need = 0;
    pcdf_surrogate_finish_workspace_bytes(T, H, N, &need);
    if (workspace_bytes < need)
        return fail(PCDF_ENOMEM, "workspace %zu bytes < %zu needed", workspace_bytes, need);
    std::vector<pcdf::CapInfo> ci;
    int zlo = 0, zhi = -1;
    if (int rc = make_capinfo(grid, T, H, caps_host, ci, &zlo, &zhi))
        return rc;
    for (const pcdf::CapInfo &c : ci)
        if (c.cyl)
            return fail(PCDF_EINVAL, "the surrogate models capsules only (a cylinder was given)");
    char *ws = (char *)workspace;
    int *count = (int *)ws;
    int *list = (int *)(ws + align_up(sizeof(int)));
    pcdf::CapInfo *dcaps = (pcdf::CapInfo *)(ws + align_up(sizeof(int)) + align_up((size_t)N * sizeof(int)));
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), st);
    for (size_t i0 = 0; e == cudaSuccess && i0 < ci.size(); i0 += pcdf::kMaxCapsPerLaunch) {
        static thread_local pcdf::CapBatch batch;  // 24 KB: kept off the stack
        const size_t n = std::min(ci.size() - i0, (size_t)pcdf::kMaxCapsPerLaunch);
        batch.count = (int32_t)n;
        std::copy(ci.begin() + i0, ci.begin() + i0 + n, batch.caps);
        k_put_caps<<<1, 128, 0, st>>>(batch, dcaps + i0);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "surrogate setup");
    const FeatGrid G = feat_grid(grid);
    k_sur_combine<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(G.g, static_sdf, (const float4 *)spheres, tidx, T,
                                                              dcaps, N, H, y, y_index, (const float2 *)bounds, eps, band,
                                                              h, d_out, list, count);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dyn_mid)
        k_sur_fallback_slab<<<sms * 8, 256, 0, st>>>(G.g, static_sq, static_sdf, (const float4 *)spheres, tidx, T,
                                                    dyn_mid, *map, zlo_slab, S_slab, eps, list, count, h, d_out);
    else
        k_sur_fallback<<<sms * 8, 256, 0, st>>>(G.g, static_sq, static_sdf, (const float4 *)spheres, tidx, T, H,
                                               dcaps, eps, list, count, h, d_out);
    if (n_fallback)
        e = cudaMemcpyAsync(n_fallback, count, sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "surrogate finish");
}

}  // namespace

extern "C" {

int pcdf_surrogate_finish(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf,
                          const float *spheres, const int32_t *tidx, int64_t N, int32_t T, int32_t H,
                          const int32_t *caps_host, const float *y, const int32_t *y_index, const float *bounds,
                          float eps, float band, float *h, float *d_out, int32_t *n_fallback, void *workspace,
                          size_t workspace_bytes, void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (N < 0 || T < 1 || H < 1 || !caps_host)
        return fail(PCDF_EINVAL, "bad surrogate arguments");
    if (N == 0)
        return PCDF_OK;
    return surrogate_finish(grid, static_sq, static_sdf, spheres, tidx, N, T, H, caps_host, nullptr, nullptr, 0, 0, y,
                            y_index, bounds, eps, band, h, d_out, n_fallback, workspace, workspace_bytes, stream);
}

int pcdf_surrogate_finish_slab(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf,
                               const float *spheres, const int32_t *tidx, int64_t N, int32_t T, int32_t H,
                               const int32_t *caps_host, const void *comp_workspace, size_t comp_workspace_bytes,
                               const float *y, const int32_t *y_index, const float *bounds, float eps, float band,
                               float *h, float *d_out, int32_t *n_fallback, void *workspace, size_t workspace_bytes,
                               void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (N < 0 || T < 1 || H < 1 || !caps_host)
        return fail(PCDF_EINVAL, "bad surrogate arguments");
    CompositePlan p;
    if (int rc = plan_composite(grid, T, H, caps_host, p))
        return rc;
    if (int rc = check_ws(p, const_cast<void *>(comp_workspace), comp_workspace_bytes))
        return rc;
    if (N == 0)
        return PCDF_OK;
    const int32_t *mid = p.S > 0 ? plan_mid(p, const_cast<void *>(comp_workspace)) : nullptr;
    // no capsule in the grid: the dynamic field is +INF everywhere (an empty slab)
    static const int32_t none = 0;
    // the slices of equal capsule cross-sections that the prepare stage computed once
    static thread_local pcdf::SlabMap map;
    slab_map(p, map);
    return surrogate_finish(grid, static_sq, static_sdf, spheres, tidx, N, T, H, caps_host, mid ? mid : &none, &map,
                            p.zlo, p.S, y, y_index, bounds, eps, band, h, d_out, n_fallback, workspace,
                            workspace_bytes, stream);
}

}  // extern "C"

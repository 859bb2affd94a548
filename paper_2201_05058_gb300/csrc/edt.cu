// Exact signed squared Euclidean distance transform on sm_103a.
//
// The transform is separable: a row pass along x gives, per voxel, the 1-D
// distance to the nearest voxel of the other state; two lower-envelope passes
// (y, then z) turn it into the exact 3-D squared distance (the separable exact
// EDT of Meijster et al. / Felzenszwalb-Huttenlocher; the paper's own system
// uses the Parallel Banding Algorithm, Sec. 6).  Both site sets are carried in
// one signed value per voxel: its sign is the voxel's own state and its
// magnitude the partial distance to the other state, because each voxel is a
// zero-distance site of its own set.
//
// The composite fields of Sec. 6 (per-voxel min of the static field and the
// field of the humans at each predicted time, Sec. 8) come out of one fused
// z-pass that reads the static field once per column block, runs the dynamic
// envelope over the z-slab that the capsules touch, takes the min and writes
// the int32 and fp32 fields for every t.
//
// All arithmetic is integer except the IEEE sqrt and product of the float
// epilogue, so the results are bit-exact.
#include <cuda_runtime.h>

#include "pcdf_internal.cuh"

namespace pcdf {
namespace {

constexpr int kBig = 1 << 20;  // "no site" offset, beyond any grid coordinate
constexpr int kRowWarps = 8;   // rows (one warp each) per CTA of the row pass
constexpr uint32_t kG22 = (1u << 22) - 1;

// ---------------------------------------------------------------------------
// capsule test (exact, int64)
// ---------------------------------------------------------------------------

// Is the centre of voxel (i, j, k) inside the closed capsule?  The squared
// distance from p to the segment is compared with r^2 without rounding: with
// s = (p-a).(b-a) and L = |b-a|^2 the nearest point is a (s <= 0), b (s >= L)
// or interior, where |p-a|^2 L - s^2 <= r^2 L.
__device__ __forceinline__ bool capsule_contains(const CapInfo &c, int i, int j, int k)
{
    const long long px = 16LL * i + 8, py = 16LL * j + 8, pz = 16LL * k + 8;
    const long long wx = px - c.a[0], wy = py - c.a[1], wz = pz - c.a[2];
    const long long dx = (long long)c.b[0] - c.a[0], dy = (long long)c.b[1] - c.a[1],
                    dz = (long long)c.b[2] - c.a[2];
    const long long L = dx * dx + dy * dy + dz * dz;
    const long long s = wx * dx + wy * dy + wz * dz;
    const long long r2 = (long long)c.r * c.r;
    if (L == 0 || s <= 0)
        return wx * wx + wy * wy + wz * wz <= r2;
    if (s >= L) {
        const long long ex = px - c.b[0], ey = py - c.b[1], ez = pz - c.b[2];
        return ex * ex + ey * ey + ez * ez <= r2;
    }
    return (wx * wx + wy * wy + wz * wz) * L - s * s <= r2 * L;
}

__device__ __forceinline__ float sq_to_sdf(int32_t s, float vox)
{
    if (s == kInf32)
        return __int_as_float(0x7f800000);
    if (s == -kInf32)
        return __int_as_float(0xff800000);
    const int32_t a = s < 0 ? -s : s;
    const float m = __fmul_rn(__fsqrt_rn(__int2float_rn(a)), vox);  // |S| < 2^24: exact conversion
    return s < 0 ? -m : m;
}

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

// ---------------------------------------------------------------------------
// lower-envelope pass (y or z)
// ---------------------------------------------------------------------------
// Thread (column c, site set).  Set O (sites: occupied voxels) outputs at free
// voxels, set F (sites: free voxels) at occupied voxels.  The input value v of
// element e carries the previous passes: g_O(e) = 0 if e is occupied, else the
// squared partial distance |v| (none if infinite); symmetrically for F.
//
// Each thread keeps its envelope as a stack in shared memory, one packed word
// (site << 22 | g) per entry, laid out [entry][thread] so that every access is
// bank-conflict free.  Sites are pushed in increasing order; the top site s1
// (with predecessor s0) is popped when the new site e makes it useless, i.e.
// when the intersection of the parabolas of s1 and e lies at or left of the
// intersection of s0 and s1.  Intersections are compared as exact fractions
// (N1 / D1 <= N2 / D2 with D > 0), so no division is needed.  The evaluation
// sweeps e upwards and advances along the stack while the next site is at
// least as close.
//
// Only elements within one step of the first/last output element can matter:
// every element outside that range is a zero-distance site of this set, and
// the nearest of them dominates the rest.

__device__ __forceinline__ int site_g(int16_t v, bool target)
{
    if (!target)
        return 0;
    const int a = v < 0 ? -(int)v : (int)v;
    return a == kInf16 ? -1 : a * a;
}
__device__ __forceinline__ int site_g(int32_t v, bool target)
{
    if (!target)
        return 0;
    const int a = v < 0 ? -v : v;
    return a == kInf32 ? -1 : a;
}

template <typename TIn, bool kSdf>
__global__ void __launch_bounds__(2 * kEnvCols)
    k_envelope(const TIn *__restrict__ in, int32_t *__restrict__ out, float *__restrict__ sdf, float vox, int n,
               int nx, long long ncols, long long outer_stride, long long stride)
{
    extern __shared__ uint32_t smem[];
    constexpr int nthr = 2 * kEnvCols;
    const int tid = threadIdx.x;
    const bool setO = tid < kEnvCols;
    const long long c = (long long)blockIdx.x * kEnvCols + (tid % kEnvCols);
    if (c >= ncols)
        return;  // no block-level synchronisation below
    const long long base = (c / nx) * outer_stride + (c % nx);
    const TIn *col = in + base;
    uint32_t *stack = smem + tid;                     // entry q at stack[q * nthr]
    uint32_t *mask = smem + (size_t)n * nthr + tid;   // word w at mask[w * nthr]
    const int nw = (n + 31) >> 5;

    // 1. which elements need an output (free for O, occupied for F)
    int first = n, last = -1;
    for (int w = 0; w < nw; ++w) {
        uint32_t bits = 0;
        const int e0 = w << 5;
        const int cnt = min(32, n - e0);
#pragma unroll 8
        for (int b = 0; b < cnt; ++b) {
            const TIn v = col[(long long)(e0 + b) * stride];
            const bool target = setO ? (v > 0) : (v < 0);
            bits |= (uint32_t)target << b;
        }
        mask[w * nthr] = bits;
        if (bits) {
            if (first == n)
                first = e0 + __ffs(bits) - 1;
            last = e0 + 31 - __clz(bits);
        }
    }
    if (last < 0)
        return;

    // 2. envelope of the sites in [first-1, last+1]
    const int lo = max(first - 1, 0), hi = min(last + 1, n - 1);
    int top = -1, s0 = 0, g0 = 0, s1 = 0, g1 = 0;
    for (int e = lo; e <= hi; ++e) {
        const bool target = (mask[(e >> 5) * nthr] >> (e & 31)) & 1u;
        const int g = target ? site_g(col[(long long)e * stride], true) : 0;
        if (g < 0)
            continue;
        const int fe = e * e + g;
        while (top >= 1) {
            const int f1 = s1 * s1 + g1;
            const int N1 = fe - f1, D1 = e - s1;
            const int N2 = f1 - (s0 * s0 + g0), D2 = s1 - s0;
            if (N1 * D2 > N2 * D1)
                break;
            --top;
            s1 = s0;
            g1 = g0;
            if (top >= 1) {
                const uint32_t w = stack[(top - 1) * nthr];
                s0 = (int)(w >> 22);
                g0 = (int)(w & kG22);
            }
        }
        ++top;
        stack[top * nthr] = ((uint32_t)e << 22) | (uint32_t)g;
        s0 = s1;
        g0 = g1;
        s1 = e;
        g1 = g;
    }

    // 3. evaluate at the output elements
    int q = 0, sc = 0, gc = 0, sn = 0, gn = 0;
    if (top >= 0) {
        const uint32_t w = stack[0];
        sc = (int)(w >> 22);
        gc = (int)(w & kG22);
    }
    if (top >= 1) {
        const uint32_t w = stack[nthr];
        sn = (int)(w >> 22);
        gn = (int)(w & kG22);
    }
    for (int w = first >> 5; w <= (last >> 5); ++w) {
        uint32_t bits = mask[w * nthr];
        while (bits) {
            const int e = (w << 5) + __ffs(bits) - 1;
            bits &= bits - 1;
            int32_t val;
            if (top < 0) {
                val = kInf32;
            } else {
                int fc = (e - sc) * (e - sc) + gc;
                while (q < top) {
                    const int fn = (e - sn) * (e - sn) + gn;
                    if (fn > fc)
                        break;
                    ++q;
                    sc = sn;
                    gc = gn;
                    fc = fn;
                    if (q < top) {
                        const uint32_t x = stack[(q + 1) * nthr];
                        sn = (int)(x >> 22);
                        gn = (int)(x & kG22);
                    }
                }
                val = fc;
            }
            const long long o = base + (long long)e * stride;
            out[o] = setO ? val : -val;
            if (kSdf)
                sdf[o] = sq_to_sdf(setO ? val : -val, vox);
        }
    }
}

// ---------------------------------------------------------------------------
// fused dynamic z-pass + composite min + float epilogue
// ---------------------------------------------------------------------------
// Thread (column (x, y), time t); CTAs are ordered t-fastest so the T CTAs
// that read the same static column block run together and share it in L2.
// The dynamic field's sites lie in the slab [zlo, zlo + S): the set-O
// envelope is built from the slab only and evaluated at every z; the set-F
// envelope (distance to free voxels, needed at the few occupied slab voxels)
// spans one voxel beyond the occupied run, outside which everything is free.
__global__ void k_composite_z(const int32_t *__restrict__ static_sq, const int32_t *__restrict__ dyn_mid, int nx,
                              int ny, int nz, int zlo, int S, int T, int32_t *__restrict__ comp_sq,
                              float *__restrict__ comp_sdf, float vox)
{
    extern __shared__ uint32_t smem[];
    const int nthr = blockDim.x, tid = threadIdx.x;
    const long long V2 = (long long)nx * ny;
    const int t = blockIdx.x % T;
    const long long c = (long long)(blockIdx.x / T) * nthr + tid;
    if (c >= V2)
        return;
    uint32_t *sO = smem + tid;
    uint32_t *sF = smem + (size_t)S * nthr + tid;
    uint32_t *mk = smem + (size_t)(2 * S + 2) * nthr + tid;
    const int nw = (S + 31) >> 5;
    const int32_t *dcol = dyn_mid + (long long)t * S * V2 + c;

    // set-O envelope over the slab (occupied slab voxels are zero-distance sites)
    int topO = -1, a0 = 0, b0 = 0, a1 = 0, b1 = 0;
    int firstOcc = S, lastOcc = -1;
    for (int w = 0; w < nw; ++w) {
        uint32_t bits = 0;
        const int e0 = w << 5;
        const int cnt = min(32, S - e0);
        for (int b = 0; b < cnt; ++b) {
            const int e = e0 + b;
            const int32_t v = dcol[(long long)e * V2];
            int g;
            if (v < 0) {
                bits |= 1u << b;
                g = 0;
            } else {
                g = v == kInf32 ? -1 : v;
            }
            if (g < 0)
                continue;
            const int z = zlo + e;
            const int fz = z * z + g;
            while (topO >= 1) {
                const int f1 = a1 * a1 + b1;
                const int N1 = fz - f1, D1 = z - a1;
                const int N2 = f1 - (a0 * a0 + b0), D2 = a1 - a0;
                if (N1 * D2 > N2 * D1)
                    break;
                --topO;
                a1 = a0;
                b1 = b0;
                if (topO >= 1) {
                    const uint32_t x = sO[(topO - 1) * nthr];
                    a0 = (int)(x >> 22);
                    b0 = (int)(x & kG22);
                }
            }
            ++topO;
            sO[topO * nthr] = ((uint32_t)z << 22) | (uint32_t)g;
            a0 = a1;
            b0 = b1;
            a1 = z;
            b1 = g;
        }
        mk[w * nthr] = bits;
        if (bits) {
            if (firstOcc == S)
                firstOcc = e0 + __ffs(bits) - 1;
            lastOcc = e0 + 31 - __clz(bits);
        }
    }

    // set-F envelope around the occupied run
    int topF = -1;
    const int zo0 = zlo + firstOcc, zo1 = zlo + lastOcc;  // empty if lastOcc < 0
    if (lastOcc >= 0) {
        a0 = b0 = a1 = b1 = 0;
        const int zr0 = max(zo0 - 1, 0), zr1 = min(zo1 + 1, nz - 1);
        for (int z = zr0; z <= zr1; ++z) {
            int g = 0;
            const int e = z - zlo;
            if (e >= 0 && e < S && ((mk[(e >> 5) * nthr] >> (e & 31)) & 1u)) {
                const int32_t v = dcol[(long long)e * V2];
                g = v == -kInf32 ? -1 : -v;
            }
            if (g < 0)
                continue;
            const int fz = z * z + g;
            while (topF >= 1) {
                const int f1 = a1 * a1 + b1;
                const int N1 = fz - f1, D1 = z - a1;
                const int N2 = f1 - (a0 * a0 + b0), D2 = a1 - a0;
                if (N1 * D2 > N2 * D1)
                    break;
                --topF;
                a1 = a0;
                b1 = b0;
                if (topF >= 1) {
                    const uint32_t x = sF[(topF - 1) * nthr];
                    a0 = (int)(x >> 22);
                    b0 = (int)(x & kG22);
                }
            }
            ++topF;
            sF[topF * nthr] = ((uint32_t)z << 22) | (uint32_t)g;
            a0 = a1;
            b0 = b1;
            a1 = z;
            b1 = g;
        }
    }

    // evaluation at every z, min with the static field, epilogue
    int qO = 0, oc_s = 0, oc_g = 0, on_s = 0, on_g = 0;
    if (topO >= 0) {
        const uint32_t x = sO[0];
        oc_s = (int)(x >> 22);
        oc_g = (int)(x & kG22);
    }
    if (topO >= 1) {
        const uint32_t x = sO[nthr];
        on_s = (int)(x >> 22);
        on_g = (int)(x & kG22);
    }
    int qF = 0, fc_s = 0, fc_g = 0, fn_s = 0, fn_g = 0;
    if (topF >= 0) {
        const uint32_t x = sF[0];
        fc_s = (int)(x >> 22);
        fc_g = (int)(x & kG22);
    }
    if (topF >= 1) {
        const uint32_t x = sF[nthr];
        fn_s = (int)(x >> 22);
        fn_g = (int)(x & kG22);
    }
    const long long V = V2 * nz;
    const int32_t *scol = static_sq + c;
    int32_t *ocol = comp_sq ? comp_sq + (long long)t * V + c : nullptr;
    float *fcol = comp_sdf ? comp_sdf + (long long)t * V + c : nullptr;
#pragma unroll 4
    for (int z = 0; z < nz; ++z) {
        const int32_t sv = __ldg(scol + (long long)z * V2);
        bool occz = false;
        if (z >= zo0 && z <= zo1) {
            const int e = z - zlo;
            occz = (mk[(e >> 5) * nthr] >> (e & 31)) & 1u;
        }
        int32_t d;
        if (occz) {
            if (topF < 0) {
                d = -kInf32;
            } else {
                int fc = (z - fc_s) * (z - fc_s) + fc_g;
                while (qF < topF) {
                    const int fn = (z - fn_s) * (z - fn_s) + fn_g;
                    if (fn > fc)
                        break;
                    ++qF;
                    fc_s = fn_s;
                    fc_g = fn_g;
                    fc = fn;
                    if (qF < topF) {
                        const uint32_t x = sF[(qF + 1) * nthr];
                        fn_s = (int)(x >> 22);
                        fn_g = (int)(x & kG22);
                    }
                }
                d = -fc;
            }
        } else {
            if (topO < 0) {
                d = kInf32;
            } else {
                int fc = (z - oc_s) * (z - oc_s) + oc_g;
                while (qO < topO) {
                    const int fn = (z - on_s) * (z - on_s) + on_g;
                    if (fn > fc)
                        break;
                    ++qO;
                    oc_s = on_s;
                    oc_g = on_g;
                    fc = fn;
                    if (qO < topO) {
                        const uint32_t x = sO[(qO + 1) * nthr];
                        on_s = (int)(x >> 22);
                        on_g = (int)(x & kG22);
                    }
                }
                d = fc;
            }
        }
        const int32_t cv = min(sv, d);
        const long long o = (long long)z * V2;
        if (ocol)
            __stcs(ocol + o, cv);
        if (fcol)
            __stcs(fcol + o, sq_to_sdf(cv, vox));
    }
}

__global__ void k_broadcast_static(const int32_t *__restrict__ static_sq, long long V, int T,
                                   int32_t *__restrict__ comp_sq, float *__restrict__ comp_sdf, float vox)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
        const int32_t s = __ldg(static_sq + v);
        const float f = sq_to_sdf(s, vox);
        for (int t = 0; t < T; ++t) {
            if (comp_sq)
                __stcs(comp_sq + (long long)t * V + v, s);
            if (comp_sdf)
                __stcs(comp_sdf + (long long)t * V + v, f);
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

template <typename TIn, bool kSdf>
cudaError_t launch_envelope_t(const TIn *in, int32_t *out, float *sdf, float vox, int n, int nx, long long ncols,
                              long long outer_stride, long long stride, cudaStream_t stream)
{
    if (ncols <= 0 || n <= 0)
        return cudaSuccess;
    const size_t smem = (size_t)2 * kEnvCols * (n + (n + 31) / 32) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_envelope<TIn, kSdf>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long nblk = (ncols + kEnvCols - 1) / kEnvCols;
    k_envelope<TIn, kSdf><<<(unsigned)nblk, 2 * kEnvCols, smem, stream>>>(in, out, sdf, vox, n, nx, ncols,
                                                                           outer_stride, stride);
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

cudaError_t launch_envelope_i16(const int16_t *in, int32_t *out, int n, int nx, long long ncols,
                                long long outer_stride, long long stride, cudaStream_t stream)
{
    return launch_envelope_t<int16_t, false>(in, out, nullptr, 0.f, n, nx, ncols, outer_stride, stride, stream);
}

cudaError_t launch_envelope_i32(const int32_t *in, int32_t *out, float *sdf, float vox, int n, int nx,
                                long long ncols, long long outer_stride, long long stride, cudaStream_t stream)
{
    if (sdf)
        return launch_envelope_t<int32_t, true>(in, out, sdf, vox, n, nx, ncols, outer_stride, stride, stream);
    return launch_envelope_t<int32_t, false>(in, out, nullptr, vox, n, nx, ncols, outer_stride, stride, stream);
}

cudaError_t launch_composite_z(const int32_t *static_sq, const int32_t *dyn_mid, int nx, int ny, int nz, int zlo,
                               int S, int T, int32_t *comp_sq, float *comp_sdf, float vox, cudaStream_t stream)
{
    const long long V2 = (long long)nx * ny;
    const int words = 2 * S + 2 + (S + 31) / 32;
    int nthr = 128;
    while (nthr > 32 && (size_t)nthr * words * sizeof(uint32_t) > 200 * 1024)
        nthr >>= 1;
    const size_t smem = (size_t)nthr * words * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_composite_z, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long nblk = (V2 + nthr - 1) / nthr * T;
    k_composite_z<<<(unsigned)nblk, nthr, smem, stream>>>(static_sq, dyn_mid, nx, ny, nz, zlo, S, T, comp_sq,
                                                          comp_sdf, vox);
    return cudaGetLastError();
}

cudaError_t launch_broadcast_static(const int32_t *static_sq, long long V, int T, int32_t *comp_sq,
                                    float *comp_sdf, float vox, cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long nblk = (V + 255) / 256;
    if (nblk > (long long)sms * 8)
        nblk = (long long)sms * 8;
    k_broadcast_static<<<(unsigned)nblk, 256, 0, stream>>>(static_sq, V, T, comp_sq, comp_sdf, vox);
    return cudaGetLastError();
}

}  // namespace pcdf

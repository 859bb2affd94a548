// Exact signed EDT of a whole grid: device code shared by the stand-alone
// kernels (edt_full.cu) and the batched persistent kernel (batched.cu).
//
//   row_bits_row   one warp per row (y, z): the row's occupancy as 32-bit
//                  words (bit l of word w: voxel x = 32 w + l) and, per word,
//                  the nearest occupied and free voxel left of it and right
//                  of it.
//   edt_xy_block   a CTA of kB threads per column for slice z and the 32
//                  columns of word w: each voxel's 1-D distance along x from
//                  its word and the carries, then the y pass by the
//                  run-split banded envelope of lean.cuh; output the signed
//                  2-D partial field (int32) of the slice.
//   edt_z_block    a CTA of kB threads per column for 32 consecutive columns
//                  (x, y) of the partial field: the z pass by the same
//                  envelope, with the float field sign(S) sqrt|S| vox and,
//                  optionally, each column's largest value.
// The 1-D row distances never reach memory, so the grid is read once as
// bytes and the 2-D partial field is written and read once.  kCoherent: the
// inputs were written earlier in the same launch (L2-coherent loads).
#pragma once

#include "lean.cuh"

namespace pcdf {
namespace full {

using lean::kCols;

constexpr int kLoNone = -16384;  // "no voxel on the left" (beyond any row)
constexpr int kHiNone = 16384;   // "no voxel on the right"

template <bool kCoherent, class T>
__device__ __forceinline__ T ld(const T *p)
{
    if (kCoherent)
        return __ldcg(p);
    return __ldg(p);
}

__device__ __forceinline__ uint32_t pack16(int lo, int hi)
{
    return (uint32_t)(uint16_t)(int16_t)lo | ((uint32_t)(uint16_t)(int16_t)hi << 16);
}

// 0x01 in every byte of w that is non-zero, 0x00 elsewhere
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t w)
{
    uint32_t t = w | (w >> 4);
    t |= t >> 2;
    t |= t >> 1;
    return t & 0x01010101u;
}

// One warp: row `row` = z * ny + y.  kMode 0: occupancy, 1: occupancy OR the
// capsules caps[0 .. H), 2: the capsules alone.  W = ceil(nx / 32) <= 16.
// nrows: the grid's rows (for the bounds checks).  vec4 (mode 0 only; needs
// nx % 4 == 0 and a 4-byte aligned occ): the occupancy is read four bytes per
// lane, and the eight lanes of a row word assemble its bits by shuffles.
template <int kMode>
__device__ __forceinline__ void row_bits_row(const uint8_t *__restrict__ occ, const CapInfo *caps, int H, int nx,
                                             int ny, long long row, long long nrows, int W,
                                             uint32_t *__restrict__ bits, uint2 *__restrict__ carry, int lane,
                                             bool vec4 = false)
{
    const int y = (int)(row % ny), z = (int)(row / ny);
    unsigned long long active = 0;  // capsules whose box crosses this row (H <= 64)
    if (kMode != 0) {
        for (int h = 0; h < H; ++h) {
            const CapInfo &ci = caps[h];
            if (ci.lo[0] <= ci.hi[0] && y >= ci.lo[1] && y <= ci.hi[1] && z >= ci.lo[2] && z <= ci.hi[2])
                active |= 1ull << h;
        }
    }
    const uint8_t *src = occ + row * nx;
    uint32_t mine = 0;  // word `lane` of the row
    if (kMode == 0 && vec4) {
        // pass p: lane l reads voxels 128 p + 4 l .. + 3; lanes 8 g .. 8 g + 7
        // hold word 4 p + g, four bits each
        const uint32_t *src4 = reinterpret_cast<const uint32_t *>(src);
        for (int p = 0; 4 * p < W; ++p) {
            const int x = 128 * p + 4 * lane;
            uint32_t v = 0;
            if (x < nx && PCDF_IN(row * nx + x + 3, nrows * nx))
                v = __ldg(src4 + (x >> 2));
            uint32_t m = ((nonzero_bytes(v) * 0x01020408u) >> 24) << (4 * (lane & 7));
            m |= __shfl_xor_sync(0xffffffffu, m, 1);
            m |= __shfl_xor_sync(0xffffffffu, m, 2);
            m |= __shfl_xor_sync(0xffffffffu, m, 4);
            const uint32_t word = __shfl_sync(0xffffffffu, m, 8 * ((lane - 4 * p) & 3));
            if (lane >= 4 * p && lane < 4 * p + 4)
                mine = word;
        }
    }
    for (int w = 0; w < W && !(kMode == 0 && vec4); ++w) {
        const int x = 32 * w + lane;
        bool o = false;
        if (x < nx) {
            if (kMode != 2 && PCDF_IN(row * nx + x, nrows * nx))
                o = __ldg(src + x) != 0;
            if (kMode != 0 && !o) {
                for (unsigned long long m = active; m; m &= m - 1) {
                    const CapInfo &ci = caps[__ffsll((long long)m) - 1];
                    if (x >= ci.lo[0] && x <= ci.hi[0] && capsule_contains(ci, x, y, z)) {
                        o = true;
                        break;
                    }
                }
            }
        }
        const uint32_t b = __ballot_sync(0xffffffffu, o);
        if (lane == w)
            mine = b;
    }
    const int xb = 32 * lane;
    const uint32_t vm = lane >= W ? 0u : (nx - xb >= 32 ? 0xffffffffu : (1u << (nx - xb)) - 1u);
    const uint32_t mo = mine, mf = ~mine & vm;
    int lO = mo ? xb + 31 - __clz(mo) : kLoNone, lF = mf ? xb + 31 - __clz(mf) : kLoNone;
    int fO = mo ? xb + __ffs(mo) - 1 : kHiNone, fF = mf ? xb + __ffs(mf) - 1 : kHiNone;
    // inclusive prefix maxima and suffix minima over the row's words (W <= 16 lanes)
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, lO, d), b = __shfl_up_sync(0xffffffffu, lF, d);
        const int p = __shfl_down_sync(0xffffffffu, fO, d), q = __shfl_down_sync(0xffffffffu, fF, d);
        if (lane >= d) {
            lO = max(lO, a);
            lF = max(lF, b);
        }
        if (lane + d < 32) {
            fO = min(fO, p);
            fF = min(fF, q);
        }
    }
    int LO = __shfl_up_sync(0xffffffffu, lO, 1), LF = __shfl_up_sync(0xffffffffu, lF, 1);
    int RO = __shfl_down_sync(0xffffffffu, fO, 1), RF = __shfl_down_sync(0xffffffffu, fF, 1);
    if (lane == 0)
        LO = LF = kLoNone;
    if (lane == 31)
        RO = RF = kHiNone;
    if (lane < W && PCDF_IN(row * W + lane, nrows * W)) {
        bits[row * W + lane] = mine;
        carry[row * W + lane] = make_uint2(pack16(LO, RO), pack16(LF, RF));
    }
}

// Signed 1-D squared distance along x of voxel x = 32 w + c of a row: the
// nearest voxel of the other state in the word m, else the carried one.
// vm: the word's in-grid bits.
__device__ __forceinline__ int32_t row_value(uint32_t m, uint2 cr, int c, int x, int nx, uint32_t vm)
{
    const bool o = (m >> c) & 1u;
    const uint32_t s = o ? (~m & vm) : m;
    const uint32_t cw = o ? cr.y : cr.x;
    const int lo = (int16_t)(cw & 0xffffu), hi = (int16_t)(cw >> 16);
    const uint32_t below = s & ((1u << c) - 1u), above = s & (0xfffffffeu << c);
    const int base = x - c;
    const int xl = below ? base + 31 - __clz(below) : lo;
    const int xr = above ? base + __ffs(above) - 1 : hi;
    const int d = min(x - xl, xr - x);
    if (d >= nx)
        return o ? -kInf32 : kInf32;
    return o ? -(d * d) : d * d;
}

// Seam merges of the CTA's columns, as a tree (thread of column c, band b);
// ends with a barrier.
template <int kB>
__device__ __forceinline__ void merge_tree(uint32_t *tile, lean::Seg<kB> &seg, int n, int c, int b)
{
#pragma unroll
    for (int r = 0; (1 << r) < kB; ++r) {
        const int sb = lean::tree_seam(kB, r, b);
        if (sb)
            lean::merge_seam<kB>(tile, seg, n, c, sb, sb - (1 << r), min(sb + (1 << r), kB));
        __syncthreads();
    }
}

// The CTA (kCols * kB threads) computes slice z, columns 32 w .. 32 w + 31;
// smem holds kCols * (ny + ceil(ny / 32)) words.
template <int kB, bool kCoherent>
__device__ __forceinline__ void edt_xy_block(const uint32_t *__restrict__ bits, const uint2 *__restrict__ carry,
                                             int nx, int ny, int nz, int W, int w, int z, int32_t *__restrict__ mid,
                                             uint32_t *smem)
{
    __shared__ lean::Seg<kB> seg;
    const int c = threadIdx.x % kCols, b = threadIdx.x / kCols;
    const int x = 32 * w + c;
    const bool live = x < nx;
    const int n = ny, L = lean::band_len(n, kB);
    uint32_t *tile = smem, *mk = smem + n * kCols;
    const int e0 = b * L, e1 = min(e0 + L, n);
    const uint32_t vm = nx - 32 * w >= 32 ? 0xffffffffu : (1u << (nx - 32 * w)) - 1u;
    const long long rbase = (long long)z * ny * W + w;  // word of row y: rbase + y * W
    // warp b is band b and its lanes are the 32 columns, which share each
    // row's word and carries: lane i loads those of row y0 + i (all loads in
    // flight at once) and the warp reads them by shuffles
    for (int y0 = e0; y0 < e1; y0 += 32) {
        const int cnt = min(32, e1 - y0);  // warp-uniform
        uint32_t ob = 0;
        uint32_t mi = 0;
        uint2 ci = make_uint2(0, 0);
        const long long wi = rbase + (long long)(y0 + c) * W;
        if (c < cnt && PCDF_IN(wi, (long long)nz * ny * W)) {
            mi = ld<kCoherent>(bits + wi);
            ci = ld<kCoherent>(carry + wi);
        }
#pragma unroll 8
        for (int i = 0; i < cnt; ++i) {
            const uint32_t m = __shfl_sync(0xffffffffu, mi, i);
            const uint2 cr = make_uint2(__shfl_sync(0xffffffffu, ci.x, i), __shfl_sync(0xffffffffu, ci.y, i));
            const int32_t v = live ? row_value(m, cr, c, x, nx, vm) : kInf32;
            if (PCDF_IN(y0 + i, n))
                tile[(y0 + i) * kCols + c] = (uint32_t)v;
            ob |= (uint32_t)(v < 0) << i;
        }
        if (PCDF_IN(y0 >> 5, (n + 31) >> 5))
            mk[(y0 >> 5) * kCols + c] = ob;
    }
    __syncthreads();
    lean::build_band<kB>(tile, seg, n, L, c, b);
    __syncthreads();
    merge_tree<kB>(tile, seg, n, c, b);
    if (live) {
        // elements are emitted in order e0, e0 + 1, ...: running output pointer
        int32_t *dst = mid + ((long long)z * ny + e0) * nx + x;
        const long long V = (long long)nz * ny * nx, o0 = (long long)z * ny * nx + x;
        auto out = [=](int e, int v) mutable {
            if (PCDF_IN(o0 + (long long)e * nx, V))
                *dst = v;
            dst += nx;
        };
        lean::eval_band<kB>(tile, mk, seg, n, L, c, b, out);
    }
}

// Output of the z pass: elements come in order e0, e0 + 1, ... (running
// pointers); the largest value is kept for the column maximum.
template <bool kSdf>
struct ZOut {
    int32_t *dq;
    float *df;
    long long ncols;
    float vox;
    int32_t mx;
    long long cl, V;  // the column and the field's size (bounds checks)
    __device__ __forceinline__ void operator()(int e, int v)
    {
        const bool ok = PCDF_IN(cl + (long long)e * ncols, V);
        if (ok)
            __stcs(dq, v);
        dq += ncols;
        mx = max(mx, v);
        if (kSdf) {
            if (ok)
                __stcs(df, sq_to_sdf_fast(v, vox));
            df += ncols;
        }
    }
};

// The CTA (kCols * kB threads) computes columns col0 .. col0 + 31 of the
// partial field [n][ncols]; smem holds kCols * (n + ceil(n / 32)) words.
// colmax (non-NULL): each column's largest output value, indexed by column;
// then every thread of the CTA must call (one more barrier).
template <int kB, bool kSdf, bool kCoherent>
__device__ __forceinline__ void edt_z_block(const int32_t *__restrict__ mid, int32_t *__restrict__ sq,
                                            float *__restrict__ sdf, float vox, int n, long long ncols,
                                            long long col0, uint32_t *smem, int32_t *__restrict__ colmax)
{
    __shared__ lean::Seg<kB> seg;
    const int c = threadIdx.x % kCols, b = threadIdx.x / kCols;
    const long long cl = col0 + c;
    const bool live = cl < ncols;
    const int L = lean::band_len(n, kB);
    uint32_t *tile = smem, *mk = smem + n * kCols;
    const int e0 = b * L, e1 = min(e0 + L, n);
    const int32_t *src = mid + (live ? cl : 0);
    for (int z0 = e0; z0 < e1; z0 += 32) {
        const int cnt = min(32, e1 - z0);
        uint32_t ob = 0;
        if (cnt == 32) {
            int32_t v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i)
                v[i] = live && PCDF_IN(cl + (long long)(z0 + i) * ncols, (long long)n * ncols)
                           ? ld<kCoherent>(src + (long long)(z0 + i) * ncols)
                           : kInf32;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (PCDF_IN(z0 + i, n))
                    tile[(z0 + i) * kCols + c] = (uint32_t)v[i];
                ob |= (uint32_t)(v[i] < 0) << i;
            }
        } else {
            for (int i = 0; i < cnt; ++i) {
                const int32_t v = live && PCDF_IN(cl + (long long)(z0 + i) * ncols, (long long)n * ncols)
                                      ? ld<kCoherent>(src + (long long)(z0 + i) * ncols)
                                      : kInf32;
                if (PCDF_IN(z0 + i, n))
                    tile[(z0 + i) * kCols + c] = (uint32_t)v;
                ob |= (uint32_t)(v < 0) << i;
            }
        }
        if (PCDF_IN(z0 >> 5, (n + 31) >> 5))
            mk[(z0 >> 5) * kCols + c] = ob;
    }
    __syncthreads();
    lean::build_band<kB>(tile, seg, n, L, c, b);
    __syncthreads();
    merge_tree<kB>(tile, seg, n, c, b);
    int32_t mx = INT32_MIN;
    if (live) {
        ZOut<kSdf> out{sq + cl + (long long)e0 * ncols, kSdf ? sdf + cl + (long long)e0 * ncols : nullptr, ncols,
                       vox, INT32_MIN, cl, (long long)n * ncols};
        mx = lean::eval_band<kB>(tile, mk, seg, n, L, c, b, out).mx;
    }
    if (colmax) {  // uniform over the CTA
        // the band table is done with once every band has been evaluated:
        // its storage holds the bands' maxima
        static_assert(sizeof(lean::Seg<kB>) >= sizeof(int32_t) * kB * kCols, "band table too small");
        __syncthreads();
        int32_t(*s_max)[kCols] = reinterpret_cast<int32_t(*)[kCols]>(&seg);
        s_max[b][c] = mx;
        __syncthreads();
        if (b == 0 && live && PCDF_IN(cl, ncols)) {
            int32_t m = s_max[0][c];
#pragma unroll
            for (int k = 1; k < kB; ++k)
                m = max(m, s_max[k][c]);
            colmax[cl] = m;
        }
    }
}

}  // namespace full
}  // namespace pcdf

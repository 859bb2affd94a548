// Exact signed EDT of a whole grid (sm_103a): the static map (Sec. 6: the
// environment's exact distance field), the union of the map and the humans'
// primitives at one t (the full per-field recompute that the composite is
// compared against), and a primitive alone on its box (the template of the
// translated primitive field).
//
// Three launches:
//   k_row_bits  one warp per row (y, z): the row's occupancy as 32-bit words
//               (bit l of word w: voxel x = 32 w + l) and, per word, the
//               nearest occupied and free voxel left of it and right of it.
//   k_edt_xy    one CTA per (slice z, 32-column word w), kB threads per
//               column: the 1-D distance along x of every voxel of its 32
//               columns from the word and its carries, then the y pass by
//               the run-split banded envelope of lean.cuh.  Output: the
//               signed 2-D partial field (int32) of the slice.
//   k_edt_z     one CTA per 32 consecutive columns (x, y) of the partial
//               field, kB threads per column: the z pass by the same
//               envelope, with the float field sign(S) sqrt|S| vox.
// The 1-D row distances never reach memory, so the grid is read once as
// bytes and the 2-D partial field is written and read once.
#include <cuda_runtime.h>

#include "lean.cuh"

namespace pcdf {
namespace {

using lean::kCols;

constexpr int kRowsPerCta = 8;          // k_row_bits: rows (warps) per CTA
constexpr int kLoNone = -16384;         // "no voxel on the left" (beyond any row)
constexpr int kHiNone = 16384;          // "no voxel on the right"
#ifndef PCDF_XY_BANDS
#define PCDF_XY_BANDS 8
#endif
#ifndef PCDF_Z_BANDS
#define PCDF_Z_BANDS 8
#endif
constexpr int kXyBands = PCDF_XY_BANDS;  // envelope threads per column, y pass
constexpr int kZBands = PCDF_Z_BANDS;    // envelope threads per column, z pass

__device__ __forceinline__ uint32_t pack16(int lo, int hi)
{
    return (uint32_t)(uint16_t)(int16_t)lo | ((uint32_t)(uint16_t)(int16_t)hi << 16);
}

// kMode 0: occupancy, 1: occupancy OR the capsules of this launch, 2: the
// capsules alone.  W = ceil(nx / 32) <= 16.
template <int kMode>
__global__ void __launch_bounds__(32 * kRowsPerCta)
    k_row_bits(const uint8_t *__restrict__ occ, const __grid_constant__ CapBatch caps, int H, int nx, int ny,
               long long nrows, int W, uint32_t *__restrict__ bits, uint2 *__restrict__ carry)
{
    const int lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * kRowsPerCta + (threadIdx.x >> 5);
    if (row >= nrows)
        return;  // warp-uniform
    const int y = (int)(row % ny), z = (int)(row / ny);

    unsigned long long active = 0;  // capsules whose box crosses this row (H <= 64)
    if (kMode != 0) {
        for (int h = 0; h < H; ++h) {
            const CapInfo &ci = caps.caps[h];
            if (ci.lo[0] <= ci.hi[0] && y >= ci.lo[1] && y <= ci.hi[1] && z >= ci.lo[2] && z <= ci.hi[2])
                active |= 1ull << h;
        }
    }
    const uint8_t *src = occ + row * nx;
    uint32_t mine = 0;  // word `lane` of the row
    for (int w = 0; w < W; ++w) {
        const int x = 32 * w + lane;
        bool o = false;
        if (x < nx) {
            if (kMode != 2)
                o = __ldg(src + x) != 0;
            if (kMode != 0 && !o) {
                for (unsigned long long m = active; m; m &= m - 1) {
                    const CapInfo &ci = caps.caps[__ffsll((long long)m) - 1];
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
    if (lane < W) {
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
__device__ __forceinline__ void merge_tree(uint32_t *tile, lean::Seg<kB> &seg, int c, int b)
{
#pragma unroll
    for (int r = 0; (1 << r) < kB; ++r) {
        const int sb = lean::tree_seam(kB, r, b);
        if (sb)
            lean::merge_seam<kB>(tile, seg, c, sb, sb - (1 << r), min(sb + (1 << r), kB));
        __syncthreads();
    }
}

template <int kB>
__global__ void __launch_bounds__(kCols * kB)
    k_edt_xy(const uint32_t *__restrict__ bits, const uint2 *__restrict__ carry, int nx, int ny, int W,
             int32_t *__restrict__ mid)
{
    extern __shared__ uint32_t smem[];
    __shared__ lean::Seg<kB> seg;
    const int c = threadIdx.x % kCols, b = threadIdx.x / kCols;
    const int w = blockIdx.x, z = blockIdx.y;
    const int x = 32 * w + c;
    const bool live = x < nx;
    const int n = ny, L = lean::band_len(n, kB);
    uint32_t *tile = smem, *mk = smem + n * kCols;
    const int e0 = b * L, e1 = min(e0 + L, n);
    const uint32_t vm = nx - 32 * w >= 32 ? 0xffffffffu : (1u << (nx - 32 * w)) - 1u;
    const long long rbase = (long long)z * ny * W + w;  // word of row y: rbase + y * W
    for (int y0 = e0; y0 < e1; y0 += 32) {
        const int cnt = min(32, e1 - y0);
        uint32_t ob = 0;
        const uint32_t *pb = bits + rbase + (long long)y0 * W;
        const uint2 *pc = carry + rbase + (long long)y0 * W;
#pragma unroll 8
        for (int i = 0; i < cnt; ++i) {
            const uint32_t m = __ldg(pb);
            const uint2 cr = __ldg(pc);
            pb += W;
            pc += W;
            const int32_t v = live ? row_value(m, cr, c, x, nx, vm) : kInf32;
            tile[(y0 + i) * kCols + c] = (uint32_t)v;
            ob |= (uint32_t)(v < 0) << i;
        }
        mk[(y0 >> 5) * kCols + c] = ob;
    }
    __syncthreads();
    lean::build_band<kB>(tile, seg, n, L, c, b);
    __syncthreads();
    merge_tree<kB>(tile, seg, c, b);
    if (!live)
        return;
    // elements are emitted in order e0, e0 + 1, ...: running output pointer
    int32_t *dst = mid + ((long long)z * ny + e0) * nx + x;
    auto out = [=](int, int v) mutable {
        *dst = v;
        dst += nx;
    };
    lean::eval_band<kB>(tile, mk, seg, n, L, c, b, out);
}

template <int kB, bool kSdf>
__global__ void __launch_bounds__(kCols * kB)
    k_edt_z(const int32_t *__restrict__ mid, int32_t *__restrict__ sq, float *__restrict__ sdf, float vox, int n,
            long long ncols)
{
    extern __shared__ uint32_t smem[];
    __shared__ lean::Seg<kB> seg;
    const int c = threadIdx.x % kCols, b = threadIdx.x / kCols;
    const long long cl = (long long)blockIdx.x * kCols + c;
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
                v[i] = live ? __ldg(src + (long long)(z0 + i) * ncols) : kInf32;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                tile[(z0 + i) * kCols + c] = (uint32_t)v[i];
                ob |= (uint32_t)(v[i] < 0) << i;
            }
        } else {
            for (int i = 0; i < cnt; ++i) {
                const int32_t v = live ? __ldg(src + (long long)(z0 + i) * ncols) : kInf32;
                tile[(z0 + i) * kCols + c] = (uint32_t)v;
                ob |= (uint32_t)(v < 0) << i;
            }
        }
        mk[(z0 >> 5) * kCols + c] = ob;
    }
    __syncthreads();
    lean::build_band<kB>(tile, seg, n, L, c, b);
    __syncthreads();
    merge_tree<kB>(tile, seg, c, b);
    if (!live)
        return;
    // elements are emitted in order e0, e0 + 1, ...: running output pointers
    int32_t *dq = sq + cl + (long long)e0 * ncols;
    float *df = kSdf ? sdf + cl + (long long)e0 * ncols : nullptr;
    auto out = [=](int, int v) mutable {
        __stcs(dq, v);
        dq += ncols;
        if (kSdf) {
            __stcs(df, sq_to_sdf_fast(v, vox));
            df += ncols;
        }
    };
    lean::eval_band<kB>(tile, mk, seg, n, L, c, b, out);
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

size_t tile_bytes(int n) { return (size_t)kCols * (n + (n + 31) / 32) * sizeof(uint32_t); }

}  // namespace

size_t full_edt_scratch(int nx, int ny, int nz, size_t *bits_off, size_t *carry_off, size_t *mid_off)
{
    const auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t nw = (size_t)nz * ny * ((nx + 31) / 32);
    *bits_off = 0;
    *carry_off = al(nw * sizeof(uint32_t));
    *mid_off = *carry_off + al(nw * sizeof(uint2));
    return *mid_off + al((size_t)nx * ny * nz * sizeof(int32_t));
}

cudaError_t launch_full_edt(int mode, const uint8_t *occ, const CapBatch *caps, int H, int nx, int ny, int nz,
                            int32_t *sq, float *sdf, float vox, void *ws, cudaStream_t st)
{
    size_t bo, co, mo;
    full_edt_scratch(nx, ny, nz, &bo, &co, &mo);
    uint32_t *bits = (uint32_t *)((char *)ws + bo);
    uint2 *carry = (uint2 *)((char *)ws + co);
    int32_t *mid = (int32_t *)((char *)ws + mo);
    const int W = (nx + 31) / 32;
    const long long nrows = (long long)ny * nz;
    const unsigned nb = (unsigned)((nrows + kRowsPerCta - 1) / kRowsPerCta);
    switch (mode) {
    case 0: k_row_bits<0><<<nb, 32 * kRowsPerCta, 0, st>>>(occ, *caps, H, nx, ny, nrows, W, bits, carry); break;
    case 1: k_row_bits<1><<<nb, 32 * kRowsPerCta, 0, st>>>(occ, *caps, H, nx, ny, nrows, W, bits, carry); break;
    default: k_row_bits<2><<<nb, 32 * kRowsPerCta, 0, st>>>(occ, *caps, H, nx, ny, nrows, W, bits, carry); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;

    const size_t sxy = tile_bytes(ny);
    if ((e = set_smem(k_edt_xy<kXyBands>, sxy)) != cudaSuccess)
        return e;
    k_edt_xy<kXyBands><<<dim3((unsigned)W, (unsigned)nz), kCols * kXyBands, sxy, st>>>(bits, carry, nx, ny, W, mid);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;

    const long long ncols = (long long)nx * ny;
    const unsigned nbz = (unsigned)((ncols + kCols - 1) / kCols);
    const size_t sz = tile_bytes(nz);
    if (sdf) {
        if ((e = set_smem(k_edt_z<kZBands, true>, sz)) != cudaSuccess)
            return e;
        k_edt_z<kZBands, true><<<nbz, kCols * kZBands, sz, st>>>(mid, sq, sdf, vox, nz, ncols);
    } else {
        if ((e = set_smem(k_edt_z<kZBands, false>, sz)) != cudaSuccess)
            return e;
        k_edt_z<kZBands, false><<<nbz, kCols * kZBands, sz, st>>>(mid, sq, nullptr, vox, nz, ncols);
    }
    return cudaGetLastError();
}

}  // namespace pcdf

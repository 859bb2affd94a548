// Lower-envelope pass of the exact EDT along y or z (sm_103a).
//
// A CTA owns 32 neighbouring columns (consecutive x: every global access of
// the CTA is one contiguous 128-byte row) and four threads per column, one per
// quarter ("band") of the column.  The column block is staged in shared
// memory; then, for each site set
//   set O (sites: occupied voxels; output at free voxels) and
//   set F (sites: free voxels; output at occupied voxels),
//   1. every band builds the lower envelope of the parabolas (x - i)^2 + g(i)
//      of its own sites in place over its staged slots (the entry pushed while
//      reading element e lands in a slot at or before e, already read);
//   2. the first thread of the column merges the four envelopes left to
//      right: two envelopes over disjoint, ordered site ranges merge into a
//      prefix of the left one and a suffix of the right one, found by popping
//      at the seam until both seam triples are convex (the bridge of two
//      x-separated lower hulls of the dual points (i, i^2 + g(i)));
//   3. every band binary-searches the merged envelope for the site nearest to
//      its first element and walks forward over its outputs.
// Elements of the other state are zero-distance sites; inside a run of them
// only the two run ends can be nearest to anything outside the run, so only
// run ends are pushed.  Each voxel's signed value carries both sets (sign =
// its own state, magnitude = partial distance to the other state), so one pass
// produces the signed result.
#include <cuda_runtime.h>

#include "edt_common.cuh"

namespace pcdf {
namespace {

constexpr int kCols = 32;   // columns per CTA
constexpr int kBands = 4;   // threads per column

__device__ __forceinline__ int32_t widen(int16_t v)
{
    const int a = v < 0 ? -(int)v : (int)v;
    if (a == kInf16)
        return v < 0 ? -kInf32 : kInf32;
    return v < 0 ? -(a * a) : a * a;
}
__device__ __forceinline__ int32_t widen(int32_t v) { return v; }

// The merged envelope of a column: band k contributes entries
// slots [lo_k + st_k, lo_k + st_k + len_k) of the column's tile.
struct Merged {
    int lo[kBands], st[kBands], len[kBands];
    int K;  // total entries
    // slot of global entry q (0 <= q < K)
    __device__ __forceinline__ int slot(int q) const
    {
#pragma unroll
        for (int k = 0; k < kBands - 1; ++k) {
            if (q < len[k])
                return lo[k] + st[k] + q;
            q -= len[k];
        }
        return lo[kBands - 1] + st[kBands - 1] + q;
    }
};

template <typename TIn>
__device__ __forceinline__ void stage(uint32_t *tile, const TIn *col, long long stride, int a, int b)
{
#pragma unroll 8
    for (int e = a; e < b; ++e)
        tile[e * kCols] = (uint32_t)widen(col[(long long)e * stride]);
}

template <typename TIn, bool kSdf>
__global__ void __launch_bounds__(kCols * kBands)
    k_envelope_banded(const TIn *__restrict__ in, int32_t *__restrict__ out, float *__restrict__ sdf, float vox,
                      int n, int nx, long long ncols, long long outer_stride, long long stride)
{
    extern __shared__ uint32_t smem[];
    __shared__ int seg[3][kBands][kCols];  // per column: band start-in-band, length; then any-target flag
    const int c = threadIdx.x % kCols, band = threadIdx.x / kCols;
    const long long cl = (long long)blockIdx.x * kCols + c;
    const bool live = cl < ncols;
    const long long base = live ? (cl / nx) * outer_stride + (cl % nx) : 0;
    const TIn *col = in + base;
    uint32_t *tile = smem + c;                                  // element e at tile[e * kCols]
    uint32_t *mk = smem + (size_t)n * kCols + c;                // occupied bits, word w at mk[w * kCols]
    const int bw = (n + kBands - 1) / kBands;                   // band width
    const int e0 = min(band * bw, n), e1 = min(e0 + bw, n);

    // stage this band's slots and the occupancy bits of its words
    if (live)
        stage(tile, col, stride, e0, e1);
    __syncthreads();
    const int nw = (n + 31) >> 5;
    if (live)
        for (int w = band; w < nw; w += kBands) {
            const int w0 = w << 5, cnt = min(32, n - w0);
            uint32_t occ = 0;
            for (int i = 0; i < cnt; ++i)
                occ |= (uint32_t)((int32_t)tile[(w0 + i) * kCols] < 0) << i;
            mk[w * kCols] = occ;
        }
    __syncthreads();
    auto occupied = [&](int e) { return (mk[(e >> 5) * kCols] >> (e & 31)) & 1u; };

    for (int set = 0; set < 2; ++set) {
        // 0. does this band hold outputs of this set?  (re-stage for set F)
        bool mine = false;
        if (live)
            for (int e = e0; e < e1; ++e)
                mine |= set == 0 ? !occupied(e) : occupied(e);
        if (!__syncthreads_or(mine))
            continue;
        if (set == 1 && live)
            stage(tile, col, stride, e0, e1);  // set O may have overwritten the slots
        __syncthreads();

        // 1. band envelope, in place over slots [e0, e1)
        EnvBuilder B(tile + e0 * kCols, kCols);
        if (live)
            for (int e = e0; e < e1; ++e) {
                int g;
                const bool oc = occupied(e);
                if (set == 0 ? !oc : oc) {
                    const int32_t v = (int32_t)tile[e * kCols];
                    if (v == kInf32 || v == -kInf32)
                        continue;
                    g = v < 0 ? -v : v;
                } else {
                    const bool l = e > 0 && (set == 0 ? !occupied(e - 1) : occupied(e - 1));
                    const bool r = e + 1 < n && (set == 0 ? !occupied(e + 1) : occupied(e + 1));
                    if (!l && !r)
                        continue;
                    g = 0;
                }
                B.push(e, g);
            }
        seg[0][band][c] = 0;
        seg[1][band][c] = B.top + 1;
        __syncthreads();

        // 2. merge the bands of the column (first thread of the column); the
        //    segment table lives in shared memory (indexed by band)
        if (band == 0 && live) {
            int *st = &seg[0][0][c], *len = &seg[1][0][c];  // band k at [k * kCols]
            auto ent = [&](int k, int i) { return tile[(min(k * bw, n) + st[k * kCols] + i) * kCols]; };
            for (int k = 1; k < kBands; ++k) {
                for (;;) {
                    const int lk = len[k * kCols];
                    if (lk == 0)
                        break;
                    int j = k - 1;
                    while (j >= 0 && len[j * kCols] == 0)
                        --j;
                    if (j < 0)
                        break;
                    const int lj = len[j * kCols];
                    const uint32_t wl = ent(j, lj - 1), wr = ent(k, 0);
                    uint32_t wp = 0;
                    bool has_prev = lj >= 2;
                    if (has_prev) {
                        wp = ent(j, lj - 2);
                    } else {
                        int i = j - 1;
                        while (i >= 0 && len[i * kCols] == 0)
                            --i;
                        if (i >= 0) {
                            has_prev = true;
                            wp = ent(i, len[i * kCols] - 1);
                        }
                    }
                    if (has_prev &&
                        dominated(site_of(wp), gval_of(wp), site_of(wl), gval_of(wl), site_of(wr), gval_of(wr))) {
                        len[j * kCols] = lj - 1;
                        continue;
                    }
                    if (lk >= 2) {
                        const uint32_t w2 = ent(k, 1);
                        if (dominated(site_of(wl), gval_of(wl), site_of(wr), gval_of(wr), site_of(w2), gval_of(w2))) {
                            st[k * kCols] += 1;
                            len[k * kCols] = lk - 1;
                            continue;
                        }
                    }
                    break;
                }
            }
        }
        __syncthreads();

        // 3. outputs of this band
        if (live && mine) {
            Merged M;
            M.K = 0;
#pragma unroll
            for (int k = 0; k < kBands; ++k) {
                M.lo[k] = min(k * bw, n);
                M.st[k] = seg[0][k][c];
                M.len[k] = seg[1][k][c];
                M.K += M.len[k];
            }
            int32_t *o = out + base;
            float *f = kSdf ? sdf + base : nullptr;
            if (M.K == 0) {
                for (int e = e0; e < e1; ++e)
                    if (set == 0 ? !occupied(e) : occupied(e)) {
                        const int32_t r = set == 0 ? kInf32 : -kInf32;
                        o[(long long)e * stride] = r;
                        if (kSdf)
                            f[(long long)e * stride] = sq_to_sdf(r, vox);
                    }
            } else {
                // first entry whose successor is not closer at e0
                int lq = 0, hq = M.K - 1;
                while (lq < hq) {
                    const int mid = (lq + hq) >> 1;
                    const uint32_t a = tile[M.slot(mid) * kCols], b = tile[M.slot(mid + 1) * kCols];
                    if (parab(e0, site_of(b), gval_of(b)) <= parab(e0, site_of(a), gval_of(a)))
                        lq = mid + 1;
                    else
                        hq = mid;
                }
                int q = lq;
                uint32_t w = tile[M.slot(q) * kCols];
                int sc = site_of(w), gc = gval_of(w);
                int sn = 0, gn = 0;
                if (q + 1 < M.K) {
                    w = tile[M.slot(q + 1) * kCols];
                    sn = site_of(w);
                    gn = gval_of(w);
                }
                for (int e = e0; e < e1; ++e) {
                    if (!(set == 0 ? !occupied(e) : occupied(e)))
                        continue;
                    int fc = parab(e, sc, gc);
                    while (q + 1 < M.K) {
                        const int fn = parab(e, sn, gn);
                        if (fn > fc)
                            break;
                        ++q;
                        sc = sn;
                        gc = gn;
                        fc = fn;
                        if (q + 1 < M.K) {
                            w = tile[M.slot(q + 1) * kCols];
                            sn = site_of(w);
                            gn = gval_of(w);
                        }
                    }
                    const int32_t r = set == 0 ? fc : -fc;
                    o[(long long)e * stride] = r;
                    if (kSdf)
                        f[(long long)e * stride] = sq_to_sdf(r, vox);
                }
            }
        }
        __syncthreads();
    }
}

template <typename TIn, bool kSdf>
cudaError_t launch_banded(const TIn *in, int32_t *out, float *sdf, float vox, int n, int nx, long long ncols,
                          long long outer_stride, long long stride, cudaStream_t stream)
{
    if (ncols <= 0 || n <= 0)
        return cudaSuccess;
    const size_t smem = (size_t)kCols * (n + (n + 31) / 32) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_envelope_banded<TIn, kSdf>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long nblk = (ncols + kCols - 1) / kCols;
    k_envelope_banded<TIn, kSdf><<<(unsigned)nblk, kCols * kBands, smem, stream>>>(in, out, sdf, vox, n, nx, ncols,
                                                                                    outer_stride, stride);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_envelope_i16(const int16_t *in, int32_t *out, int n, int nx, long long ncols,
                                long long outer_stride, long long stride, cudaStream_t stream)
{
    return launch_banded<int16_t, false>(in, out, nullptr, 0.f, n, nx, ncols, outer_stride, stride, stream);
}

cudaError_t launch_envelope_i32(const int32_t *in, int32_t *out, float *sdf, float vox, int n, int nx,
                                long long ncols, long long outer_stride, long long stride, cudaStream_t stream)
{
    if (sdf)
        return launch_banded<int32_t, true>(in, out, sdf, vox, n, nx, ncols, outer_stride, stride, stream);
    return launch_banded<int32_t, false>(in, out, nullptr, vox, n, nx, ncols, outer_stride, stride, stream);
}

}  // namespace pcdf

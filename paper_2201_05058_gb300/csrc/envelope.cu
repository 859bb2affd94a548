// Banded lower-envelope pass of the exact EDT along y or z (sm_103a).
//
// A CTA owns 32 neighbouring columns (consecutive x, so every global access is
// a coalesced 128-byte row) and splits each column into bands of 32 elements,
// one thread per (column, band).  The column block is staged in shared memory
// once; then, for each of the two site sets (sites = occupied voxels, output
// at free voxels; and the reverse), the CTA
//   1. builds the lower envelope of each band's sites in that band's slots of
//      a stack array (Felzenszwalb-style push with the exact pop test);
//   2. merges the bands left to right, one thread per column: two envelopes
//      over disjoint, ordered site ranges merge into a prefix of the left one
//      and a suffix of the right one, found by popping at the seam until both
//      seam triples are convex (the bridge of two x-separated lower hulls in
//      the dual point set (i, i^2 + g(i)));
//   3. evaluates each band's output elements: a binary search over the merged
//      envelope gives the site that is nearest at the band's first element,
//      then the site pointer only moves forward.
// Each voxel's signed value carries both site sets (sign = its own state,
// magnitude = partial distance to the other state), so one pass produces the
// signed result.
#include <cuda_runtime.h>

#include "edt_common.cuh"

namespace pcdf {
namespace {

constexpr int kBand = 32;  // elements per band
constexpr int kCols = 32;  // columns per CTA

__device__ __forceinline__ int32_t widen(int16_t v)
{
    const int a = v < 0 ? -(int)v : (int)v;
    if (a == kInf16)
        return v < 0 ? -kInf32 : kInf32;
    return v < 0 ? -(a * a) : a * a;
}
__device__ __forceinline__ int32_t widen(int32_t v) { return v; }

// Site value of an element for set 0 (sites: occupied) or set 1 (sites: free);
// an element of the other state is a site with g = 0; -1 = not a site.
__device__ __forceinline__ int site_value(int32_t v, int set)
{
    if (set == 0)
        return v > 0 ? (v == kInf32 ? -1 : v) : 0;
    return v < 0 ? (v == -kInf32 ? -1 : -v) : 0;
}

struct Segs {
    int *start, *len, *cum;  // [band][kCols]
};

__device__ __forceinline__ uint32_t seg_entry(const uint32_t *stk, const Segs &sg, int j, int o, int c)
{
    return stk[(j * kBand + sg.start[j * kCols + c] + o) * kCols + c];
}

// Merge the per-band envelopes of column c into one (bands 0..m-1).
__device__ void merge_bands(const uint32_t *stk, Segs sg, int m, int c)
{
    for (int k = 1; k < m; ++k) {
        for (;;) {
            const int lk = sg.len[k * kCols + c];
            if (lk == 0)
                break;
            int j = k - 1;
            while (j >= 0 && sg.len[j * kCols + c] == 0)
                --j;
            if (j < 0)
                break;
            const int lj = sg.len[j * kCols + c];
            const uint32_t wl = seg_entry(stk, sg, j, lj - 1, c);
            const uint32_t wr = seg_entry(stk, sg, k, 0, c);
            bool has_prev = false;
            uint32_t wp = 0;
            if (lj >= 2) {
                has_prev = true;
                wp = seg_entry(stk, sg, j, lj - 2, c);
            } else {
                int i = j - 1;
                while (i >= 0 && sg.len[i * kCols + c] == 0)
                    --i;
                if (i >= 0) {
                    has_prev = true;
                    wp = seg_entry(stk, sg, i, sg.len[i * kCols + c] - 1, c);
                }
            }
            if (has_prev && dominated(site_of(wp), gval_of(wp), site_of(wl), gval_of(wl), site_of(wr), gval_of(wr))) {
                sg.len[j * kCols + c] = lj - 1;
                continue;
            }
            if (lk >= 2) {
                const uint32_t w2 = seg_entry(stk, sg, k, 1, c);
                if (dominated(site_of(wl), gval_of(wl), site_of(wr), gval_of(wr), site_of(w2), gval_of(w2))) {
                    sg.start[k * kCols + c] += 1;
                    sg.len[k * kCols + c] = lk - 1;
                    continue;
                }
            }
            break;
        }
    }
    int acc = 0;
    for (int k = 0; k < m; ++k) {
        sg.cum[k * kCols + c] = acc;
        acc += sg.len[k * kCols + c];
    }
}

// Forward cursor over the merged envelope of column c.
struct Cursor {
    int q, j;  // global index, band holding it
};

__device__ __forceinline__ uint32_t entry_at(const uint32_t *stk, const Segs &sg, int q, int &j, int c)
{
    j = 0;
    while (q >= sg.cum[j * kCols + c] + sg.len[j * kCols + c])
        ++j;
    return seg_entry(stk, sg, j, q - sg.cum[j * kCols + c], c);
}

template <typename TIn, bool kSdf>
__global__ void __launch_bounds__(kCols * 16)
    k_envelope_banded(const TIn *__restrict__ in, int32_t *__restrict__ out, float *__restrict__ sdf, float vox,
                      int n, int nx, long long ncols, long long outer_stride, long long stride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = (n + kBand - 1) / kBand;
    const int c = threadIdx.x % kCols, b = threadIdx.x / kCols;
    long long *bases = reinterpret_cast<long long *>(smem_raw);          // [kCols]
    int32_t *tile = reinterpret_cast<int32_t *>(bases + kCols);         // [n][kCols]
    uint32_t *stk = reinterpret_cast<uint32_t *>(tile + n * kCols);     // [m*kBand][kCols]
    Segs sg;
    sg.start = reinterpret_cast<int *>(stk + m * kBand * kCols);        // [m][kCols] x 3
    sg.len = sg.start + m * kCols;
    sg.cum = sg.len + m * kCols;

    const long long col0 = (long long)blockIdx.x * kCols;
    if (threadIdx.x < kCols) {
        const long long cl = col0 + threadIdx.x;
        bases[threadIdx.x] = cl < ncols ? (cl / nx) * outer_stride + (cl % nx) : -1;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * kCols; idx += blockDim.x) {
        const int e = idx / kCols, cc = idx % kCols;
        const long long bs = bases[cc];
        tile[idx] = bs >= 0 ? widen(in[bs + (long long)e * stride]) : kInf32;
    }
    __syncthreads();
    const long long base = bases[c];
    const bool live = base >= 0;
    const int e0 = b * kBand, e1 = min(e0 + kBand, n);

    for (int set = 0; set < 2; ++set) {
        bool mine = false;
        if (live)
            for (int e = e0; e < e1; ++e) {
                const int32_t v = tile[e * kCols + c];
                mine |= set == 0 ? v > 0 : v < 0;
            }
        if (!__syncthreads_or(mine))
            continue;

        // 1. band envelope
        int top = -1, s0 = 0, g0 = 0, s1 = 0, g1 = 0;
        if (live) {
            for (int e = e0; e < e1; ++e) {
                const int g = site_value(tile[e * kCols + c], set);
                if (g < 0)
                    continue;
                while (top >= 1 && dominated(s0, g0, s1, g1, e, g)) {
                    --top;
                    s1 = s0;
                    g1 = g0;
                    if (top >= 1) {
                        const uint32_t w = stk[(e0 + top - 1) * kCols + c];
                        s0 = site_of(w);
                        g0 = gval_of(w);
                    }
                }
                ++top;
                stk[(e0 + top) * kCols + c] = pack_site(e, g);
                s0 = s1;
                g0 = g1;
                s1 = e;
                g1 = g;
            }
        }
        sg.start[b * kCols + c] = 0;
        sg.len[b * kCols + c] = top + 1;
        __syncthreads();

        // 2. merge the bands of each column
        if (b == 0 && live)
            merge_bands(stk, sg, m, c);
        __syncthreads();

        // 3. evaluate this band's outputs
        if (live && mine) {
            const int K = sg.cum[(m - 1) * kCols + c] + sg.len[(m - 1) * kCols + c];
            if (K == 0) {
                for (int e = e0; e < e1; ++e) {
                    const int32_t v = tile[e * kCols + c];
                    if (set == 0 ? v > 0 : v < 0) {
                        const int32_t r = set == 0 ? kInf32 : -kInf32;
                        out[base + (long long)e * stride] = r;
                        if (kSdf)
                            sdf[base + (long long)e * stride] = sq_to_sdf(r, vox);
                    }
                }
            } else {
                // nearest site at e0: first q whose successor is not closer
                int lo = 0, hi = K - 1, jj;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    const uint32_t a = entry_at(stk, sg, mid, jj, c);
                    const uint32_t bb = entry_at(stk, sg, mid + 1, jj, c);
                    if (parab(e0, site_of(bb), gval_of(bb)) <= parab(e0, site_of(a), gval_of(a)))
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                int q = lo, j;
                uint32_t cur = entry_at(stk, sg, q, j, c);
                int sc = site_of(cur), gc = gval_of(cur);
                for (int e = e0; e < e1; ++e) {
                    const int32_t v = tile[e * kCols + c];
                    if (!(set == 0 ? v > 0 : v < 0))
                        continue;
                    int fc = parab(e, sc, gc);
                    while (q + 1 < K) {
                        // successor of (q, j)
                        int jn = j, on = q + 1 - sg.cum[j * kCols + c];
                        while (on >= sg.len[jn * kCols + c]) {
                            ++jn;
                            on = 0;
                        }
                        const uint32_t nx_ = seg_entry(stk, sg, jn, on, c);
                        const int fn = parab(e, site_of(nx_), gval_of(nx_));
                        if (fn > fc)
                            break;
                        ++q;
                        j = jn;
                        sc = site_of(nx_);
                        gc = gval_of(nx_);
                        fc = fn;
                    }
                    const int32_t r = set == 0 ? fc : -fc;
                    out[base + (long long)e * stride] = r;
                    if (kSdf)
                        sdf[base + (long long)e * stride] = sq_to_sdf(r, vox);
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
    const int m = (n + kBand - 1) / kBand;
    const size_t smem = kCols * sizeof(long long) + (size_t)n * kCols * 4 + (size_t)m * kBand * kCols * 4 +
                        (size_t)3 * m * kCols * 4;
    cudaError_t e = cudaFuncSetAttribute(k_envelope_banded<TIn, kSdf>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long nblk = (ncols + kCols - 1) / kCols;
    k_envelope_banded<TIn, kSdf><<<(unsigned)nblk, kCols * m, smem, stream>>>(in, out, sdf, vox, n, nx, ncols,
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

// Lower-envelope pass of the exact EDT along y or z: device code shared by the
// stand-alone kernel and the batched persistent kernel (sm_103a).
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
#pragma once

#include "edt_common.cuh"

namespace pcdf {
namespace env {

constexpr int kCols = 32;   // columns per CTA
constexpr int kBands = 4;   // threads per column

// Global loads of stage inputs: through the read-only path, or (kCoherent)
// L2-coherent loads for data written earlier in the same launch.
template <bool kCoherent, class T>
__device__ __forceinline__ T load(const T *p)
{
    if (kCoherent)
        return __ldcg(p);
    return __ldg(p);
}

__device__ __forceinline__ int32_t widen(int16_t v)
{
    const int a = v < 0 ? -(int)v : (int)v;
    if (a == kInf16)
        return v < 0 ? -kInf32 : kInf32;
    return v < 0 ? -(a * a) : a * a;
}
__device__ __forceinline__ int32_t widen(int32_t v) { return v; }

// The merged envelope of a column: band k contributes the entries in slots
// [lo_k + st_k, lo_k + st_k + len_k) of the column's tile; global entry q of
// band k sits in slot q + (lo_k + st_k - (len_0 + ... + len_{k-1})).
struct Merged {
    int c1, c2, c3, K;      // running entry counts after bands 0, 1, 2, 3
    int b0, b1, b2, b3;     // slot offsets
    __device__ __forceinline__ void init(const int (*seg)[kBands][kCols], int c, int wpb, int n)
    {
        const int l0 = seg[1][0][c], l1 = seg[1][1][c], l2 = seg[1][2][c], l3 = seg[1][3][c];
        c1 = l0;
        c2 = c1 + l1;
        c3 = c2 + l2;
        K = c3 + l3;
        b0 = seg[0][0][c];
        b1 = min(wpb * 32, n) + seg[0][1][c] - c1;
        b2 = min(2 * wpb * 32, n) + seg[0][2][c] - c2;
        b3 = min(3 * wpb * 32, n) + seg[0][3][c] - c3;
    }
    __device__ __forceinline__ int slot(int q) const
    {
        return q + (q < c1 ? b0 : (q < c2 ? b1 : (q < c3 ? b2 : b3)));
    }
};
static_assert(kBands == 4, "Merged assumes four bands");

// The CTA (kCols * kBands threads) computes columns [col0, col0 + kCols);
// smem holds kCols * (n + ceil(n / 32)) words.  colmax (non-NULL: every
// column's largest output value, indexed by column) is written at the end.
template <typename TIn, bool kSdf, bool kCoherent>
__device__ __forceinline__ void envelope_tile(const TIn *__restrict__ in, int32_t *__restrict__ out,
                                              float *__restrict__ sdf, float vox, int n, int nx, long long ncols,
                                              long long outer_stride, int stride, long long col0, uint32_t *smem,
                                              int32_t *__restrict__ colmax = nullptr)
{
    __shared__ int seg[2][kBands][kCols];  // per column and band: first surviving entry, number of entries
    __shared__ int32_t s_max[kBands][kCols];
    int32_t mx = INT32_MIN;  // largest value this thread writes
    const int c = threadIdx.x % kCols, band = threadIdx.x / kCols;
    const long long cl = col0 + c;
    const bool live = cl < ncols;
    const long long base = live ? (cl / nx) * outer_stride + (cl % nx) : 0;
    const TIn *col = in + base;
    uint32_t *tile = smem + c;                                  // element e at tile[e * kCols]
    uint32_t *mk = smem + (size_t)n * kCols + c;                // occupied bits, word w at mk[w * kCols]
    const int nw = (n + 31) >> 5;
    const int wpb = (nw + kBands - 1) / kBands;                 // mask words per band
    const int w0 = min(band * wpb, nw), w1 = min(w0 + wpb, nw);
    const int e0 = min(w0 << 5, n), e1 = min(w1 << 5, n);

    // stage this band's slots and their occupancy words
    if (live) {
        for (int w = w0; w < w1; ++w) {
            const int a = w << 5, cnt = min(32, n - a);
            uint32_t occ = 0;
#pragma unroll 8
            for (int i = 0; i < cnt; ++i) {
                const int32_t v = widen(load<kCoherent>(col + (a + i) * stride));
                tile[(a + i) * kCols] = (uint32_t)v;
                occ |= (uint32_t)(v < 0) << i;
            }
            mk[w * kCols] = occ;
        }
    }
    __syncthreads();
    auto valid = [&](int w) { const int cnt = n - (w << 5); return cnt >= 32 ? 0xffffffffu : ((1u << cnt) - 1u); };
    auto occw = [&](int w) { return (w >= 0 && w < nw) ? mk[w * kCols] : 0u; };

    for (int set = 0; set < 2; ++set) {
        // targets: free voxels for set O, occupied voxels for set F
        bool mine = false;
        if (live)
            for (int w = w0; w < w1; ++w) {
                const uint32_t o = occw(w);
                mine |= (set == 0 ? (~o & valid(w)) : o) != 0;
            }
        if (!__syncthreads_or(mine))
            continue;

        // 1. band envelope, in place over slots [e0, e1).  Sites: the targets
        //    with a finite partial distance, and the run ends of the other
        //    state (zero distance) next to a target.
        EnvBuilder B(tile + e0 * kCols, kCols);
        if (live) {
            for (int w = w0; w < w1; ++w) {
                const uint32_t vm = valid(w);
                const uint32_t o = occw(w), op = occw(w - 1), on = occw(w + 1);
                const uint32_t vp = w > 0 ? 0xffffffffu : 0u, vn = w + 1 < nw ? valid(w + 1) : 0u;
                uint32_t tgt, zs;
                if (set == 0) {
                    const uint32_t fr = ~o & vm, frp = ~op & vp, frn = ~on & vn;
                    tgt = fr;
                    zs = o & vm & ((fr << 1) | (frp >> 31) | (fr >> 1) | (frn << 31));
                } else {
                    tgt = o & vm;
                    zs = ~o & vm & ((o << 1) | ((op & vp) >> 31) | (o >> 1) | ((on & vn) << 31));
                    // set O overwrote the slots: restage the values of the targets
                    for (uint32_t m = tgt; m; m &= m - 1) {
                        const int e = (w << 5) + __ffs(m) - 1;
                        tile[e * kCols] = (uint32_t)widen(load<kCoherent>(col + e * stride));
                    }
                }
                for (uint32_t m = tgt | zs; m; m &= m - 1) {
                    const int i = __ffs(m) - 1, e = (w << 5) + i;
                    int g = 0;
                    if ((tgt >> i) & 1u) {
                        const int32_t v = (int32_t)tile[e * kCols];
                        const int32_t a = v < 0 ? -v : v;
                        if (a == kInf32)
                            continue;
                        g = a;
                    }
                    B.push(e, g);
                }
            }
        }
        seg[0][band][c] = 0;
        seg[1][band][c] = B.top + 1;
        __syncthreads();
        // 2. merge the bands of the column (first thread of the column); the
        //    segment table lives in shared memory (indexed by band)
        if (band == 0 && live) {
            int *st = &seg[0][0][c], *len = &seg[1][0][c];  // band k at [k * kCols]
            auto ent = [&](int k, int i) { return tile[(min(k * wpb * 32, n) + st[k * kCols] + i) * kCols]; };
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
            M.init(seg, c, wpb, n);
            int32_t *o = out + base;
            float *f = kSdf ? sdf + base : nullptr;
            int q = 0, sc = 0, gc = 0, sn = 0, gn = 0;
            if (M.K > 0) {
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
                q = lq;
                uint32_t w = tile[M.slot(q) * kCols];
                sc = site_of(w);
                gc = gval_of(w);
                if (q + 1 < M.K) {
                    w = tile[M.slot(q + 1) * kCols];
                    sn = site_of(w);
                    gn = gval_of(w);
                }
            }
            for (int w = w0; w < w1; ++w) {
                const uint32_t ow = occw(w);
                const uint32_t tgt = set == 0 ? (~ow & valid(w)) : ow;
                for (uint32_t m = tgt; m; m &= m - 1) {
                    const int e = (w << 5) + __ffs(m) - 1;
                    int32_t r;
                    if (M.K == 0) {
                        r = kInf32;
                    } else {
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
                                const uint32_t x = tile[M.slot(q + 1) * kCols];
                                sn = site_of(x);
                                gn = gval_of(x);
                            }
                        }
                        r = fc;
                    }
                    r = set == 0 ? r : -r;
                    o[e * stride] = r;
                    mx = max(mx, r);
                    if (kSdf)
                        f[e * stride] = sq_to_sdf_fast(r, vox);
                }
            }
        }
        __syncthreads();
    }
    if (colmax) {  // every thread reaches here (no early exits above)
        s_max[band][c] = mx;
        __syncthreads();
        if (band == 0 && live) {
            int32_t m = s_max[0][c];
#pragma unroll
            for (int k = 1; k < kBands; ++k)
                m = max(m, s_max[k][c]);
            colmax[cl] = m;
        }
        __syncthreads();
    }
}

}  // namespace env
}  // namespace pcdf

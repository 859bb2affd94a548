// Predicted composite fields (Sec. 6 composition, Sec. 8 sequence of fields)
// on sm_103a: device code shared by the stand-alone kernels and the batched
// persistent kernel.
//
// The field of the humans at time t is the exact signed EDT of the voxels
// inside their capsules; its sites all lie in the z-slab [zlo, zlo + S) that
// the capsules touch.  Two kernels build the composite of every t:
//
//  k_dyn_xy      one CTA per (slab slice, t): the exact x-interval of each
//                capsule on every row of the slice, then per column x the
//                y lower envelopes of the row distances to those intervals.
//                Output: the 2-D partial field of the slice (signed int32),
//                with no row-pass intermediate in memory.
//  k_colmax     the largest static value of every column (x, y).
//  k_composite_z thread per (column (x, y), t): the z envelope of the slab's
//                2-D partials, evaluated at every z, min with the static
//                field, float epilogue; the T CTAs that share a static column
//                block run together so that block is read from DRAM once.
//
// The humans' field of a column is never below gmin, the least 2-D partial of
// its slab, and at z outside the slab it is at least gmin plus the squared
// distance to the slab.  Where the column's largest static value does not
// exceed that bound the composite is the static field: a column with
// colmax <= gmin is a copy of the static column, a CTA of such columns copies
// its block with 16-byte accesses, and other columns evaluate the envelope
// only in the z window around the slab where the humans can be nearer.
#pragma once

#include "edt_common.cuh"

#ifndef PCDF_EMIT_CHUNK
#define PCDF_EMIT_CHUNK 6  // static values loaded ahead per lane in the z loops
#endif

namespace pcdf {
namespace comp {


// ---------------------------------------------------------------------------
// k_dyn_xy
// ---------------------------------------------------------------------------
// Shared memory: rows[ny][H + 1] = interval count, then the merged maximal
// occupied runs of the row as (xa << 16 | xb); then a stack of `cap` words per
// thread, laid out [entry][thread].

__device__ __forceinline__ bool row_inside(const int32_t *r, int x)
{
    const int cnt = r[0];
    for (int i = 1; i <= cnt; ++i)
        if (x >= (r[i] >> 16) && x <= (r[i] & 0xFFFF))
            return true;
    return false;
}

// squared distance along the row from x to the nearest occupied voxel (-1: none)
__device__ __forceinline__ int row_g_occ(const int32_t *r, int x)
{
    const int cnt = r[0];
    if (cnt == 0)
        return -1;
    int d = 1 << 20;
    for (int i = 1; i <= cnt; ++i) {
        const int a = r[i] >> 16, b = r[i] & 0xFFFF;
        const int di = x < a ? a - x : (x > b ? x - b : 0);
        d = min(d, di);
    }
    return d * d;
}

// squared distance along the row from an occupied x to the nearest free voxel
// (-1: the whole row is occupied); runs are maximal, so the neighbours of the
// run holding x are free
__device__ __forceinline__ int row_g_free(const int32_t *r, int x, int nx)
{
    const int cnt = r[0];
    for (int i = 1; i <= cnt; ++i) {
        const int a = r[i] >> 16, b = r[i] & 0xFFFF;
        if (x >= a && x <= b) {
            int d = 1 << 20;
            if (a - 1 >= 0)
                d = x - a + 1;
            if (b + 1 <= nx - 1)
                d = min(d, b - x + 1);
            return d == (1 << 20) ? -1 : d * d;
        }
    }
    return 0;
}

// The CTA computes columns [x0, x1) of slab slice s of time t (the capsules'
// runs of every row of the slice are found first; several CTAs can share a
// slice by its columns).  caps_t: the H capsules of t; sm: ny * (H + 1) +
// cap * blockDim.x words.
__device__ __forceinline__ void dyn_xy_slice(const CapInfo *caps_t, int H, int nx, int ny, int zlo, int S, int t,
                                             int s, int cap, int32_t *__restrict__ dyn_mid, int32_t *sm, int x0,
                                             int x1)
{
    __shared__ int s_ylo, s_yhi;
    __shared__ uint32_t s_rowbits[(PCDF_MAX_DIM + 31) / 32];  // rows holding a run
    const int z = zlo + s;
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int rw = H + 1;
    int32_t *rows = sm;
    uint32_t *stk = reinterpret_cast<uint32_t *>(sm + ny * rw) + tid;  // entry q at stk[q * nthr]
    if (tid == 0) {
        s_ylo = ny;
        s_yhi = -1;
    }
    for (int w = tid; w < (ny + 31) / 32; w += nthr)
        s_rowbits[w] = 0;
    __syncthreads();

    // rows: merged occupied runs of every capsule crossing this slice
    for (int y = tid; y < ny; y += nthr) {
        int32_t *r = rows + y * rw;
        int cnt = 0;
        for (int h = 0; h < H; ++h) {
            const CapInfo &ci = caps_t[h];
            if (ci.lo[0] > ci.hi[0] || z < ci.lo[2] || z > ci.hi[2] || y < ci.lo[1] || y > ci.hi[1])
                continue;
            // the capsule is convex, so its voxels on this row form one run
            int xa = -1, xb = -2;
            for (int x = ci.lo[0]; x <= ci.hi[0]; ++x) {
                if (capsule_contains(ci, x, y, z)) {
                    if (xa < 0)
                        xa = x;
                    xb = x;
                } else if (xa >= 0) {
                    break;
                }
            }
            if (xa < 0)
                continue;
            int i = cnt;
            while (i > 0 && (r[i] >> 16) > xa) {
                r[i + 1] = r[i];
                --i;
            }
            r[i + 1] = (xa << 16) | xb;
            ++cnt;
        }
        int m = 0;  // merge overlapping or touching runs
        for (int i = 1; i <= cnt; ++i) {
            const int a = r[i] >> 16, b = r[i] & 0xFFFF;
            if (m > 0 && a <= (r[m] & 0xFFFF) + 1) {
                if (b > (r[m] & 0xFFFF))
                    r[m] = (r[m] & ~0xFFFF) | b;
            } else {
                r[++m] = r[i];
            }
        }
        r[0] = m;
        if (m) {
            atomicMin(&s_ylo, y);
            atomicMax(&s_yhi, y);
            atomicOr(&s_rowbits[y >> 5], 1u << (y & 31));
        }
    }
    __syncthreads();
    const int ylo = s_ylo, yhi = s_yhi;
    const long long V2 = (long long)nx * ny;

    for (int x = x0 + tid; x < x1; x += nthr) {
        int32_t *oc = dyn_mid + ((long long)t * S + s) * V2 + x;  // element y at oc[y * nx]
        if (!PCDF_IN(x, nx) || !PCDF_IN(s, S))
            continue;
        if (yhi < 0) {
            for (int y = 0; y < ny; ++y)
                oc[(long long)y * nx] = kInf32;
            continue;
        }
        int fo = ny, lo_ = -1;  // first / last occupied row of this column
        for (int w = ylo >> 5; w <= yhi >> 5; ++w)
            for (uint32_t b = s_rowbits[w]; b; b &= b - 1) {
                const int y = (w << 5) + __ffs(b) - 1;
                if (row_inside(rows + y * rw, x)) {
                    if (fo == ny)
                        fo = y;
                    lo_ = y;
                }
            }

        // distances to free voxels at the occupied voxels (set F).  Free rows
        // matter only next to an occupied row: the nearest free voxel of any
        // occupied voxel is the first free row out of its run.
        if (lo_ >= 0) {
            const int y0 = max(fo - 1, 0), y1 = min(lo_ + 1, ny - 1);
            EnvBuilder B(stk, nthr, cap);
            bool prev_occ = false;  // y0 - 1 lies before the first occupied row
            bool cur_occ = y0 >= ylo && y0 <= yhi && row_inside(rows + y0 * rw, x);
            for (int y = y0; y <= y1; ++y) {
                const bool next_occ = y + 1 <= y1 && y + 1 >= ylo && y + 1 <= yhi && row_inside(rows + (y + 1) * rw, x);
                int g;
                if (cur_occ)
                    g = row_g_free(rows + y * rw, x, nx);
                else
                    g = (prev_occ || next_occ) ? 0 : -1;
                prev_occ = cur_occ;
                cur_occ = next_occ;
                if (g >= 0)
                    B.push(y, g);
            }
            EnvCursor F(stk, nthr, B.top);
            for (int y = fo; y <= lo_; ++y) {
                if (!row_inside(rows + y * rw, x))
                    continue;
                const int f = F.eval(y);
                if (PCDF_IN(y, ny))
                    oc[(long long)y * nx] = f < 0 ? -kInf32 : -f;
            }
        }

        // distances to occupied voxels at the free voxels (set O): sites are
        // the rows holding a run (g = 0 where x is inside one)
        EnvBuilder B(stk, nthr, cap);
        for (int w = ylo >> 5; w <= yhi >> 5; ++w)
            for (uint32_t b = s_rowbits[w]; b; b &= b - 1) {
                const int y = (w << 5) + __ffs(b) - 1;
                B.push(y, row_g_occ(rows + y * rw, x));
            }
        EnvCursor O(stk, nthr, B.top);  // B.top >= 0: some row of [ylo, yhi] holds a run
        // rows before the column's occupied range, the range (skipping its
        // occupied rows, which set F wrote), rows after it
        const int ya = min(fo, ny), yb = lo_ >= 0 ? lo_ + 1 : ny;
        O.fill(0, ya, oc, nx);
        for (int y = ya; y < yb; ++y)
            if (!row_inside(rows + y * rw, x) && PCDF_IN(y, ny))
                oc[(long long)y * nx] = O.eval(y);
        O.fill(yb, ny, oc, nx);
    }
}

// ---------------------------------------------------------------------------
// k_composite_z
// ---------------------------------------------------------------------------
// Shared memory per thread, [slot][thread]: slots 1..S hold the staged slab
// column (slab element e in slot e + 1); slot 0 and slot S + 1 give the
// in-place stacks room for the sites just below and above the slab; then the
// occupancy bits of the slab column.
//
// Set F (distance to free voxels, output at the voxels inside a human) runs
// first, in place over the staged column, and writes its outputs directly;
// the column is then reloaded and set O (distance to the humans, output
// everywhere else) is built in place and walked along z.  Where the static
// field is nearer than the humans the float output is the static float field
// itself (same value, no square root).

// Output flags: which of the two fields are written, whether the static
// float field is available.
template <bool kSq, bool kSdfOut, bool kStaticSdf>
struct Out {
    int32_t *ocol;
    float *fcol;
    float vox;
    __device__ __forceinline__ void put(int o, int32_t sv, float sf, int32_t d) const
    {
        const int32_t cv = min(sv, d);
        if (kSq)
            __stcs(ocol + o, cv);
        if (kSdfOut) {
            float f;
            if (kStaticSdf && sv <= d)
                f = sf;
            else
                f = sq_to_sdf_fast(cv, vox);
            __stcs(fcol + o, f);
        }
    }
};

template <bool kCoherent, class T>
__device__ __forceinline__ T ldx(const T *p)
{
    if (kCoherent)
        return __ldcg(p);
    return __ldg(p);
}

// Outputs for z in [z0, z1).  kEval: the humans' distance is the envelope O
// where useO holds (else +INF: the static field); kCheck: skip the occupied
// slab voxels where useMk holds (set F wrote them).  Lanes of a warp that
// share the bounds keep the loads and stores of a z coalesced; offsets
// z * V2 stay below 2^31.
template <bool kCheck, bool kEval, bool kCoherent, class O_t>
__device__ __forceinline__ void emit_range(int z0, int z1, EnvCursor &O, bool useO, const uint32_t *mk, bool useMk,
                                           int zlo, int nthr, const int32_t *scol, const float *sfcol, int V2,
                                           const O_t &out, int nz_chk = 1 << 30)
{
    constexpr bool kStaticSdf = O_t::kHaveStatic;
    constexpr int kC = PCDF_EMIT_CHUNK;
    int z = z0;
    for (; z + kC <= z1; z += kC) {
        int32_t sv[kC];
        float sf[kC];
#pragma unroll
        for (int i = 0; i < kC; ++i) {
            const bool ok = PCDF_IN(z + i, nz_chk);
            sv[i] = ok ? ldx<kCoherent>(scol + (z + i) * V2) : kInf32;
            if (kStaticSdf)
                sf[i] = ok ? ldx<kCoherent>(sfcol + (z + i) * V2) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < kC; ++i) {
            const int zz = z + i;
            if (kCheck && useMk) {
                const int e = zz - zlo;
                if ((mk[(e >> 5) * nthr] >> (e & 31)) & 1u)
                    continue;
            }
            const int32_t d = (kEval && useO) ? O.eval(zz) : kInf32;
            if (PCDF_IN(zz, nz_chk))
                out.put(zz * V2, sv[i], kStaticSdf ? sf[i] : 0.f, d);
        }
    }
    for (; z < z1; ++z) {
        if (kCheck && useMk) {
            const int e = z - zlo;
            if ((mk[(e >> 5) * nthr] >> (e & 31)) & 1u)
                continue;
        }
        const int32_t d = (kEval && useO) ? O.eval(z) : kInf32;
        if (PCDF_IN(z, nz_chk))
            out.put(z * V2, ldx<kCoherent>(scol + z * V2), kStaticSdf ? ldx<kCoherent>(sfcol + z * V2) : 0.f, d);
    }
}

// Outputs of one column over [0, nz) with the column's own bounds: below
// its occupied run, the run (skipping its voxels), above it; `empty`: set O
// has no site.
template <bool kCoherent, class O_t>
__device__ __forceinline__ void emit_all(int za, int zb, int nz, bool empty, EnvCursor &O, const uint32_t *mk,
                                         int zlo, int nthr, const int32_t *scol, const float *sfcol, int V2,
                                         const O_t &out)
{
    if (empty) {
        emit_range<false, false, kCoherent>(0, za, O, false, mk, false, zlo, nthr, scol, sfcol, V2, out);
        emit_range<true, false, kCoherent>(za, zb, O, false, mk, true, zlo, nthr, scol, sfcol, V2, out);
        emit_range<false, false, kCoherent>(zb, nz, O, false, mk, false, zlo, nthr, scol, sfcol, V2, out);
    } else {
        emit_range<false, true, kCoherent>(0, za, O, true, mk, false, zlo, nthr, scol, sfcol, V2, out);
        emit_range<true, true, kCoherent>(za, zb, O, true, mk, true, zlo, nthr, scol, sfcol, V2, out);
        emit_range<false, true, kCoherent>(zb, nz, O, true, mk, false, zlo, nthr, scol, sfcol, V2, out);
    }
}

template <bool kSq, bool kSdfOut, bool kStaticSdf>
struct OutT : Out<kSq, kSdfOut, kStaticSdf> {
    static constexpr bool kHaveStatic = kStaticSdf;
};

// 4-byte asynchronous copy global -> shared (no register staging); the
// thread's copies complete at cp_async_wait_all.
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a
// multiple of 16); nothing waits for it.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Largest value of each column c of a field [nz][V2]: warp w of the CTA reads
// the z quarter w of 32 consecutive columns (lane = column).
__device__ __forceinline__ void colmax_block(const int32_t *__restrict__ sq, long long V2, int nz,
                                             int32_t *__restrict__ colmax)
{
    __shared__ int32_t part[4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long c = (long long)blockIdx.x * 32 + lane;
    const int z0 = (int)((long long)nz * w / 4), z1 = (int)((long long)nz * (w + 1) / 4);
    int32_t m = INT32_MIN;
    if (c < V2) {
        const int32_t *col = sq + c;
#pragma unroll 8
        for (int z = z0; z < z1; ++z)
            if (PCDF_IN(z, nz))
                m = max(m, __ldg(col + (long long)z * V2));
    }
    part[w][lane] = m;
    __syncthreads();
    if (w == 0 && c < V2 && PCDF_IN(c, V2))
        colmax[c] = max(max(part[0][lane], part[1][lane]), max(part[2][lane], part[3][lane]));
}

// The static field as the composite of time t on planes [z0, z1) of columns
// [col0, col0 + ncols) (ncols a multiple of 4): 16-byte loads and stores,
// thread tid on the column quad tid % nq of the planes z0 + tid / nq,
// z0 + tid / nq + nthr / nq, ...  Needs V2 % 4 == 0, col0 % 4 == 0 and 16-byte
// aligned fields.
template <bool kSq, bool kSdfOut, bool kStaticSdf, bool kCoherent>
__device__ __forceinline__ void copy_static_planes(const int32_t *__restrict__ static_sq,
                                                   const float *__restrict__ static_sdf, long long V2, int nz, int z0,
                                                   int z1, long long col0, int ncols, int32_t *__restrict__ osq,
                                                   float *__restrict__ osdf, float vox)
{
    const int nq = ncols >> 2;
    const int zstep = blockDim.x / nq;
    const int qd = threadIdx.x % nq, zfirst = threadIdx.x / nq;
    if (zfirst >= zstep)
        return;
    const long long base = col0 + 4 * qd;
#pragma unroll 4
    for (int z = z0 + zfirst; z < z1; z += zstep) {
        const long long o = (long long)z * V2 + base;
        if (!PCDF_IN(o + 3, V2 * nz))
            continue;
        const int4 sv = ldx<kCoherent>(reinterpret_cast<const int4 *>(static_sq + o));
        if (kSq)
            __stcs(reinterpret_cast<int4 *>(osq + o), sv);
        if (kSdfOut) {
            float4 f;
            if (kStaticSdf)
                f = ldx<kCoherent>(reinterpret_cast<const float4 *>(static_sdf + o));
            else
                f = make_float4(sq_to_sdf_fast(sv.x, vox), sq_to_sdf_fast(sv.y, vox), sq_to_sdf_fast(sv.z, vox),
                                sq_to_sdf_fast(sv.w, vox));
            __stcs(reinterpret_cast<float4 *>(osdf + o), f);
        }
    }
}

// Sets F and O of the column staged in tile (slot e + 1 holds slab element
// e).  occ: some slab voxel of the column may lie inside a human; then mk
// receives the occupancy bits, set F is built in place over the staged
// column, its outputs (the occupied voxels) are written and the column is
// staged again.  Set O is then built in place.  Returns the top of the set O
// stack (-1: no site); [za, zb) is the z range of the occupied voxels
// ([nz, nz) if none).
template <bool kCoherent, class O_t>
__device__ __forceinline__ int build_sets(uint32_t *tile, uint32_t *mk, bool occ, int nthr, int S, int nz, int zlo,
                                          const int32_t *scol, const float *sfcol, const int32_t *dcol, long long V2,
                                          const O_t &out, int &za, int &zb, const uint8_t *rep = nullptr)
{
    constexpr bool kStaticSdf = O_t::kHaveStatic;
    const int nw = (S + 31) >> 5;
    const int V2i = (int)V2;
    int firstOcc = S, lastOcc = -1;
    if (occ) {
        for (int w = 0; w < nw; ++w) {
            uint32_t bits = 0;
            const int e0 = w << 5, cnt = min(32, S - e0);
            for (int b = 0; b < cnt; ++b)
                bits |= (uint32_t)((int32_t)tile[(e0 + b + 1) * nthr] < 0) << b;
            mk[w * nthr] = bits;
            if (bits) {
                if (firstOcc == S)
                    firstOcc = e0 + __ffs(bits) - 1;
                lastOcc = e0 + 31 - __clz(bits);
            }
        }
    }
    auto occupied = [&](int z) {
        const int e = z - zlo;
        return occ && e >= 0 && e < S && ((mk[(e >> 5) * nthr] >> (e & 31)) & 1u);
    };

    const int zo0 = zlo + firstOcc, zo1 = zlo + lastOcc;
    if (lastOcc >= 0) {
        // set F over [zo0 - 1, zo1 + 1]; free voxels are sites only next to an
        // occupied one.  Site z sits in slot z - zlo + 1, read before written.
        const int zr0 = max(zo0 - 1, 0), zr1 = min(zo1 + 1, nz - 1);
        EnvBuilder B(tile + (zr0 - zlo + 1) * nthr, nthr, S + 2 - (zr0 - zlo + 1));
        for (int z = zr0; z <= zr1; ++z) {
            int g;
            if (occupied(z)) {
                const int32_t v = (int32_t)tile[(z - zlo + 1) * nthr];
                if (v == -kInf32)
                    continue;
                g = -v;
            } else {
                if (!occupied(z - 1) && !occupied(z + 1))
                    continue;
                g = 0;
            }
            B.push(z, g);
        }
        EnvCursor F(tile + (zr0 - zlo + 1) * nthr, nthr, B.top);
        for (int z = zo0; z <= zo1; ++z) {
            if (!occupied(z))
                continue;
            const int f = F.eval(z);
            const int o = z * V2i;
            if (PCDF_IN(z, nz))
                out.put(o, ldx<kCoherent>(scol + o), kStaticSdf ? ldx<kCoherent>(sfcol + o) : 0.f,
                        f < 0 ? -kInf32 : -f);
        }
        // restore the staged column for set O
#pragma unroll 8
        for (int e = 0; e < S; ++e)
            if (PCDF_IN(rep ? rep[e] : e, S))
                tile[(e + 1) * nthr] = (uint32_t)ldx<kCoherent>(dcol + (long long)(rep ? rep[e] : e) * V2);
    }

    // set O over the slab: sites are the free slab voxels with a finite
    // partial and the ends of the occupied runs (zero distance)
    EnvBuilder B(tile + nthr, nthr, S + 1);
    for (int e = 0; e < S; ++e) {
        const int32_t v = (int32_t)tile[(e + 1) * nthr];
        int g;
        if (v >= 0) {
            if (v == kInf32)
                continue;
            g = v;
        } else {
            const int z = zlo + e;
            if (occupied(z - 1) && occupied(z + 1))
                continue;
            g = 0;
        }
        B.push(zlo + e, g);
    }
    za = lastOcc >= 0 ? zo0 : nz;
    zb = lastOcc >= 0 ? zo1 + 1 : nz;
    return B.top;
}

// The CTA computes columns [col0, col0 + blockDim.x) of time t, one column
// per thread with the column's own z ranges (used inside the batched kernel;
// no block-level synchronisation); smem holds
// blockDim.x * (S + 2 + ceil(S / 32)) words.
template <bool kSq, bool kSdfOut, bool kStaticSdf, bool kCoherent>
__device__ __forceinline__ void composite_block(const int32_t *__restrict__ static_sq,
                                                const float *__restrict__ static_sdf,
                                                const int32_t *__restrict__ dyn_mid, int nx, int ny, int nz, int zlo,
                                                int S, int t, long long col0, int32_t *__restrict__ comp_sq,
                                                float *__restrict__ comp_sdf, float vox, uint32_t *smem,
                                                const uint8_t *__restrict__ rep = nullptr)
{
    const int nthr = blockDim.x, tid = threadIdx.x;
    const long long V2 = (long long)nx * ny;
    const long long c = col0 + tid;
    if (c >= V2)
        return;
    uint32_t *tile = smem + tid;                              // slot k at tile[k * nthr]
    uint32_t *mk = smem + (size_t)(S + 2) * nthr + tid;       // word w at mk[w * nthr]
    const int32_t *dcol = dyn_mid + (long long)t * S * V2 + c;

#pragma unroll 8
    for (int e = 0; e < S; ++e) {
        const int32_t *src = dcol + (long long)(rep ? rep[e] : e) * V2;
        tile[(e + 1) * nthr] = (uint32_t)(kCoherent ? __ldcg(src) : __ldcs(src));
    }

    const long long V = V2 * nz;
    const int32_t *scol = static_sq + c;
    const float *sfcol = kStaticSdf ? static_sdf + c : nullptr;
    OutT<kSq, kSdfOut, kStaticSdf> out;
    out.ocol = kSq ? comp_sq + (long long)t * V + c : nullptr;
    out.fcol = kSdfOut ? comp_sdf + (long long)t * V + c : nullptr;
    out.vox = vox;
    int za, zb;
    const int top = build_sets<kCoherent>(tile, mk, true, nthr, S, nz, zlo, scol, sfcol, dcol, V2, out, za, zb, rep);
    EnvCursor O(tile + nthr, nthr, top);
    emit_all<kCoherent>(za, zb, nz, top < 0, O, mk, zlo, nthr, scol, sfcol, (int)V2, out);
}

// The CTA of k_composite_z: columns [col0, col0 + blockDim.x) of time t with
// the static shortcuts.  colmax: the largest static value of every column;
// rep (nullable: the identity): slab element e of time t is stored in slice
// rep[e] (slices of equal capsule cross-sections computed once); vec: the
// CTA may copy with 16-byte accesses.  pf_parts > 0 (needs vec): the CTA
// first asks L2 to prefetch planes pf_part, pf_part + pf_parts, ... of its
// static column block (bulk prefetches, no registers held), so that the
// CTAs that share the block (one per t) split the block between them and
// their loads of it hit L2.  Block-wide barriers: every thread of the CTA
// calls.
//  * every column static (colmax <= gmin): the CTA copies the static block;
//  * else each column with dynamic influence has a window [w0, w1) (the slab
//    and every z less than R slices from it, R the least integer with
//    gmin + R^2 >= colmax; beyond it the static field wins).  Outside the
//    union of the windows the block is copied (16-byte accesses when vec,
//    else per column); inside it every lane of a warp runs the same z loops,
//    so the accesses of a z stay coalesced, with the envelope (+INF for the
//    static columns).
template <bool kSq, bool kSdfOut, bool kStaticSdf>
__device__ __forceinline__ void composite_block_short(const int32_t *__restrict__ static_sq,
                                                      const float *__restrict__ static_sdf,
                                                      const int32_t *__restrict__ colmax,
                                                      const int32_t *__restrict__ dyn_mid,
                                                      const uint8_t *__restrict__ rep, int nx, int ny, int nz,
                                                      int zlo, int S, int t, long long col0,
                                                      int32_t *__restrict__ comp_sq, float *__restrict__ comp_sdf,
                                                      float vox, bool vec, uint32_t *smem, int pf_part = 0,
                                                      int pf_parts = 0)
{
    __shared__ int s_w0, s_w1, s_occ;
    const int nthr = blockDim.x, tid = threadIdx.x;
    const long long V2 = (long long)nx * ny;
    const long long c = col0 + tid;
    const bool live = c < V2;
    if (pf_parts > 0) {
        // the block's columns of one plane: a multiple of 16 bytes from a
        // 16-byte boundary (V2 % 4 == 0, col0 % 4 == 0, aligned fields)
        const uint32_t nb = (uint32_t)min((long long)nthr, V2 - col0) * 4u;
        for (int z = pf_part + pf_parts * tid; z < nz; z += pf_parts * nthr) {
            const long long o = (long long)z * V2 + col0;
            if (!PCDF_IN(o + nb / 4 - 1, V2 * nz))
                continue;
            prefetch_l2(static_sq + o, nb);
            if (kStaticSdf)
                prefetch_l2(static_sdf + o, nb);
        }
    }
    uint32_t *tile = smem + tid;                              // slot k at tile[k * nthr]
    uint32_t *mk = smem + (size_t)(S + 2) * nthr + tid;       // word w at mk[w * nthr]
    const int32_t *dcol = dyn_mid + (long long)t * S * V2 + c;
    const long long V = V2 * nz;
    if (tid == 0) {
        s_w0 = nz;
        s_w1 = 0;
        s_occ = 0;
    }

    // stage the slab column with every load in flight at once
    int32_t gmin = kInf32;
    const int32_t cmax = live && PCDF_IN(c, V2) ? __ldg(colmax + c) : kInf32;
    if (live) {
        for (int e = 0; e < S; ++e)
            if (PCDF_IN(rep ? rep[e] : e, S))
                cp_async4(tile + (e + 1) * nthr, dcol + (long long)(rep ? rep[e] : e) * V2);
        cp_async_wait_all();
#pragma unroll 8
        for (int e = 0; e < S; ++e)
            gmin = min(gmin, (int32_t)tile[(e + 1) * nthr]);
    }
    // the humans' field of the column is >= gmin everywhere
    const bool col_static = cmax <= gmin;
    const int32_t *scol = static_sq + c;
    const float *sfcol = kStaticSdf ? static_sdf + c : nullptr;
    OutT<kSq, kSdfOut, kStaticSdf> out;
    out.ocol = kSq ? comp_sq + (long long)t * V + c : nullptr;
    out.fcol = kSdfOut ? comp_sdf + (long long)t * V + c : nullptr;
    out.vox = vox;
    const int V2i = (int)V2;
    if (__syncthreads_and(!live || col_static)) {
        if (vec) {
            copy_static_planes<kSq, kSdfOut, kStaticSdf, false>(
                static_sq, static_sdf, V2, nz, 0, nz, col0, (int)min((long long)nthr, V2 - col0),
                kSq ? comp_sq + (long long)t * V : nullptr, kSdfOut ? comp_sdf + (long long)t * V : nullptr, vox);
        } else if (live) {
            EnvCursor none(tile, nthr, -1);
            emit_range<false, false, false>(0, nz, none, false, mk, false, zlo, nthr, scol, sfcol, V2i, out, nz);
        }
        return;
    }

    const bool dyn = live && !col_static;
    const bool occ = dyn && gmin < 0;  // some slab voxel of the column lies inside a human
    if (dyn) {
        int w0 = 0, w1 = nz;
        const long long diff = (long long)cmax - gmin;  // > 0
        if (diff < (long long)nz * nz) {
            int R = (int)sqrtf((float)diff);
            while ((long long)R * R < diff)
                ++R;
            while (R > 1 && (long long)(R - 1) * (R - 1) >= diff)
                --R;
            w0 = max(zlo - R + 1, 0);
            w1 = min(zlo + S + R - 1, nz);
        }
        atomicMin(&s_w0, w0);
        atomicMax(&s_w1, w1);
        if (occ)
            s_occ = 1;
    }
    __syncthreads();
    const int ww0 = s_w0, ww1 = s_w1;  // some column is dynamic: ww0 <= zlo, ww1 >= zlo + S
    const bool any_occ = s_occ != 0;
    // the planes outside the window union are copies of the static block:
    // 16-byte accesses by all threads first (the CTA's per-column loops below
    // are what its time depends on)
    if (vec) {
        const int nc = (int)min((long long)nthr, V2 - col0);
        int32_t *osq = kSq ? comp_sq + (long long)t * V : nullptr;
        float *osdf = kSdfOut ? comp_sdf + (long long)t * V : nullptr;
        copy_static_planes<kSq, kSdfOut, kStaticSdf, false>(static_sq, static_sdf, V2, nz, 0, ww0, col0, nc, osq,
                                                            osdf, vox);
        copy_static_planes<kSq, kSdfOut, kStaticSdf, false>(static_sq, static_sdf, V2, nz, ww1, nz, col0, nc, osq,
                                                            osdf, vox);
    }
    if (!live)
        return;  // no block-level synchronisation below

    int top = -1;  // set O stack top (-1: no site, or a static column)
    if (dyn) {
        int za, zb;
        top = build_sets<false>(tile, mk, occ, nthr, S, nz, zlo, scol, sfcol, dcol, V2, out, za, zb, rep);
    }
    EnvCursor O(tile + nthr, nthr, top);
    const bool useO = top >= 0;
    const int sa = zlo, sb = zlo + S;
    if (!vec)
        emit_range<false, false, false>(0, ww0, O, false, mk, false, zlo, nthr, scol, sfcol, V2i, out, nz);
    emit_range<false, true, false>(ww0, sa, O, useO, mk, false, zlo, nthr, scol, sfcol, V2i, out, nz);
    if (any_occ)  // skip the occupied slab voxels (set F wrote them)
        emit_range<true, true, false>(sa, sb, O, useO, mk, occ, zlo, nthr, scol, sfcol, V2i, out, nz);
    else
        emit_range<false, true, false>(sa, sb, O, useO, mk, false, zlo, nthr, scol, sfcol, V2i, out, nz);
    emit_range<false, true, false>(sb, ww1, O, useO, mk, false, zlo, nthr, scol, sfcol, V2i, out, nz);
    if (!vec)
        emit_range<false, false, false>(ww1, nz, O, false, mk, false, zlo, nthr, scol, sfcol, V2i, out, nz);
}

}  // namespace comp
}  // namespace pcdf

// Run-split banded lower envelopes along one axis: the y and z passes of the
// exact EDT of the static map and of the from-scratch comparator (Sec. 6:
// the environment's exact distance field; the full per-field recompute).
//
// Input: a CTA's tile of kCols columns of n elements in shared memory, element
// e of column c at tile[e * kCols + c].  Each is a signed value v: v >= 0 a
// free voxel whose partial squared distance to the nearest occupied voxel
// (over the axes already done) is v, v < 0 an occupied voxel whose partial
// squared distance to the nearest free voxel is -v; magnitude kInf32 means
// "none".  Output, per element, the squared distance with this axis added,
// same sign convention.
//
// Runs.  At a free voxel e of a maximal free run [a, b] the result is
//   min( min over s in [a, b] with finite G(s) of (e - s)^2 + G(s),
//        (e - (a - 1))^2 if a > 0,  ((b + 1) - e)^2 if b + 1 < n )
// because the occupied voxels a - 1 and b + 1 are sites at distance zero and
// every site beyond one of them is farther from e than it is.  Occupied runs
// and their free neighbours behave the same way.  So every run is its own
// lower-envelope problem over its own sites, the two voxels that bound it
// enter as plain distances, and free and occupied voxels are handled in the
// same sweep.
//
// Bands.  kB threads per column each own a band of L elements (L a multiple
// of 32, so a band owns whole words of the column's occupancy bit mask).
//  1. Build: a band walks its elements once.  For every piece (a run cut to
//     the band) it keeps the lower envelope of the piece's sites as a stack
//     stored in place over the piece's own slots: entry q of a piece that
//     starts at slot a lives in slot a + q, at or before the element being
//     read.  A piece that ends inside the band and whose stack does not reach
//     its last slot writes its entry count there, tagged with the top bit
//     (no packed entry has it).  The band's first and last pieces, which may
//     continue a run across a band seam, are recorded in a table.
//  2. Merge: one thread per column visits the seams left to right.  Where a
//     run crosses a seam, the chain of pieces on the left (reaching back over
//     bands that the run spans whole) and the first piece on the right are
//     joined by popping at the seam until both seam triples are convex: the
//     bridge of two x-separated lower hulls of the points (s, s^2 + G(s)).
//  3. Eval: a band walks its elements again.  For each piece a cursor runs
//     over the run's chain of pieces.  A piece that continues a run from the
//     left starts at the entry nearest its first element, found by walking
//     back from the seam (the envelope's values at a fixed point decrease to
//     the minimum and then increase, since its breakpoints are strictly
//     increasing after the pops).
#pragma once

#include "edt_common.cuh"

namespace pcdf {
namespace lean {

constexpr int kCols = 32;               // columns per CTA (one lane each)
constexpr uint32_t kMark = 0x80000000u;  // entry-count tag in a piece's last slot
constexpr int kFar = 1 << 20;           // "no boundary voxel" coordinate offset
constexpr int kMaxSide = 512;           // longest axis (PCDF_MAX_DIM)

enum : int { kSingle = 1, kFirstOcc = 2, kLastOcc = 4, kEmpty = 8 };

// Per band and column: the first piece (start slot, entries), the last piece
// (unused when kSingle: the band is one piece) and flags.  16-bit entries
// (slots and counts are at most kMaxSide), so that the table takes half the
// shared memory of 32-bit ones.
template <int kB>
struct alignas(16) Seg {
    int16_t fS[kB][kCols], fK[kB][kCols];
    int16_t lS[kB][kCols], lK[kB][kCols];
    int16_t fl[kB][kCols];
};

PCDF_HD int clz32(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return __clz(x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}
PCDF_HD int ffs32(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return __ffs(x);
#else
    return __builtin_ffs(x);
#endif
}

// band length: ceil(n / kB) rounded up to a multiple of 32
PCDF_HD int band_len(int n, int kB) { return ((n + kB - 1) / kB + 31) & ~31; }

// Occupancy bit of element e; the column's mask word w is at m[w * kCols].
PCDF_HD bool occ_bit(const uint32_t *m, int e) { return (m[(e >> 5) * kCols] >> (e & 31)) & 1u; }

// Smallest e' > e whose state differs from st, or n.
PCDF_HD int next_change(const uint32_t *m, int e, bool st, int n)
{
    int w = e >> 5;
    uint32_t d = (st ? ~m[w * kCols] : m[w * kCols]) & (0xFFFFFFFEu << (e & 31));
    while (!d) {
        ++w;
        if ((w << 5) >= n || !PCDF_IN(w, (n + 31) >> 5))
            return n;
        d = st ? ~m[w * kCols] : m[w * kCols];
    }
    const int p = (w << 5) + ffs32(d) - 1;
    return p < n ? p : n;
}

// First element of the run holding e (state st): one past the largest e' < e
// of the other state, or 0.
PCDF_HD int run_start(const uint32_t *m, int e, bool st)
{
    int w = e >> 5;
    uint32_t d = (st ? ~m[w * kCols] : m[w * kCols]) & ((1u << (e & 31)) - 1u);
    while (!d) {
        if (w == 0)
            return 0;
        --w;
        d = st ? ~m[w * kCols] : m[w * kCols];
    }
    return (w << 5) + 31 - clz32(d) + 1;
}

// 1. Build the band's piece envelopes (thread of column c, band b).
template <int kB>
PCDF_HD void build_band(uint32_t *tile, Seg<kB> &S, int n, int L, int c, int b)
{
    const int e0 = b * L, e1 = min(e0 + L, n);
    if (e0 >= e1) {
        S.fl[b][c] = kEmpty | kSingle;
        S.fS[b][c] = S.lS[b][c] = e0;
        S.fK[b][c] = S.lK[b][c] = 0;
        return;
    }
    uint32_t *col = tile + c;
    int a = e0, top = -1;            // current piece: first slot, index of its top entry
    int s0 = 0, f0 = 0, s1 = 0, f1 = 0;  // top two entries: site and s^2 + G
    bool cur = (int32_t)col[e0 * kCols] < 0;
    const bool first_occ = cur;
    bool first_open = true;
    for (int e = e0; e < e1; ++e) {
        const int32_t v = PCDF_IN(e, n) ? (int32_t)col[e * kCols] : kInf32;
        const bool st = v < 0;
        if (st != cur) {  // the piece [a, e) ends
            if (first_open) {
                S.fS[b][c] = e0;
                S.fK[b][c] = top + 1;
                first_open = false;
            } else if (top + 1 < e - a && PCDF_IN(e - 1, n)) {
                col[(e - 1) * kCols] = kMark | (uint32_t)(top + 1);
            }
            a = e;
            top = -1;
            cur = st;
        }
        const int g = st ? -v : v;
        if (g == kInf32)
            continue;
        const int f = e * e + g;
        // pop while the top entry is nowhere strictly below both neighbours
        while (top >= 1 && (f - f1) * (s1 - s0) <= (f1 - f0) * (e - s1)) {
            --top;
            s1 = s0;
            f1 = f0;
            if (top >= 1) {
                const uint32_t w = PCDF_IN(a + top - 1, n) ? col[(a + top - 1) * kCols] : 0u;
                s0 = site_of(w);
                f0 = s0 * s0 + gval_of(w);
            }
        }
        ++top;
        if (PCDF_IN(a + top, n))
            col[(a + top) * kCols] = pack_site(e, g);
        s0 = s1;
        f0 = f1;
        s1 = e;
        f1 = f;
    }
    int fl = (first_occ ? kFirstOcc : 0) | (cur ? kLastOcc : 0);
    if (first_open) {
        fl |= kSingle;
        S.fS[b][c] = e0;
        S.fK[b][c] = top + 1;
    }
    S.lS[b][c] = a;
    S.lK[b][c] = top + 1;
    S.fl[b][c] = fl;
}

// Navigation over the pieces of one run in the table of column c.
template <int kB>
struct Chain {
    const uint32_t *col;
    Seg<kB> *S;
    int c;
    int n;  // slots of the column (bounds checks)

    struct Pos {
        int j, start, slot, end;  // band, first slot of the piece, current slot, one past its last slot
        bool first, last;         // the piece is band j's first / last piece
    };

    PCDF_HD bool single(int j) const { return (S->fl[j][c] & kSingle) != 0; }
    // does a run cross the seam in front of band j?
    PCDF_HD bool cont(int j) const
    {
        if (j <= 0 || j >= kB || (S->fl[j][c] & kEmpty))
            return false;
        return ((S->fl[j - 1][c] & kLastOcc) != 0) == ((S->fl[j][c] & kFirstOcc) != 0);
    }
    PCDF_HD int lastS(int j) const { return single(j) ? S->fS[j][c] : S->lS[j][c]; }
    PCDF_HD int lastK(int j) const { return single(j) ? S->fK[j][c] : S->lK[j][c]; }

    // the first nonempty piece from band j's first piece on (across seam j),
    // among bands < hi
    PCDF_HD bool seek_right(int j, Pos &p, int hi = kB) const
    {
        for (;;) {
            if (j >= hi || !cont(j))
                return false;
            const int K = S->fK[j][c];
            if (K > 0) {
                p.j = j;
                p.start = p.slot = S->fS[j][c];
                p.end = p.start + K;
                p.first = true;
                p.last = single(j);
                return true;
            }
            if (!single(j))
                return false;
            ++j;
        }
    }
    // the last nonempty piece from band j's last piece back (the run crosses
    // seam j + 1), among bands >= lo; p at its last entry
    PCDF_HD bool seek_left(int j, Pos &p, int lo = 0) const
    {
        for (;;) {
            if (j < lo)
                return false;
            const int K = lastK(j);
            if (K > 0) {
                p.j = j;
                p.start = lastS(j);
                p.end = p.start + K;
                p.slot = p.end - 1;
                p.first = single(j);
                p.last = true;
                return true;
            }
            if (!single(j) || !cont(j))
                return false;
            --j;
        }
    }
    PCDF_HD bool next(const Pos &p, Pos &q, int hi = kB) const
    {
        if (p.slot + 1 < p.end) {
            q = p;
            ++q.slot;
            return true;
        }
        return p.last && seek_right(p.j + 1, q, hi);
    }
    PCDF_HD bool prev(const Pos &p, Pos &q, int lo = 0) const
    {
        if (p.slot > p.start) {
            q = p;
            --q.slot;
            return true;
        }
        return p.first && cont(p.j) && seek_left(p.j - 1, q, lo);
    }
    PCDF_HD uint32_t at(const Pos &p) const { return PCDF_IN(p.slot, n) ? col[p.slot * kCols] : 0u; }
};

// 2. Join the envelopes across seam b, where a run crosses it: the left chain
// lies in bands [lo, b), the right chain in bands [b, hi), each already one
// envelope.  The seams are merged as a tree: in round r (step 2^r) the seams
// b = step, 3 step, 5 step, ... join groups of `step` bands on either side,
// so the rounds of one column run on different threads in parallel.
template <int kB>
PCDF_HD void merge_seam(uint32_t *tile, Seg<kB> &S, int n, int c, int b, int lo, int hi)
{
    Chain<kB> ch{tile + c, &S, c, n};
    if (!ch.cont(b))
        return;
    using Pos = typename Chain<kB>::Pos;
    // the seam's entries: P, L on the left (L last), R, Q on the right (R first)
    Pos L, R, P, Q;
    if (!ch.seek_left(b - 1, L, lo) || !ch.seek_right(b, R, hi))
        return;
    uint32_t wl = ch.at(L), wr = ch.at(R), wp = 0, w2 = 0;
    bool hp = ch.prev(L, P, lo), hq = ch.next(R, Q, hi);
    if (hp)
        wp = ch.at(P);
    if (hq)
        w2 = ch.at(Q);
    for (;;) {
        if (hp && dominated(site_of(wp), gval_of(wp), site_of(wl), gval_of(wl), site_of(wr), gval_of(wr))) {
            if (ch.single(L.j))  // L leaves the end of its piece
                --S.fK[L.j][c];
            else
                --S.lK[L.j][c];
            L = P;
            wl = wp;
            hp = ch.prev(L, P, lo);
            if (hp)
                wp = ch.at(P);
            continue;
        }
        if (hq && dominated(site_of(wl), gval_of(wl), site_of(wr), gval_of(wr), site_of(w2), gval_of(w2))) {
            ++S.fS[R.j][c];  // R leaves the front of its piece
            --S.fK[R.j][c];
            R = Q;
            wr = w2;
            hq = ch.next(R, Q, hi);
            if (hq)
                w2 = ch.at(Q);
            continue;
        }
        break;
    }
}

// The seam merged by thread t (0-based) of round r, or 0 if none.
PCDF_HD int tree_seam(int kB, int r, int t) { const int b = (2 * t + 1) << r; return b < kB ? b : 0; }

// 3. Evaluate the band (thread of column c, band b); out(e, value) for every
// element of the band, in increasing e.  mk: the column-major occupancy
// words of the tile.  Returns the functor (with whatever it accumulated).
template <int kB, class Out>
PCDF_HD Out eval_band(uint32_t *tile, const uint32_t *mk, Seg<kB> &S, int n, int L, int c, int b, Out out)
{
    const int e0 = b * L, e1 = min(e0 + L, n);
    if (e0 >= e1)
        return out;
    Chain<kB> ch{tile + c, &S, c, n};
    using Pos = typename Chain<kB>::Pos;
    const uint32_t *m = mk + c;
    int e = e0;
    while (e < e1) {
        const bool st = occ_bit(m, e);
        const int nc = next_change(m, e, st, n);
        const int se = min(nc, e1) - 1;  // this piece: [e, se]
        const bool is_first = e == e0, is_last = se == e1 - 1;
        const int ra = is_first && e0 > 0 ? run_start(m, e0, st) : e;
        const int rb = nc - 1;
        const int bl = ra > 0 ? ra - 1 : -kFar, br = rb + 1 < n ? rb + 1 : kFar;

        // this piece's own entries
        Pos own;
        own.j = b;
        own.first = is_first;
        own.last = is_last;
        int K;
        if (is_first) {
            own.start = S.fS[b][c];
            K = S.fK[b][c];
        } else if (is_last) {
            own.start = S.lS[b][c];
            K = S.lK[b][c];
        } else {
            own.start = e;
            const uint32_t w = PCDF_IN(se, n) ? tile[se * kCols + c] : 0u;
            K = (w & kMark) ? (int)(w & ~kMark) : se - e + 1;
        }
        own.slot = own.start;
        own.end = own.start + K;

        Pos cur;
        bool have;
        if (ra < e && ch.seek_left(b - 1, cur)) {
            // continue a run from the left: walk back to the entry nearest e
            uint32_t w = ch.at(cur);
            int fc = parab(e, site_of(w), gval_of(w));
            Pos p;
            while (ch.prev(cur, p)) {
                const uint32_t wp = ch.at(p);
                const int fp = parab(e, site_of(wp), gval_of(wp));
                if (fp > fc)
                    break;
                cur = p;
                fc = fp;
            }
            have = true;
        } else if (K > 0) {
            cur = own;
            have = true;
        } else {
            have = is_last && ch.seek_right(b + 1, cur);
        }

        // current entry (s, g); next entry (sn, gn) at slot nslot of the piece
        // ending before nend (band nj; nlast: band nj's last piece)
        int s = 0, g = 0, sn = 0, gn = 0, nslot = 0, nend = 0, nj = 0;
        bool hn = false, nlast = false;
        if (have) {
            const uint32_t w = ch.at(cur);
            s = site_of(w);
            g = gval_of(w);
            if (cur.slot + 1 < cur.end) {
                hn = true;
                nslot = cur.slot + 1;
                nend = cur.end;
                nj = cur.j;
                nlast = cur.last;
            } else {
                Pos q;
                hn = cur.last && ch.seek_right(cur.j + 1, q);
                if (hn) {
                    nslot = q.slot;
                    nend = q.end;
                    nj = q.j;
                    nlast = q.last;
                }
            }
            if (hn) {
                const uint32_t w2 = PCDF_IN(nslot, n) ? tile[nslot * kCols + c] : 0u;
                sn = site_of(w2);
                gn = gval_of(w2);
            }
        }
        const int sgn = st ? -1 : 0;  // r -> -r for occupied voxels: (r ^ sgn) - sgn
        for (int z = e; z <= se; ++z) {
            int r = kInf32;
            if (have) {
                int fc = parab(z, s, g);
                while (hn) {
                    const int fn = parab(z, sn, gn);
                    if (fn > fc)
                        break;
                    s = sn;
                    g = gn;
                    fc = fn;
                    if (nslot + 1 < nend) {
                        ++nslot;
                    } else {
                        Pos q;
                        hn = nlast && ch.seek_right(nj + 1, q);
                        if (hn) {
                            nslot = q.slot;
                            nend = q.end;
                            nj = q.j;
                            nlast = q.last;
                        }
                    }
                    if (hn) {
                        const uint32_t w2 = PCDF_IN(nslot, n) ? tile[nslot * kCols + c] : 0u;
                        sn = site_of(w2);
                        gn = gval_of(w2);
                    }
                }
                r = fc;
            }
            const int d = min(z - bl, br - z);
            r = min(r, d <= kMaxSide ? d * d : kInf32);
            out(z, (r ^ sgn) - sgn);
        }
        e = se + 1;
    }
    return out;
}

}  // namespace lean
}  // namespace pcdf

/*
 * oracle.c -- plain CPU oracle for predicted composite distance fields.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it, and it shares no
 * code, header or table with that path.
 *
 * Every routine is single-threaded, unblocked C written from the definitions
 * of the method (Sec. 6 "Mapping - Predicted Composite Distance Fields" and
 * the GPMP2 obstacle factor of Sec. 7):
 *
 *   - capsule occupancy: exact int64 point-to-segment test, and the paper's
 *     own human primitive, the finite cylinder (Sec. 6), selected by a flag
 *     in the radius word.
 *   - signed squared Euclidean distance transform (EDT), by its definition
 *     (brute-force minimum over all in-grid voxels of the opposite state) and
 *     by the separable lower-envelope algorithm of Meijster, Roerdink and
 *     Hesselink (2000), which the test suite pins against the definition.
 *   - composite field = per-voxel minimum of the static field and the field of
 *     the dynamic obstacles at one predicted time (Sec. 6).
 *   - float field = sign(S) * sqrtf(|S|) * voxel size, in IEEE fp32.
 *   - trilinear sampling, hinge obstacle cost and its gradient with respect to
 *     the sphere centre, in double precision (Sec. 7, hinge form of the
 *     robot-avoidance factor, applied to the environment field as in GPMP2).
 *   - the static-map clean-up of Sec. 8: occupied voxels with fewer than a
 *     given number of occupied voxels among their 26 neighbours are cleared.
 *   - the 2-D map of Sec. 8: the 3-D grid collapsed over a range of slices
 *     (a column is occupied if any of its voxels in the range is), whose EDT
 *     is the 3-D EDT above on a grid one slice thick.
 *
 * Conventions (shared with the library by specification, not by code):
 *   grid index v = (k*ny + j)*nx + i, x fastest; voxel (i,j,k) has its centre
 *   at origin + (i+1/2, j+1/2, k+1/2)*vox.  S(v) = +min |v-u|^2 over occupied
 *   in-grid u if v is free, -min |v-u|^2 over free in-grid u if v is
 *   occupied, in voxel-index units; an empty opposite set gives +/-INT32_MAX.
 *   Capsule = 7 int32 in 1/16-voxel fixed point relative to the grid corner
 *   (a_xyz, b_xyz, radius); the centre of voxel (i,j,k) is 16*(i,j,k)+8.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_INF32 2147483647
#define OR_BIG ((int64_t)1 << 60) /* "no site" marker inside the oracle */
#define OR_CYLINDER (1 << 30)       /* radius-word flag: finite cylinder instead of capsule */

/* ------------------------------------------------------------------------ */
/* Capsule occupancy                                                         */
/* ------------------------------------------------------------------------ */

/* Is the fixed-point point p inside the closed capsule (segment a-b, radius r)?
 * With the cylinder flag in the radius word: inside the closed finite
 * cylinder of radius r around a-b, flat ends through a and b.
 * The squared distance from p to the segment is compared with r^2 exactly:
 *   projection parameter s = (p-a).(b-a), L = |b-a|^2;
 *   s <= 0 (or L == 0): nearest point is a;  s >= L: nearest point is b;
 *   otherwise |p-a|^2 - s^2/L <= r^2, multiplied through by L > 0. */
int or_capsule_inside(int64_t px, int64_t py, int64_t pz, const int32_t *cap)
{
    const int cylinder = (cap[6] & OR_CYLINDER) != 0;
    const int64_t ax = cap[0], ay = cap[1], az = cap[2];
    const int64_t bx = cap[3], by = cap[4], bz = cap[5], r = cap[6] & ~OR_CYLINDER;
    const int64_t wx = px - ax, wy = py - ay, wz = pz - az;
    const int64_t dx = bx - ax, dy = by - ay, dz = bz - az;
    const int64_t L = dx * dx + dy * dy + dz * dz;
    const int64_t s = wx * dx + wy * dy + wz * dz;
    const int64_t ww = wx * wx + wy * wy + wz * wz;
    if (cylinder) /* closed finite cylinder (Sec. 6): 0 <= s <= L, distance to the line <= r */
        return L > 0 && s >= 0 && s <= L && ww * L - s * s <= r * r * L;
    if (L == 0 || s <= 0)
        return ww <= r * r;
    if (s >= L) {
        const int64_t ex = px - bx, ey = py - by, ez = pz - bz;
        return ex * ex + ey * ey + ez * ez <= r * r;
    }
    return ww * L - s * s <= r * r * L;
}

/* occ[v] |= 1 for every voxel whose centre lies inside any of the H capsules. */
void or_capsule_occupancy(int nx, int ny, int nz, int H, const int32_t *caps, uint8_t *occ)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t px = 16 * (int64_t)i + 8, py = 16 * (int64_t)j + 8, pz = 16 * (int64_t)k + 8;
                for (int h = 0; h < H; ++h)
                    if (or_capsule_inside(px, py, pz, caps + 7 * h)) {
                        occ[((size_t)k * ny + j) * nx + i] = 1;
                        break;
                    }
            }
}

/* ------------------------------------------------------------------------ */
/* Signed squared EDT by its definition                                      */
/* ------------------------------------------------------------------------ */

/* S at one voxel: minimum squared distance to an in-grid voxel of the other
 * state, signed by the voxel's own state.  O(V) per voxel. */
int32_t or_edt_at(int nx, int ny, int nz, const uint8_t *occ, int i, int j, int k)
{
    const int mine = occ[((size_t)k * ny + j) * nx + i] != 0;
    int64_t best = OR_BIG;
    for (int kk = 0; kk < nz; ++kk)
        for (int jj = 0; jj < ny; ++jj)
            for (int ii = 0; ii < nx; ++ii) {
                if ((occ[((size_t)kk * ny + jj) * nx + ii] != 0) == mine)
                    continue;
                const int64_t d = (int64_t)(ii - i) * (ii - i) + (int64_t)(jj - j) * (jj - j) +
                                  (int64_t)(kk - k) * (kk - k);
                if (d < best)
                    best = d;
            }
    const int32_t mag = best == OR_BIG ? OR_INF32 : (int32_t)best;
    return mine ? -mag : mag;
}

/* Whole field by the definition: for every voxel, scan the list of voxels of
 * the other state.  O(V * |other|); meant for grids of a few ten thousand
 * voxels. */
void or_edt_brute(int nx, int ny, int nz, const uint8_t *occ, int32_t *S)
{
    const size_t V = (size_t)nx * ny * nz;
    int32_t *occ_xyz = (int32_t *)malloc(3 * V * sizeof(int32_t));
    int32_t *free_xyz = (int32_t *)malloc(3 * V * sizeof(int32_t));
    size_t n_occ = 0, n_free = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int32_t *dst = occ[((size_t)k * ny + j) * nx + i] ? occ_xyz + 3 * n_occ++ : free_xyz + 3 * n_free++;
                dst[0] = i;
                dst[1] = j;
                dst[2] = k;
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t v = ((size_t)k * ny + j) * nx + i;
                const int mine = occ[v] != 0;
                const int32_t *other = mine ? free_xyz : occ_xyz;
                const size_t n_other = mine ? n_free : n_occ;
                int64_t best = OR_BIG;
                for (size_t q = 0; q < n_other; ++q) {
                    const int64_t di = other[3 * q] - i, dj = other[3 * q + 1] - j, dk = other[3 * q + 2] - k;
                    const int64_t d = di * di + dj * dj + dk * dk;
                    if (d < best)
                        best = d;
                }
                const int32_t mag = best == OR_BIG ? OR_INF32 : (int32_t)best;
                S[v] = mine ? -mag : mag;
            }
    free(occ_xyz);
    free(free_xyz);
}

/* ------------------------------------------------------------------------ */
/* Signed squared EDT, separable (Meijster et al. 2000)                      */
/* ------------------------------------------------------------------------ */

/* Phase 1 on one line: g[x] = distance to the nearest site on the line
 * (OR_BIG if the line has none).  Two scans, as in the paper's first phase. */
static void or_phase1(int m, const uint8_t *site, int64_t *g)
{
    int64_t last = -1;
    for (int x = 0; x < m; ++x) {
        if (site[x])
            last = x;
        g[x] = last < 0 ? OR_BIG : x - last;
    }
    last = -1;
    for (int x = m - 1; x >= 0; --x) {
        if (site[x])
            last = x;
        if (last >= 0 && last - x < g[x])
            g[x] = last - x;
    }
}

/* Phases 2 and 3 on one line: out[x] = min_i (x-i)^2 + G[i] over the indices i
 * with G[i] < OR_BIG, by Meijster's forward scan (stack of sites s[] with the
 * first abscissa t[] of each site's region, separator Sep) followed by the
 * backward scan.  out[x] = OR_BIG when the line has no site. */
static int64_t or_f(int64_t x, int64_t i, const int64_t *G) { return (x - i) * (x - i) + G[i]; }

static int64_t or_sep(int64_t i, int64_t u, const int64_t *G)
{
    /* Floor of the abscissa where the parabolas of i < u intersect.  The
     * caller only asks when the numerator is non-negative. */
    const int64_t num = u * u - i * i + G[u] - G[i];
    const int64_t den = 2 * (u - i);
    return num >= 0 ? num / den : -((-num + den - 1) / den);
}

static void or_envelope(int m, const int64_t *G, int64_t *out, int64_t *s, int64_t *t)
{
    int q = -1;
    for (int u = 0; u < m; ++u) {
        if (G[u] >= OR_BIG)
            continue;
        while (q >= 0 && or_f(t[q], s[q], G) > or_f(t[q], u, G))
            --q;
        if (q < 0) {
            q = 0;
            s[0] = u;
            t[0] = 0;
        } else {
            const int64_t w = 1 + or_sep(s[q], u, G);
            if (w < m) {
                ++q;
                s[q] = u;
                t[q] = w;
            }
        }
    }
    if (q < 0) {
        for (int x = 0; x < m; ++x)
            out[x] = OR_BIG;
        return;
    }
    for (int x = m - 1; x >= 0; --x) {
        out[x] = or_f(x, s[q], G);
        if (x == t[q])
            --q;
    }
}

/* Unsigned squared EDT to the site set (site[v] != 0), OR_BIG where no site. */
static void or_edt_sites(int nx, int ny, int nz, const uint8_t *site, int64_t *D)
{
    const int mmax = nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz);
    int64_t *G = (int64_t *)malloc(mmax * sizeof(int64_t));
    int64_t *o = (int64_t *)malloc(mmax * sizeof(int64_t));
    int64_t *s = (int64_t *)malloc(mmax * sizeof(int64_t));
    int64_t *t = (int64_t *)malloc(mmax * sizeof(int64_t));
    uint8_t *line = (uint8_t *)malloc(mmax);
    /* phase 1: rows along x, squared */
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) {
            const size_t base = ((size_t)k * ny + j) * nx;
            for (int i = 0; i < nx; ++i)
                line[i] = site[base + i] != 0;
            or_phase1(nx, line, o);
            for (int i = 0; i < nx; ++i)
                D[base + i] = o[i] >= OR_BIG ? OR_BIG : o[i] * o[i];
        }
    /* phase 2: columns along y */
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i) {
            for (int j = 0; j < ny; ++j)
                G[j] = D[((size_t)k * ny + j) * nx + i];
            or_envelope(ny, G, o, s, t);
            for (int j = 0; j < ny; ++j)
                D[((size_t)k * ny + j) * nx + i] = o[j];
        }
    /* phase 3: pillars along z */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            for (int k = 0; k < nz; ++k)
                G[k] = D[((size_t)k * ny + j) * nx + i];
            or_envelope(nz, G, o, s, t);
            for (int k = 0; k < nz; ++k)
                D[((size_t)k * ny + j) * nx + i] = o[k];
        }
    free(G);
    free(o);
    free(s);
    free(t);
    free(line);
}

/* Signed squared EDT: the unsigned transform to the occupied set read at free
 * voxels, minus the transform to the free set read at occupied voxels. */
void or_edt_separable(int nx, int ny, int nz, const uint8_t *occ, int32_t *S)
{
    const size_t V = (size_t)nx * ny * nz;
    uint8_t *fr = (uint8_t *)malloc(V);
    int64_t *DO = (int64_t *)malloc(V * sizeof(int64_t));
    int64_t *DF = (int64_t *)malloc(V * sizeof(int64_t));
    for (size_t v = 0; v < V; ++v)
        fr[v] = occ[v] == 0;
    or_edt_sites(nx, ny, nz, occ, DO);
    or_edt_sites(nx, ny, nz, fr, DF);
    for (size_t v = 0; v < V; ++v) {
        if (occ[v])
            S[v] = DF[v] >= OR_BIG ? -OR_INF32 : -(int32_t)DF[v];
        else
            S[v] = DO[v] >= OR_BIG ? OR_INF32 : (int32_t)DO[v];
    }
    free(fr);
    free(DO);
    free(DF);
}

/* ------------------------------------------------------------------------ */
/* Composite, float field                                                    */
/* ------------------------------------------------------------------------ */

/* comp = min(static, dynamic), per voxel (Sec. 6: the composition is a
 * parallel min between the environment field and the obstacle field). */
void or_composite(size_t n, const int32_t *S_static, const int32_t *S_dyn, int32_t *out)
{
    for (size_t v = 0; v < n; ++v)
        out[v] = S_static[v] < S_dyn[v] ? S_static[v] : S_dyn[v];
}

/* sdf = sign(S) * sqrtf((float)|S|) * vox in fp32; +/-INT32_MAX -> +/-inf. */
void or_sdf_from_sq(size_t n, const int32_t *S, float vox, float *sdf)
{
    for (size_t v = 0; v < n; ++v) {
        const int32_t s = S[v];
        if (s == OR_INF32) {
            sdf[v] = INFINITY;
        } else if (s == -OR_INF32) {
            sdf[v] = -INFINITY;
        } else {
            const float a = (float)(s < 0 ? -s : s);
            const float m = sqrtf(a) * vox;
            sdf[v] = s < 0 ? -m : m;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Trilinear sampling, hinge cost and its gradient                           */
/* ------------------------------------------------------------------------ */

/* Sample field (one time slice, [nz][ny][nx] fp32) at world point p.
 * Per axis the continuous index u = (p - origin)/vox - 1/2 is formed in fp32
 * (this decides the cell, so it is taken in the kernel's precision), clamped
 * to [0, n-1] (NaN -> 0), the lower corner is i0 = min(floor(u), n-2) (0 when
 * n == 1) and f = u - i0.  The lerps along x, then y, then z are done in
 * double.  Any -inf corner gives -inf, else any +inf corner gives +inf.
 * Returns d; *oob = 1 if any axis was clamped; grad (may be NULL) receives the
 * analytic derivative of d with respect to p (zero along clamped or
 * single-voxel axes; zero if d is not finite). */
double or_trilinear(const float *field, int nx, int ny, int nz, const float *origin, float vox,
                    const float *p, int *oob, double *grad)
{
    const int n[3] = {nx, ny, nz};
    int i0[3], i1[3], live[3];
    double f[3];
    *oob = 0;
    for (int a = 0; a < 3; ++a) {
        const float d0 = p[a] - origin[a];
        const float q = d0 / vox;
        float u = q - 0.5f;
        const float hi = (float)(n[a] - 1);
        const int inside = (u >= 0.0f) && (u <= hi);
        if (!inside)
            *oob = 1;
        u = fminf(fmaxf(u, 0.0f), hi);
        int lo = (int)floorf(u);
        const int lo_max = n[a] >= 2 ? n[a] - 2 : 0;
        if (lo > lo_max)
            lo = lo_max;
        i0[a] = lo;
        i1[a] = lo + 1 < n[a] ? lo + 1 : n[a] - 1;
        f[a] = (double)(u - (float)lo);
        live[a] = inside && n[a] >= 2;
    }
    double c[2][2][2];
    int has_pinf = 0, has_ninf = 0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int ii = dx ? i1[0] : i0[0], jj = dy ? i1[1] : i0[1], kk = dz ? i1[2] : i0[2];
                const float v = field[((size_t)kk * ny + jj) * nx + ii];
                if (isinf(v)) {
                    if (v < 0)
                        has_ninf = 1;
                    else
                        has_pinf = 1;
                }
                c[dz][dy][dx] = (double)v;
            }
    if (grad)
        grad[0] = grad[1] = grad[2] = 0.0;
    if (has_ninf)
        return -INFINITY;
    if (has_pinf)
        return INFINITY;
    /* lerp along x */
    double cx[2][2];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            cx[dz][dy] = c[dz][dy][0] + f[0] * (c[dz][dy][1] - c[dz][dy][0]);
    /* along y */
    double cy[2];
    for (int dz = 0; dz < 2; ++dz)
        cy[dz] = cx[dz][0] + f[1] * (cx[dz][1] - cx[dz][0]);
    /* along z */
    const double d = cy[0] + f[2] * (cy[1] - cy[0]);
    if (grad) {
        /* d/du_x: difference along x, lerped in y and z; likewise for y, z. */
        double ex[2][2], gx[2], gy[2];
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                ex[dz][dy] = c[dz][dy][1] - c[dz][dy][0];
        for (int dz = 0; dz < 2; ++dz) {
            gx[dz] = ex[dz][0] + f[1] * (ex[dz][1] - ex[dz][0]);
            gy[dz] = cx[dz][1] - cx[dz][0];
        }
        const double du[3] = {gx[0] + f[2] * (gx[1] - gx[0]), gy[0] + f[2] * (gy[1] - gy[0]), cy[1] - cy[0]};
        for (int a = 0; a < 3; ++a)
            grad[a] = live[a] ? du[a] / (double)vox : 0.0;
    }
    return d;
}

/* Hinge obstacle cost over N spheres (x, y, z, r) against the fields
 * sdf[T][nz][ny][nx]:  t = clamp(tidx, 0, T-1)  (obstacle factor i uses field
 * min(i, n), Sec. 8),  d = trilinear(sdf_t, centre),  h = max(0, eps + r - d).
 * Returns the number of spheres whose centre was clamped on some axis.
 * grad_c (may be NULL) receives dh/dc = -grad d where h > 0 and d is finite,
 * else 0; grad_r (may be NULL) receives dh/dr = [h > 0 and d finite]. */
int64_t or_hinge_cost(const float *sdf, int T, int nx, int ny, int nz, const float *origin, float vox,
                      const float *spheres, const int32_t *tidx, int64_t N, float eps, double *h,
                      double *grad_c, double *grad_r)
{
    int64_t n_oob = 0;
    const size_t V = (size_t)nx * ny * nz;
    for (int64_t q = 0; q < N; ++q) {
        int t = tidx[q];
        if (t < 0)
            t = 0;
        if (t > T - 1)
            t = T - 1;
        int oob = 0;
        double g[3];
        const double d = or_trilinear(sdf + (size_t)t * V, nx, ny, nz, origin, vox, spheres + 4 * q, &oob, g);
        n_oob += oob;
        const double r = spheres[4 * q + 3];
        double hv = (double)eps + r - d;
        if (!(hv > 0.0))
            hv = 0.0;
        h[q] = hv;
        const int active = hv > 0.0 && isfinite(d);
        if (grad_c)
            for (int a = 0; a < 3; ++a)
                grad_c[3 * q + a] = active ? -g[a] : 0.0;
        if (grad_r)
            grad_r[q] = active ? 1.0 : 0.0;
    }
    return n_oob;
}

/* Sec. 8 voxel filter: out(v) = occ(v) and (number of occupied in-grid voxels
 * among the 26 neighbours of v) >= min_neighbours. */
void or_voxel_filter(int nx, int ny, int nz, const uint8_t *occ, int min_neighbours, uint8_t *out)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t v = ((size_t)k * ny + j) * nx + i;
                int n = 0;
                for (int dk = -1; dk <= 1; ++dk)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            const int a = i + di, b = j + dj, c = k + dk;
                            if ((di || dj || dk) && a >= 0 && a < nx && b >= 0 && b < ny && c >= 0 && c < nz &&
                                occ[((size_t)c * ny + b) * nx + a])
                                ++n;
                        }
                out[v] = (uint8_t)(occ[v] && n >= min_neighbours);
            }
}

/* Sec. 8 collapsed map: out[j][i] = 1 iff occ[k][j][i] for some k in [z0, z1). */
void or_collapse(int nx, int ny, int nz, const uint8_t *occ, int z0, int z1, uint8_t *out)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            uint8_t o = 0;
            for (int k = z0 < 0 ? 0 : z0; k < z1 && k < nz; ++k)
                o |= occ[((size_t)k * ny + j) * nx + i] != 0;
            out[(size_t)j * nx + i] = o;
        }
}

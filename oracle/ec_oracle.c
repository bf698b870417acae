/*
 * ec_oracle.c -- plain CPU oracle for Euler-characteristic, perimeter, area and
 * volume curves of 2D/3D fields under sublevel filtration.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests, the smoke check and the CPU-baseline leg of the bench
 * do.  It shares no code, table or constant with the CUDA path.
 *
 * What it computes is the plain definition, written out:
 *   - Sublevel filtration (Eq. sublevel_set): a top cell (pixel / voxel) with
 *     value x is active at level k iff x <= t_k, compared in the field's own
 *     type (float32 or unsigned integer).  A NaN is never active.
 *   - Including a top cell includes all its faces, edges and vertices
 *     (Sec. 2, text after Eq. sublevel_set): the complex K_k at level k is the
 *     closure of the active top cells.  A lower-dimensional cell therefore
 *     belongs to K_k exactly when at least one of its incident top cells is
 *     active, i.e. from the level  entry = min(bin of incident top cells).
 *   - EC (Eq. EC_formula): chi_k = #V - #E + #F (- #C in 3D) of K_k.  With
 *     count[dim][entry] the number of dim-cells entering at each level, the
 *     curve is the running sum of the alternating counts.
 *   - Perimeter (2D, Table 1) / area (3D, Table 2): the number of (d-1)-cells
 *     with exactly one active incident top cell; a top cell outside the domain
 *     is never active.  Such a cell is on the boundary from the smaller to the
 *     larger of its two incident bins.
 *   - Area (2D) / volume (3D): the number of active top cells.
 *   - 3D "Perimeter" column of Table 2: crease length.  Every edge carries a
 *     weight fixed by which of its 4 incident voxels are active: one -> 1,
 *     two sharing a face -> 0, two diagonal -> 2, three -> 1, zero or four -> 0.
 *     (The paper prints only the per-vertex values; this is the reading that
 *     reproduces every row of Table 2.)  Per edge the weight changes only when
 *     one of its incident voxels enters, so the oracle walks the 4 incident bins
 *     in increasing order and records each change at the level it happens.
 *   - 2D EC under 4-connectivity (Table 1, "4-C" columns): identical to the
 *     8-connected complex except that a vertex whose two active pixels touch
 *     only diagonally (type QD) counts as two vertices.  So
 *     chi4_k = chi8_k + #(vertices of type QD at level k).
 *   - 3D EC under 6-connectivity (the paper fixes 26-connectivity in 3D and
 *     gives the other connectivity only for 2D, Table 1's 4-C columns; this is
 *     the reading taken): under face adjacency, cells join the active set
 *     through shared cells only when every voxel around the shared cell is
 *     active.  So the complex at level k has a cell exactly when ALL of its
 *     incident top cells are active (exit = max(bin of incident top cells),
 *     top cells outside the domain never active), and by the duality between
 *     this complex and the voxel adjacency structure (voxels, face-adjacent
 *     pairs, 2x2 squares, 2x2x2 cubes)
 *         chi6_k = #C - #F + #E - #V   over the cells with exit <= k,
 *     i.e. #voxels - #face pairs + #squares - #cubes.  The same reading in 2D,
 *     chi = #F - #E + #V over cells with exit <= k, is the 4-connected EC of
 *     Table 1 (oracle_ec_dual_2d, used to check this reading).
 *
 * Levels: thresholds t_0 <= ... <= t_{L-1}; bin(x) = min{k : x <= t_k}, or L
 * when x exceeds every threshold (or is NaN).  Bin L is "never active".
 * Curves are int64 arrays of length L; index k is the value at threshold t_k.
 *
 * Parallelism: OpenMP over the outermost axis into private count arrays that
 * are summed afterwards; the arithmetic is the same as the serial loop.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ binning */

/* Smallest k with x <= t[k] (float32 comparison), L if none.  NaN -> L. */
static int32_t lower_bound_f32(float x, const float *t, int32_t L)
{
    int32_t lo = 0, hi = L;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (x <= t[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static int32_t lower_bound_u32(uint32_t x, const uint32_t *t, int32_t L)
{
    int32_t lo = 0, hi = L;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (x <= t[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* dtype: 0 = uint8, 1 = uint16, 2 = float32 (same codes as the public API).
 * thresholds: L values of the field's type; NULL means identity levels
 * t_k = k (integer types only). */
int oracle_bin(const void *field, int64_t n, int dtype, const void *thresholds,
               int32_t L, int32_t *bins)
{
    if (L < 1) return -1;
    if (dtype == 2) {
        const float *x = (const float *)field;
        const float *t = (const float *)thresholds;
        if (!t) return -1;
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) bins[i] = lower_bound_f32(x[i], t, L);
        return 0;
    }
    if (dtype != 0 && dtype != 1) return -1;
    uint32_t *t32 = NULL;
    if (thresholds) {
        t32 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)L);
        if (!t32) return -2;
        for (int32_t k = 0; k < L; k++)
            t32[k] = dtype == 0 ? ((const uint8_t *)thresholds)[k]
                                : ((const uint16_t *)thresholds)[k];
    }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        uint32_t v = dtype == 0 ? ((const uint8_t *)field)[i] : ((const uint16_t *)field)[i];
        int32_t b;
        if (t32) b = lower_bound_u32(v, t32, L);
        else b = (v < (uint32_t)L) ? (int32_t)v : L; /* identity: x <= k iff k >= x */
        bins[i] = b;
    }
    free(t32);
    return 0;
}

/* ------------------------------------------------------- shared helpers */

/* Incident top-cell indices along one axis for a doubled coordinate C in
 * [0, 2N]: odd C = 2i+1 is the span of top cell i; even C = 2i is the plane
 * between top cells i-1 and i.  Returns how many of the two slots exist and
 * writes them; slot 0 is the lower one.  A slot outside [0, N) is reported
 * as -1 (outside the domain: never active). */
static inline int axis_slots(int64_t C, int64_t N, int64_t s[2])
{
    if (C & 1) { s[0] = (C - 1) / 2; s[1] = -1; return 1; }
    int64_t i = C / 2;
    s[0] = (i - 1 >= 0) ? i - 1 : -1;
    s[1] = (i < N) ? i : -1;
    return 2;
}

static int32_t imin(int32_t a, int32_t b) { return a < b ? a : b; }
static int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }

/* Sort 4 (bin, slot) pairs by bin, insertion sort (ties keep slot order; any
 * order of equal bins gives the same running sums). */
static void sort4(int32_t b[4], int s[4])
{
    for (int i = 1; i < 4; i++) {
        int32_t kb = b[i]; int ks = s[i]; int j = i - 1;
        while (j >= 0 && b[j] > kb) { b[j + 1] = b[j]; s[j + 1] = s[j]; j--; }
        b[j + 1] = kb; s[j + 1] = ks;
    }
}

/* Crease weight of an edge from the set of its active incident voxels.
 * Slots are numbered a + 2b over the two axes perpendicular to the edge, so
 * two slots are diagonal iff they differ in both bits (XOR == 3). */
static int crease_weight(unsigned mask)
{
    int m = __builtin_popcount(mask);
    if (m == 1 || m == 3) return 1;
    if (m == 2) return (mask == 0x9u || mask == 0x6u) ? 2 : 0;
    return 0;
}

/* ------------------------------------------------------------------- 2D */

/* bins: h*w row-major (index y*w + x).  Any output pointer may be NULL. */
int oracle_curves_2d(const int32_t *bins, int64_t h, int64_t w, int32_t L,
                     int64_t *ec8, int64_t *ec4, int64_t *perim, int64_t *area)
{
    if (h < 1 || w < 1 || L < 1) return -1;
    const int64_t W2 = 2 * w, H2 = 2 * h, NB = (int64_t)L + 1;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    /* per thread: cnt[3][NB], per_d[NB], area_d[NB], qd_d[NB] */
    const int64_t per_thread = 6 * NB;
    int64_t *acc = (int64_t *)calloc((size_t)(per_thread * nthr), sizeof(int64_t));
    if (!acc) return -2;

    #pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int64_t *cnt = acc + tid * per_thread;       /* cnt[dim*NB + level] */
        int64_t *per_d = cnt + 3 * NB, *area_d = cnt + 4 * NB, *qd_d = cnt + 5 * NB;
        #pragma omp for schedule(dynamic, 4)
        for (int64_t Y = 0; Y <= H2; Y++) {
            int64_t sy[2]; int ny = axis_slots(Y, h, sy);
            for (int64_t X = 0; X <= W2; X++) {
                int64_t sx[2]; int nx = axis_slots(X, w, sx);
                /* gather incident pixel bins, outside the domain = L */
                int32_t b[4]; int slot[4]; int n = 0;
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        int32_t v = L;
                        if (sy[j] >= 0 && sx[i] >= 0) v = bins[sy[j] * w + sx[i]];
                        b[n] = v; slot[n] = i + 2 * j; n++;
                    }
                int dim = (int)(X & 1) + (int)(Y & 1);
                int32_t entry = b[0];
                for (int q = 1; q < n; q++) entry = imin(entry, b[q]);
                cnt[dim * NB + entry] += 1;
                if (dim == 2) {              /* pixel: area */
                    area_d[entry] += 1;
                } else if (dim == 1) {       /* edge: boundary while exactly one side active */
                    per_d[imin(b[0], b[1])] += 1;
                    per_d[imax(b[0], b[1])] -= 1;
                } else {                     /* vertex: QD interval for 4-connectivity */
                    sort4(b, slot);
                    if (b[1] < b[2] && (slot[0] ^ slot[1]) == 3) {
                        qd_d[b[1]] += 1;
                        qd_d[b[2]] -= 1;
                    }
                }
            }
        }
    }
    /* sum thread arrays and form running sums over levels 0..L-1 */
    int64_t c0 = 0, c1 = 0, c2 = 0, pr = 0, ar = 0, qd = 0;
    for (int64_t k = 0; k < L; k++) {
        int64_t v0 = 0, v1 = 0, v2 = 0, vp = 0, va = 0, vq = 0;
        for (int t = 0; t < nthr; t++) {
            const int64_t *cnt = acc + t * per_thread;
            v0 += cnt[0 * NB + k]; v1 += cnt[1 * NB + k]; v2 += cnt[2 * NB + k];
            vp += cnt[3 * NB + k]; va += cnt[4 * NB + k]; vq += cnt[5 * NB + k];
        }
        c0 += v0; c1 += v1; c2 += v2; pr += vp; ar += va; qd += vq;
        int64_t chi8 = c0 - c1 + c2;
        if (ec8) ec8[k] = chi8;
        if (ec4) ec4[k] = chi8 + qd;
        if (perim) perim[k] = pr;
        if (area) area[k] = ar;
    }
    free(acc);
    return 0;
}

/* ------------------------------------------------------------------- 3D */

/* bins: d*h*w, index (z*h + y)*w + x.  Any output pointer may be NULL.
 * Only cells whose doubled z coordinate Z lies in [zlo, zhi] are counted;
 * the full curves use [0, 2d].  The counts of Eq. EC_formula (and of every
 * boundary measure) are sums over cells, so curves of disjoint Z ranges add
 * up to the curves of their union. */
int oracle_curves_3d_zrange(const int32_t *bins, int64_t d, int64_t h, int64_t w, int32_t L,
                            int64_t zlo, int64_t zhi,
                            int64_t *ec, int64_t *perim, int64_t *area, int64_t *vol)
{
    if (d < 1 || h < 1 || w < 1 || L < 1) return -1;
    if (zlo < 0) zlo = 0;
    if (zhi > 2 * d) zhi = 2 * d;
    const int64_t W2 = 2 * w, H2 = 2 * h, D2 = 2 * d, NB = (int64_t)L + 1;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    /* per thread: cnt[4][NB], per_d, area_d, vol_d */
    const int64_t per_thread = 7 * NB;
    int64_t *acc = (int64_t *)calloc((size_t)(per_thread * nthr), sizeof(int64_t));
    if (!acc) return -2;

    #pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int64_t *cnt = acc + tid * per_thread;
        int64_t *per_d = cnt + 4 * NB, *area_d = cnt + 5 * NB, *vol_d = cnt + 6 * NB;
        #pragma omp for schedule(dynamic, 1)
        for (int64_t Z = zlo; Z <= zhi; Z++) {
            int64_t sz[2]; int nz = axis_slots(Z, d, sz);
            for (int64_t Y = 0; Y <= H2; Y++) {
                int64_t sy[2]; int ny = axis_slots(Y, h, sy);
                for (int64_t X = 0; X <= W2; X++) {
                    int64_t sx[2]; int nx = axis_slots(X, w, sx);
                    int32_t b[8]; int n = 0;
                    for (int k = 0; k < nz; k++)
                        for (int j = 0; j < ny; j++)
                            for (int i = 0; i < nx; i++) {
                                int32_t v = L;
                                if (sz[k] >= 0 && sy[j] >= 0 && sx[i] >= 0)
                                    v = bins[(sz[k] * h + sy[j]) * w + sx[i]];
                                b[n++] = v;
                            }
                    int dim = (int)(X & 1) + (int)(Y & 1) + (int)(Z & 1);
                    int32_t entry = b[0];
                    for (int q = 1; q < n; q++) entry = imin(entry, b[q]);
                    cnt[dim * NB + entry] += 1;
                    if (dim == 3) {
                        vol_d[entry] += 1;
                    } else if (dim == 2) {
                        /* face: two incident voxels along its normal axis */
                        area_d[imin(b[0], b[1])] += 1;
                        area_d[imax(b[0], b[1])] -= 1;
                    } else if (dim == 1) {
                        /* edge: the loops above listed its 4 incident voxels with
                         * the two perpendicular axes in (lower, higher) order, so
                         * list position p = a + 2b with a, b the slot bits. */
                        int slot[4] = {0, 1, 2, 3};
                        sort4(b, slot);
                        unsigned mask = 0; int prev = 0;
                        for (int q = 0; q < 4; q++) {
                            mask |= 1u << slot[q];
                            int wgt = crease_weight(mask);
                            per_d[b[q]] += wgt - prev;
                            prev = wgt;
                        }
                    }
                }
            }
        }
    }
    int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, pr = 0, ar = 0, vo = 0;
    for (int64_t k = 0; k < L; k++) {
        int64_t v[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int t = 0; t < nthr; t++) {
            const int64_t *cnt = acc + t * per_thread;
            for (int q = 0; q < 7; q++) v[q] += cnt[q * NB + k];
        }
        c0 += v[0]; c1 += v[1]; c2 += v[2]; c3 += v[3];
        pr += v[4]; ar += v[5]; vo += v[6];
        if (ec) ec[k] = c0 - c1 + c2 - c3;
        if (perim) perim[k] = pr;
        if (area) area[k] = ar;
        if (vol) vol[k] = vo;
    }
    free(acc);
    return 0;
}

int oracle_curves_3d(const int32_t *bins, int64_t d, int64_t h, int64_t w, int32_t L,
                     int64_t *ec, int64_t *perim, int64_t *area, int64_t *vol)
{
    return oracle_curves_3d_zrange(bins, d, h, w, L, 0, 2 * d, ec, perim, area, vol);
}

/* ------------------------------------------------ 6-connected EC (3D) and
 * its 2D counterpart: a cell is in the complex when all incident top cells
 * are active, from the level exit = max(bin of incident top cells); the
 * curve is the running sum of the counts with sign (-1)^(n - dim). */
static int ec_dual(const int32_t *bins, int64_t d, int64_t h, int64_t w, int32_t L, int ndim, int64_t *out)
{
    if (d < 1 || h < 1 || w < 1 || L < 1) return -1;
    const int64_t D2 = ndim == 3 ? 2 * d : 0, H2 = 2 * h, W2 = 2 * w, NB = (int64_t)L + 1;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    int64_t *acc = (int64_t *)calloc((size_t)(NB * nthr), sizeof(int64_t));
    if (!acc) return -2;
    #pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int64_t *sgn = acc + tid * NB;   /* signed cell count per exit level */
        #pragma omp for schedule(dynamic, 1)
        for (int64_t Z = 0; Z <= D2; Z++) {
            int64_t sz[2] = {0, -1}; int nz = 1;
            if (ndim == 3) nz = axis_slots(Z, d, sz);
            for (int64_t Y = 0; Y <= H2; Y++) {
                int64_t sy[2]; int ny = axis_slots(Y, h, sy);
                for (int64_t X = 0; X <= W2; X++) {
                    int64_t sx[2]; int nx = axis_slots(X, w, sx);
                    int32_t ex = -1;
                    for (int k = 0; k < nz; k++)
                        for (int j = 0; j < ny; j++)
                            for (int i = 0; i < nx; i++) {
                                int32_t v = L;
                                if (sz[k] >= 0 && sy[j] >= 0 && sx[i] >= 0)
                                    v = bins[(sz[k] * h + sy[j]) * w + sx[i]];
                                ex = imax(ex, v);
                            }
                    const int dim = (int)(X & 1) + (int)(Y & 1) + (ndim == 3 ? (int)(Z & 1) : 0);
                    sgn[ex] += ((ndim - dim) & 1) ? -1 : 1;
                }
            }
        }
    }
    int64_t run = 0;
    for (int64_t k = 0; k < L; k++) {
        for (int t = 0; t < nthr; t++) run += acc[t * NB + k];
        out[k] = run;
    }
    free(acc);
    return 0;
}

int oracle_ec6_3d(const int32_t *bins, int64_t d, int64_t h, int64_t w, int32_t L, int64_t *ec6)
{
    return ec_dual(bins, d, h, w, L, 3, ec6);
}

int oracle_ec_dual_2d(const int32_t *bins, int64_t h, int64_t w, int32_t L, int64_t *ec)
{
    return ec_dual(bins, 1, h, w, L, 2, ec);
}

/* ------------------------------------------- hash-box field (workload input)
 *
 * Counter-based generator for the low-memory streaming workload, implemented
 * here on its own from the published MurmurHash3 32-bit finaliser (Austin
 * Appleby, MurmurHash3, public domain: u ^= u >> 16; u *= 0x85EBCA6B;
 * u ^= u >> 13; u *= 0xC2B2AE35; u ^= u >> 16), called m below.
 *
 * a        = m(lo32(seed) ^ m(hi32(seed)))
 * u(p,y,z) = m(m(m(a ^ z) ^ y) ^ p)                     (p, y, z mod 2^32)
 * h(x,y,z) = low 16 bits of u(floor(x/2), y, z) for even x, high 16 bits
 *            for odd x
 * v(x,y,z) = floor( sum_{|dx|,|dy|,|dz| <= 2} h(x+dx, y+dy, z+dz) * 4096
 *                   / (125 * 65536) )                       in [0, 4095]
 * defined for all integer coordinates (no border case).
 */
static uint32_t murmur_fmix32(uint32_t u)
{
    u ^= u >> 16;
    u *= 0x85EBCA6Bu;
    u ^= u >> 13;
    u *= 0xC2B2AE35u;
    u ^= u >> 16;
    return u;
}

static uint32_t hash16(uint64_t seed, int64_t x, int64_t y, int64_t z)
{
    const uint32_t a = murmur_fmix32((uint32_t)seed ^ murmur_fmix32((uint32_t)(seed >> 32)));
    const uint32_t hz = murmur_fmix32(a ^ (uint32_t)z);
    const uint32_t hy = murmur_fmix32(hz ^ (uint32_t)y);
    const int64_t p = (x - (x & 1)) / 2;   /* floor(x / 2) */
    const uint32_t u = murmur_fmix32(hy ^ (uint32_t)p);
    return (x & 1) ? (u >> 16) : (u & 0xFFFFu);
}

int oracle_hashbox_u16(uint64_t seed, int64_t x0, int64_t y0, int64_t z0,
                       int64_t nx, int64_t ny, int64_t nz, uint16_t *out)
{
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    /* the hash of every point of the box grown by 2 on each side, then the
     * 125-term sum of the definition for every output point */
    const int64_t px = nx + 4, py = ny + 4, pz = nz + 4;
    uint16_t *hh = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)(px * py * pz));
    if (!hh) return -2;
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < pz; k++)
        for (int64_t j = 0; j < py; j++)
            for (int64_t i = 0; i < px; i++)
                hh[(k * py + j) * px + i] = (uint16_t)hash16(seed, x0 - 2 + i, y0 - 2 + j, z0 - 2 + k);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nz; k++)
        for (int64_t j = 0; j < ny; j++)
            for (int64_t i = 0; i < nx; i++) {
                uint64_t s = 0;
                for (int dz = 0; dz < 5; dz++)
                    for (int dy = 0; dy < 5; dy++)
                        for (int dx = 0; dx < 5; dx++)
                            s += hh[((k + dz) * py + (j + dy)) * px + (i + dx)];
                out[(k * ny + j) * nx + i] = (uint16_t)((s * 4096ull) / (125ull * 65536ull));
            }
    free(hh);
    return 0;
}

/* Threads later calls use (timing the oracle on one core or on all of them;
 * n < 1 restores the OpenMP default).  Results do not depend on it. */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    static int dflt = 0;
    if (!dflt) dflt = omp_get_max_threads();
    omp_set_num_threads(n >= 1 ? n : dflt);
#else
    (void)n;
#endif
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

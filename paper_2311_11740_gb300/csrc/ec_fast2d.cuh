// ec_fast2d.cuh -- device building blocks of the fast per-pixel 2D path,
// shared by the single-field kernel (ec_fast2d.cu) and the batched kernel
// (ec_batch.cu).  See ec_fast2d.cu for the data flow.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ec_fast3d.cuh"

namespace ec {

namespace fast2d {

using fast3d::FBin;
using fast3d::fbin;
using fast3d::fbin_uniform;
using fast3d::IBin;

constexpr int kThreads = 256;
constexpr int SW = 1024;               // pixels per strip
constexpr int RWORDS = (SW + 4) / 2;   // key words per row: x0-2 .. x0+SW+1
constexpr int NR = 4;                  // ring rows
constexpr int kThrSmem = 4096;
constexpr int KA = 3;                  // raw rows copied ahead (asynchronous path)
constexpr int NRAW = KA + 2;           // raw row ring: row being binned, row waited for, KA in flight

// Raw row of the asynchronous path: the strip's pixels x0-A .. x0+SW+A-1
// with A elements (16 bytes) of halo on each side, so that every 16-byte
// chunk starts aligned.
template <typename T>
constexpr int raw_pad() { return 16 / (int)sizeof(T); }
template <typename T>
constexpr int raw_bytes() { return (SW + 2 * raw_pad<T>()) * (int)sizeof(T); }

// Banded strips (cover staging only): a field at most ~SW/nb - 2 pixels wide
// is walked as nb row bands of kBandRows rows side by side in one strip, each
// in its own SW/nb-pixel segment; the pixels between a band's right edge and
// the next segment are never active, so the bands do not touch, and each
// band's halo rows are its true neighbour rows.
constexpr int kBandRows = 64;
static_assert(SW == 1024, "banded segments are 256 or 512 pixels");
template <typename T>
constexpr int band_seg_bytes(int nb) { return (raw_bytes<T>() / nb) & ~15; }
// Widest field that nb bands fit (0 if none): a band's 16-byte cover must fit
// its segment and leave at least two never-active pixels before the next band.
template <typename T>
constexpr int band_max_width(int nb)
{
    return nb <= 1 ? 0
                   : ((band_seg_bytes<T>(nb) - 15) / (int)sizeof(T) < SW / nb - 2
                          ? (band_seg_bytes<T>(nb) - 15) / (int)sizeof(T)
                          : SW / nb - 2);
}

struct Params {
    const void *field;
    int64_t H, W;
    int nstrips, nrows_items, ry;
    int32_t L;
    const void *thr;
    long long *hist;
    int rows[kMaxDesc];
    int nd;
    int smem_hist;
    int conn4;
    const int *uni;
};

template <typename T>
struct Ctx2 {
    Params p;
    uint32_t *ring;
    unsigned char *raw;   // raw row ring (asynchronous path)
    int *sh_hist;
    FBin fb;
    IBin<T> ib;
    int x0, y0, y1;
    bool interior;
    int nb = 1;          // row bands side by side in the strip (banded walk when > 1)
    int since = 0;       // rows counted since the packed words were last exchanged (DM 7)
    int64_t yb0 = 0;     // first field row of band 0; band b, virtual row v -> row yb0 + b*kBandRows + v
};

template <typename T>
__device__ __forceinline__ uint32_t bin_value2(const Ctx2<T> &c, T v)
{
    if constexpr (sizeof(T) == 4) return c.fb.uniform ? fbin_uniform(v, c.fb) : fbin(v, c.fb);
    else return c.ib(v);
}

// Raw values of one row share of a thread (words tid, tid+256, tid+512 of
// the row: pixels x0-2+2w and x0-1+2w), loaded one row step ahead of their
// binning so that the global-load latency overlaps the counting of a row.
// The loads go through the read-only path (the field is never written by
// the kernel), which the row barrier does not have to wait for.
template <typename T>
struct RowRaw {
    T v[3][2];
    uint32_t ok;   // bit 2*it + j: value v[it][j] lies in the field
};

template <typename T>
__device__ __forceinline__ void load_row(const Ctx2<T> &c, int64_t y, RowRaw<T> &r)
{
    const T *f = (const T *)c.p.field;
    r.ok = 0;
    if (y < 0 || y >= c.p.H) return;
    const T *row = f + y * c.p.W;
#pragma unroll
    for (int it = 0; it < (RWORDS + kThreads - 1) / kThreads; it++) {
        const int w = threadIdx.x + it * kThreads;
        if (w < RWORDS) {
            const int64_t gx = (int64_t)c.x0 - 2 + 2 * w;
            if (c.interior || (gx >= 0 && gx < c.p.W)) { r.v[it][0] = __ldg(row + gx); r.ok |= 1u << (2 * it); }
            if (c.interior || (gx + 1 >= 0 && gx + 1 < c.p.W)) { r.v[it][1] = __ldg(row + gx + 1); r.ok |= 2u << (2 * it); }
        }
    }
}

// Bin a loaded row into ring slot (y mod NR); values outside the field bin to L.
template <typename T>
__device__ __forceinline__ void bin_row(Ctx2<T> &c, int64_t y, const RowRaw<T> &r)
{
    uint32_t *kr = c.ring + (uint32_t)((y + 8) % NR) * RWORDS;
    const uint32_t L = (uint32_t)c.p.L;
#pragma unroll
    for (int it = 0; it < (RWORDS + kThreads - 1) / kThreads; it++) {
        const int w = threadIdx.x + it * kThreads;
        if (w < RWORDS) {
            const uint32_t b0 = (r.ok >> (2 * it)) & 1u ? bin_value2(c, r.v[it][0]) : L;
            const uint32_t b1 = (r.ok >> (2 * it)) & 2u ? bin_value2(c, r.v[it][1]) : L;
            kr[w] = b0 | (b1 << 16);
        }
    }
}

template <int DM, int D>
constexpr int dm_row2() { return ((DM & 1) && D > 0) + ((DM & 2) && D > 1); }

// EC + perimeter + area with compile-time rows (DM 7) keep five words per
// level (an odd stride spreads a warp's levels over the banks): EC
// (atomics), a packed word (atomics: bits 0-16 add 4 - #edge neighbours
// preceding, bits 17-31 count pixels), the perimeter and area decoded from
// it (perimeter = 2 * sum - 4 * count, area = count), and a spare word.  The packed
// words are exchanged to zero at least every kExchangeRows rows of a block
// (plus at most one row of skew between its threads), so a word collects at
// most 14 * 1024 < 2^15 pixels and 4 * 2^15 <= 2^17 between exchanges.
template <int DM>
constexpr int hist_slots2(int nd) { return DM == 7 ? 5 : nd; }
constexpr int kExchangeRows = 12;

// Exchange this thread's share of the packed words (levels tid, tid + 256,
// ...) and add them into the perimeter and area words of their levels.
__device__ __forceinline__ void exchange_packed2(int *h, int L)
{
    for (int k = threadIdx.x; k <= L; k += kThreads) {
        const uint32_t w = atomicExch((unsigned int *)(h + 5 * k + 1), 0u);
        if (w) {
            const int n = (int)(w >> 17), sum = (int)(w & 0x1FFFFu);
            h[5 * k + 2] += 2 * sum - 4 * n;
            h[5 * k + 3] += n;
        }
    }
}

// After a group of rows: exchange the packed words when due.
template <int DM, typename T>
__device__ __forceinline__ void after_rows(Ctx2<T> &c, int rows)
{
    if constexpr (DM == 7) {
        c.since += rows;
        if (c.since >= kExchangeRows) {
            c.since = 0;
            exchange_packed2(c.sh_hist, c.p.L);
        }
    }
}

// Load row y+1 into window slot (R+1)%3 (R = position of row y) and count
// row y if it belongs to the item.  SKIP (strips whose counted columns reach
// past the field): pixels at the never-active level L are left out of the
// compile-time-descriptor histogram, as the generic path always does; their
// changes belong to the discarded level L, and past the field's edge they
// would all hit one word and serialise the warp's atomics.
template <typename T, bool CONN4, int R, int DM, bool SKIP = false>
__device__ __forceinline__ void count_row(Ctx2<T> &c, uint32_t (&win)[3][5], int y)
{
    {
        const uint32_t *kr = c.ring + (uint32_t)((y + 1 + 8) % NR) * RWORDS + 2 * threadIdx.x;
        const uint2 a = *(const uint2 *)kr, b = *(const uint2 *)(kr + 2);
        constexpr int W = (R + 1) % 3;
        win[W][0] = a.y;                        // keys x, x+1
        win[W][1] = b.x;                        // keys x+2, x+3
        win[W][2] = __byte_perm(a.x, a.y, 0x5432);   // x-1, x
        win[W][3] = __byte_perm(a.y, b.x, 0x5432);   // x+1, x+2
        win[W][4] = __byte_perm(b.x, b.y, 0x5432);   // x+3, x+4
    }
    if (y >= c.y0) {
        constexpr int SL[3] = {(R + 2) % 3, R, (R + 1) % 3};   // rows y-1, y, y+1
        uint32_t n0[9], n1[9];
#pragma unroll
        for (int dy = 0; dy < 3; dy++) {
            const uint32_t *w = win[SL[dy]];
            n0[3 * dy] = w[2]; n0[3 * dy + 1] = w[0]; n0[3 * dy + 2] = w[3];
            n1[3 * dy] = w[3]; n1[3 * dy + 1] = w[1]; n1[3 * dy + 2] = w[4];
        }
        const uint32_t c0 = win[R][0], c1 = win[R][1];
        const Quad2 q = quad_delta_2d<CONN4>(n0, c0, n1, c1);
        const uint32_t key[4] = {c0 & 0xFFFFu, c0 >> 16, c1 & 0xFFFFu, c1 >> 16};
        const int ecv[4] = {sbyte<0>(q.ec), sbyte<1>(q.ec), sbyte<2>(q.ec), sbyte<3>(q.ec)};
        const int pev[4] = {sbyte<0>(q.per), sbyte<1>(q.per), sbyte<2>(q.per), sbyte<3>(q.per)};
        const int L = c.p.L;
        if constexpr (DM != 0) {
            // interleaved rows [L+1][ND] (the never-active level L has its own,
            // discarded slot): one address per pixel, rows at immediate offsets
            constexpr int ND = hist_slots2<DM>((DM & 1) + ((DM >> 1) & 1) + ((DM >> 2) & 1));
            int *const h = c.sh_hist;
#pragma unroll
            for (int v = 0; v < 4; v++) {
                if (SKIP && key[v] >= (uint32_t)L) continue;
                int *const e = h + key[v] * ND;
                if constexpr (DM == 7) {
                    atomicAdd(e, ecv[v]);
                    // (perimeter change + 4) / 2 = 4 - #edge neighbours preceding, and one pixel
                    atomicAdd((unsigned int *)(e + 1), (uint32_t)((pev[v] + 4) >> 1) | (1u << 17));
                } else {
                    if (DM & 1) atomicAdd(e + dm_row2<DM, 0>(), ecv[v]);
                    if (DM & 2) atomicAdd(e + dm_row2<DM, 1>(), pev[v]);
                    if (DM & 4) atomicAdd(e + dm_row2<DM, 2>(), 1);
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const uint32_t k = key[v];
                if (k >= (uint32_t)L) continue;
                const int vals[3] = {ecv[v], pev[v], 1};
#pragma unroll
                for (int q2 = 0; q2 < 3; q2++) {
                    const int r = c.p.rows[q2];
                    if (r < 0 || vals[q2] == 0) continue;
                    if (c.sh_hist) atomicAdd(&c.sh_hist[r * L + k], vals[q2]);
                    else atomicAdd((unsigned long long *)&c.p.hist[(size_t)r * L + k],
                                   (unsigned long long)(long long)vals[q2]);
                }
            }
        }
    }
}

// One row step, y = y0 - 2 + t: bin row y+1 (loaded by the previous step),
// start the loads of row y+2, then (after the barrier) load row y+1 into
// window slot (R+1)%3 with R = t mod 3 and count row y if it belongs to the
// item.  Rows y0-1 .. y1 pass through the window.
template <typename T, bool CONN4, int R, int DM, bool SKIP = false>
__device__ __forceinline__ void ystep(Ctx2<T> &c, uint32_t (&win)[3][5], RowRaw<T> &raw, int t)
{
    const int y = c.y0 - 2 + t;
    bin_row<T>(c, y + 1, raw);
    if (y + 2 <= c.y1) load_row<T>(c, y + 2, raw);
    __syncthreads();
    count_row<T, CONN4, R, DM, SKIP>(c, win, y);
}

// ---- asynchronous path: rows copied to shared memory KA rows ahead with
// cp.async (16-byte chunks, zero-filled outside the field); used when every
// row starts 16-byte aligned.

using fast3d::cp_async16;
using fast3d::cp_async_commit;
using fast3d::cp_async_wait;

// Banded copies of virtual row y: band b's field row yb0 + b*kBandRows + y
// (its 16-byte cover) into segment b of the raw slot.
template <typename T>
__device__ __forceinline__ void copy_row_bands(const Ctx2<T> &c, int64_t y)
{
    constexpr int sz = (int)sizeof(T);
    const int seg = band_seg_bytes<T>(c.nb), cps = seg / 16;
    unsigned char *slot = c.raw + (uint32_t)((y + 16) % NRAW) * raw_bytes<T>();
    const unsigned char *fb = (const unsigned char *)c.p.field;
    const int64_t total = c.p.H * c.p.W * sz;
    for (int q = threadIdx.x; q < c.nb * cps; q += kThreads) {
        const int b = q / cps, ch = q - b * cps;
        const int64_t yo = c.yb0 + (int64_t)b * kBandRows + y;
        if (yo < 0 || yo >= c.p.H) continue;
        const int64_t rs = yo * c.p.W * sz, cs = (rs & ~(int64_t)15) + 16 * ch;
        if (cs >= rs + c.p.W * sz) continue;
        const int64_t left = total - cs;
        cp_async16(fast3d::smem_u32(slot + b * seg + ch * 16), fb + cs, left < 16 ? (uint32_t)left : 16u);
    }
}

// Levels of virtual pixels x, x+1 (x even; strip coordinates, x0 = 0) of
// banded virtual row y as one key word.  Segments are 2^sh pixels wide (256
// or 512), so both pixels lie in one segment.
template <typename T>
__device__ __forceinline__ uint32_t band_word(Ctx2<T> &c, const unsigned char *raw, int64_t y, int x, int sh)
{
    constexpr int sz = (int)sizeof(T);
    const uint32_t L = (uint32_t)c.p.L;
    if (x < 0 || x >= SW) return L | (L << 16);
    const int b = x >> sh, xl = x & ((1 << sh) - 1);
    const int64_t yo = c.yb0 + (int64_t)b * kBandRows + y;
    if (xl >= c.p.W || yo < 0 || yo >= c.p.H) return L | (L << 16);
    const unsigned char *r = raw + b * band_seg_bytes<T>(c.nb) + (int)((yo * c.p.W * sz) & 15) + xl * sz;
    const uint32_t b0 = bin_value2(c, *(const T *)r);
    const uint32_t b1 = xl + 1 < c.p.W ? bin_value2(c, *(const T *)(r + sz)) : L;
    return b0 | (b1 << 16);
}

// Start this thread's copies of row y (empty if y is beyond the item) and
// close them as one group.  STG_ALIGNED: the row width and start are
// multiples of 16 bytes, so a chunk lies wholly inside or wholly outside the
// field.  STG_COVER (rows of any width, field start 16-byte aligned): the
// 16-byte aligned cover of the row's in-field part of x0-2 .. x0+SW+1, the
// field's last chunk clipped to its end.
template <typename T, int STG, bool BANDED = false>
__device__ __forceinline__ void copy_row(const Ctx2<T> &c, int64_t y, bool wanted)
{
    constexpr int A = raw_pad<T>(), NCH = raw_bytes<T>() / 16, sz = (int)sizeof(T);
    if (!wanted) {
        // nothing: rows past the item
    } else if constexpr (BANDED) {
        copy_row_bands<T>(c, y);
    } else if (y >= 0 && y < c.p.H) {
        unsigned char *slot = c.raw + (uint32_t)((y + 16) % NRAW) * raw_bytes<T>();
        if constexpr (STG == fast3d::STG_ALIGNED) {
            const T *base = (const T *)c.p.field;
            for (int q = threadIdx.x; q < NCH; q += kThreads) {
                const int64_t x = (int64_t)c.x0 - A + (int64_t)q * A;
                const bool in = x >= 0 && x < c.p.W;
                cp_async16(fast3d::smem_u32(slot + q * 16), in ? base + y * c.p.W + x : base, in ? 16u : 0u);
            }
        } else {
            const unsigned char *fb = (const unsigned char *)c.p.field;
            const int64_t total = c.p.H * c.p.W * sz;
            const int64_t xlo = max((int64_t)c.x0 - 2, (int64_t)0), xhi = min((int64_t)c.x0 + SW + 2, c.p.W);
            const int64_t rs = (y * c.p.W + xlo) * sz, re = (y * c.p.W + xhi) * sz;
            for (int q = threadIdx.x; q < NCH; q += kThreads) {
                const int64_t cs = (rs & ~(int64_t)15) + 16 * q;
                if (cs >= re) break;
                const int64_t left = total - cs;
                cp_async16(fast3d::smem_u32(slot + q * 16), fb + cs, left < 16 ? (uint32_t)left : 16u);
            }
        }
    }
    cp_async_commit();
}

// Bin row y from its raw slot into ring slot (y mod NR); pixels outside the
// field bin to L.
template <typename T, int STG, bool BANDED = false>
__device__ __forceinline__ void bin_row_raw(Ctx2<T> &c, int64_t y)
{
    constexpr int A = raw_pad<T>(), sz = (int)sizeof(T);
    uint32_t *kr = c.ring + (uint32_t)((y + 8) % NR) * RWORDS;
    const unsigned char *raw = c.raw + (uint32_t)((y + 16) % NRAW) * raw_bytes<T>();
    const uint32_t L = (uint32_t)c.p.L;
    const bool yin = y >= 0 && y < c.p.H;
    const int64_t xlo = max((int64_t)c.x0 - 2, (int64_t)0);
    if constexpr (BANDED) {
        const int sh = c.nb == 4 ? 8 : 9;   // log2 of SW / nb (nb is 2 or 4)
#pragma unroll
        for (int it = 0; it < (RWORDS + kThreads - 1) / kThreads; it++) {
            const int w = threadIdx.x + it * kThreads;
            if (w < RWORDS) kr[w] = band_word(c, raw, y, 2 * w - 2, sh);
        }
        return;
    }
    // byte of pixel x0-2 in the slot (may lie before the slot for the first strip: never read then)
    int64_t b0x;
    if constexpr (STG == fast3d::STG_ALIGNED) b0x = (int64_t)(A - 2) * sz;
    else b0x = (((y * c.p.W + xlo) * sz) & 15) - (xlo - ((int64_t)c.x0 - 2)) * sz;
#pragma unroll
    for (int it = 0; it < (RWORDS + kThreads - 1) / kThreads; it++) {
        const int w = threadIdx.x + it * kThreads;
        if (w < RWORDS) {
            const int64_t gx = (int64_t)c.x0 - 2 + 2 * w;
            const unsigned char *r = raw + b0x + 2 * w * sz;
            const uint32_t b0 = (yin && (c.interior || (gx >= 0 && gx < c.p.W))) ? bin_value2(c, *(const T *)r) : L;
            const uint32_t b1 =
                (yin && (c.interior || (gx + 1 >= 0 && gx + 1 < c.p.W))) ? bin_value2(c, *(const T *)(r + sz)) : L;
            kr[w] = b0 | (b1 << 16);
        }
    }
}

// Asynchronous row step, y = y0 - 2 + t: bin row y+1 (its copies finished
// before the previous barrier), start the copies of row y+2+KA, wait for
// this thread's copies of row y+2, synchronise, then count as ystep does.
template <typename T, bool CONN4, int R, int DM, int STG, bool BANDED, bool SKIP = false>
__device__ __forceinline__ void ystep_async(Ctx2<T> &c, uint32_t (&win)[3][5], int t)
{
    const int y = c.y0 - 2 + t;
    bin_row_raw<T, STG, BANDED>(c, y + 1);
    copy_row<T, STG, BANDED>(c, y + 2 + KA, y + 2 + KA <= c.y1);
    cp_async_wait<KA>();
    __syncthreads();
    count_row<T, CONN4, R, DM, SKIP>(c, win, y);
}

// Walk one item: rows y0-1 .. y1 are binned, rows y0 .. y1-1 counted.
template <typename T, bool CONN4, int DM, bool SKIP = false>
__device__ __forceinline__ void walk_item_2d(Ctx2<T> &c, uint32_t (&win)[3][5])
{
    RowRaw<T> raw;
    load_row<T>(c, c.y0 - 1, raw);
    const int nsteps = c.y1 - c.y0 + 2;
    for (int t = 0; t < nsteps; t += 3) {
        ystep<T, CONN4, 0, DM, SKIP>(c, win, raw, t);
        if (t + 1 < nsteps) ystep<T, CONN4, 1, DM, SKIP>(c, win, raw, t + 1);
        if (t + 2 < nsteps) ystep<T, CONN4, 2, DM, SKIP>(c, win, raw, t + 2);
        after_rows<DM>(c, 3);
    }
}

// Asynchronous walk of one item (same rows as walk_item_2d).
template <typename T, bool CONN4, int DM, int STG, bool BANDED = false, bool SKIP = false>
__device__ __forceinline__ void walk_item_2d_async(Ctx2<T> &c, uint32_t (&win)[3][5])
{
    for (int q = 0; q <= KA; q++) copy_row<T, STG, BANDED>(c, c.y0 - 1 + q, c.y0 - 1 + q <= c.y1);
    cp_async_wait<KA>();
    __syncthreads();
    const int nsteps = c.y1 - c.y0 + 2;
    for (int t = 0; t < nsteps; t += 3) {
        ystep_async<T, CONN4, 0, DM, STG, BANDED, SKIP>(c, win, t);
        if (t + 1 < nsteps) ystep_async<T, CONN4, 1, DM, STG, BANDED, SKIP>(c, win, t + 1);
        if (t + 2 < nsteps) ystep_async<T, CONN4, 2, DM, STG, BANDED, SKIP>(c, win, t + 2);
        after_rows<DM>(c, 3);
    }
    cp_async_wait<0>();
}

}  // namespace fast2d

}  // namespace ec

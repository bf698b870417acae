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

struct Pair2 {
    int ec[2], per[2];
};

// Changes of two horizontally adjacent pixels from their 3 x 3 neighbour
// level pairs n[(dx+1) + 3*(dy+1)] (centre index 4 = the pixels themselves).
template <bool CONN4>
__device__ __forceinline__ Pair2 pair_delta_2d(const uint32_t (&n)[9], uint32_t c)
{
    const uint32_t cm = c | 0x80008000u;
    uint32_t d[9];
#pragma unroll
    for (int i = 0; i < 9; i++) d[i] = (i == 4) ? 0u : cm - n[i] - (i > 4 ? 0x00010001u : 0u);
    const uint32_t fxm = d[3], fxp = d[5], fym = d[1], fyp = d[7];
    const uint32_t cv_mm = fxm | fym | d[0], cv_pm = fxp | fym | d[2];
    const uint32_t cv_mp = fxm | fyp | d[6], cv_pp = fxp | fyp | d[8];
    uint32_t pos = 0, neg = 0;
    pos = gather2<0, 0>(pos, fxm, fxp);
    pos = gather2<1, 1>(pos, fym, fyp);
    neg = gather2<0, 0>(neg, cv_mm, cv_pm);
    neg = gather2<1, 1>(neg, cv_mp, cv_pp);
    Pair2 r;
    const int e0 = popc32(pos & 0xFFFFu), e1 = popc32(pos >> 16);
    r.ec[0] = 1 + e0 - popc32(neg & 0xFFFFu);
    r.ec[1] = 1 + e1 - popc32(neg >> 16);
    r.per[0] = 4 - 2 * e0;
    r.per[1] = 4 - 2 * e1;
    if (CONN4) {
        // QD corners: becomes QD when only the diagonal precedes, stops when
        // exactly the two edge neighbours precede
        uint32_t qp = 0, qm = 0;
        qp = gather2<0, 0>(qp, d[0] & ~fxm & ~fym, d[2] & ~fxp & ~fym);
        qp = gather2<1, 1>(qp, d[6] & ~fxm & ~fyp, d[8] & ~fxp & ~fyp);
        qm = gather2<0, 0>(qm, fxm & fym & ~d[0], fxp & fym & ~d[2]);
        qm = gather2<1, 1>(qm, fxm & fyp & ~d[6], fxp & fyp & ~d[8]);
        r.ec[0] += popc32(qp & 0xFFFFu) - popc32(qm & 0xFFFFu);
        r.ec[1] += popc32(qp >> 16) - popc32(qm >> 16);
    }
    return r;
}

template <typename T>
struct Ctx2 {
    Params p;
    uint32_t *ring;
    int *sh_hist;
    FBin fb;
    IBin<T> ib;
    int x0, y0, y1;
    bool interior;
};

template <typename T>
__device__ __forceinline__ uint32_t bin_value2(const Ctx2<T> &c, T v)
{
    if constexpr (sizeof(T) == 4) return c.fb.uniform ? fbin_uniform(v, c.fb) : fbin(v, c.fb);
    else return c.ib(v);
}

// Bin row y of the strip into ring slot (y mod NR).
template <typename T>
__device__ __forceinline__ void bin_row(Ctx2<T> &c, int64_t y)
{
    uint32_t *kr = c.ring + (uint32_t)((y + 8) % NR) * RWORDS;
    const uint32_t L = (uint32_t)c.p.L;
    const T *f = (const T *)c.p.field;
    const bool yin = y >= 0 && y < c.p.H;
    const T *row = f + (yin ? y : 0) * c.p.W;
#pragma unroll
    for (int it = 0; it < (RWORDS + kThreads - 1) / kThreads; it++) {
        const int w = threadIdx.x + it * kThreads;
        if (w < RWORDS) {
            const int64_t gx = (int64_t)c.x0 - 2 + 2 * w;
            uint32_t b0 = L, b1 = L;
            if (yin) {
                if (c.interior || (gx >= 0 && gx < c.p.W)) b0 = bin_value2(c, row[gx]);
                if (c.interior || (gx + 1 >= 0 && gx + 1 < c.p.W)) b1 = bin_value2(c, row[gx + 1]);
            }
            kr[w] = b0 | (b1 << 16);
        }
    }
}

template <int DM, int D>
constexpr int dm_row2() { return ((DM & 1) && D > 0) + ((DM & 2) && D > 1); }

// One row step, y = y0 - 2 + t: bin row y+1, then (after the barrier) load
// it into window slot (R+1)%3 with R = t mod 3, then count row y if it
// belongs to the item.  Rows y0-1 .. y1 pass through the window.
template <typename T, bool CONN4, int R, int DM>
__device__ __forceinline__ void ystep(Ctx2<T> &c, uint32_t (&win)[3][5], int t)
{
    const int y = c.y0 - 2 + t;
    bin_row<T>(c, y + 1);
    __syncthreads();
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
        const Pair2 d0 = pair_delta_2d<CONN4>(n0, c0);
        const Pair2 d1 = pair_delta_2d<CONN4>(n1, c1);
        const uint32_t key[4] = {c0 & 0xFFFFu, c0 >> 16, c1 & 0xFFFFu, c1 >> 16};
        const int ecv[4] = {d0.ec[0], d0.ec[1], d1.ec[0], d1.ec[1]};
        const int pev[4] = {d0.per[0], d0.per[1], d1.per[0], d1.per[1]};
        const int L = c.p.L;
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const uint32_t k = key[v];
            if (k >= (uint32_t)L) continue;
            if constexpr (DM != 0) {
                int *const h = c.sh_hist;
                if (DM & 1) atomicAdd(&h[dm_row2<DM, 0>() * L + k], ecv[v]);
                if (DM & 2) atomicAdd(&h[dm_row2<DM, 1>() * L + k], pev[v]);
                if (DM & 4) atomicAdd(&h[dm_row2<DM, 2>() * L + k], 1);
            } else {
                const int vals[3] = {ecv[v], pev[v], 1};
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    const int r = c.p.rows[q];
                    if (r < 0 || vals[q] == 0) continue;
                    if (c.sh_hist) atomicAdd(&c.sh_hist[r * L + k], vals[q]);
                    else atomicAdd((unsigned long long *)&c.p.hist[(size_t)r * L + k],
                                   (unsigned long long)(long long)vals[q]);
                }
            }
        }
    }
}

}  // namespace fast2d

}  // namespace ec

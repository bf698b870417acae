// ec_fast2d.cu -- the fast per-pixel 2D histogram kernel for sm_103a.
//
// The 2D analogue of ec_fast3d.cu (Algorithms 1-2 regrouped per entering
// pixel).  A block owns a strip of 1024 columns and walks it down a range of
// rows.  Per row it bins the strip (plus a 2-pixel halo on each side) into a
// 4-deep ring of 16-bit level rows in shared memory; every thread then takes
// 4 consecutive pixels, keeps the 3 x 6 window of levels in registers
// (sliding down the rows), compares two pixels per instruction and adds each
// pixel's changes of EC (8- or 4-connected), perimeter and area at its level
// to the block's shared-memory histogram.
//
// Per pixel c with neighbours preceding it in (level, linear index) order:
//   EC(8-C) change = 1 + #edge neighbours preceding - #corners covered, a
//     corner being covered when one of its 3 other pixels precedes;
//   EC(4-C) change = EC(8-C) change + #corners that become QD (only the
//     diagonal pixel precedes) - #corners that stop being QD (exactly the two
//     edge neighbours precede);
//   perimeter change = 4 - 2 * #edge neighbours preceding; area change = 1.
// (pixel_delta_2d in ec_rules.h is the scalar form of the same counts.)
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

template <typename T, bool CONN4, int DM>
__global__ void __launch_bounds__(kThreads, 3) k_pixel2d_fast(Params p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Ctx2<T> c;
    c.p = p;
    c.ring = (uint32_t *)smem;
    unsigned char *tail = smem + (size_t)NR * RWORDS * 4;
    const int L = p.L;
    c.sh_hist = nullptr;
    if (p.smem_hist) {
        c.sh_hist = (int *)tail;
        for (int i = threadIdx.x; i < p.nd * L; i += kThreads) c.sh_hist[i] = 0;
        tail += ((size_t)p.nd * L * 4 + 15) & ~(size_t)15;
    }
    c.fb = FBin{};
    c.ib = IBin<T>{};
    if constexpr (sizeof(T) == 4) {
        const float *gt = (const float *)p.thr;
        const float *t = gt;
        if (L <= kThrSmem) {
            float *s = (float *)tail;
            for (int k = threadIdx.x; k < L; k += kThreads) s[k] = gt[k];
            t = s;
        }
        c.fb.t = t;
        c.fb.L = L;
        c.fb.t0 = gt[0];
        c.fb.tl = gt[L - 1];
        c.fb.inv = (L > 1 && c.fb.tl > c.fb.t0) ? (float)(L - 1) / (c.fb.tl - c.fb.t0) : 0.f;
        c.fb.uniform = 0;
        if (p.uni && p.uni[0]) {
            c.fb.uniform = 1;
            c.fb.inv = __int_as_float(p.uni[1]);
        }
    } else if constexpr (sizeof(T) == 2) {
        const uint16_t *gt = (const uint16_t *)p.thr;
        c.ib.L = L;
        c.ib.t = (const T *)gt;
        if (gt && L <= kThrSmem) {
            uint16_t *s = (uint16_t *)tail;
            for (int k = threadIdx.x; k < L; k += kThreads) s[k] = gt[k];
            c.ib.t = (const T *)s;
        }
    } else {
        const uint8_t *gt = (const uint8_t *)p.thr;
        uint16_t *tab = (uint16_t *)tail;
        for (int v = threadIdx.x; v < 256; v += kThreads) {
            uint32_t b;
            if (!gt) b = v < L ? (uint32_t)v : (uint32_t)L;
            else {
                int lo = 0, n = L;
                while (n > 0) {
                    const int half = n >> 1;
                    if (gt[lo + half] < v) { lo += half + 1; n -= half + 1; }
                    else n = half;
                }
                b = (uint32_t)lo;
            }
            tab[v] = (uint16_t)b;
        }
        c.ib.table = tab;
        c.ib.L = L;
    }
    __syncthreads();
    uint32_t win[3][5];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int e = 0; e < 5; e++) win[a][e] = 0;
    const int nitems = p.nstrips * p.nrows_items;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int sx = item % p.nstrips, sy = item / p.nstrips;
        c.x0 = sx * SW;
        c.y0 = sy * p.ry;
        c.y1 = (int)min((int64_t)c.y0 + p.ry, p.H);
        c.interior = c.x0 >= 2 && c.x0 + SW + 2 <= p.W;
        __syncthreads();   // ring reuse across items
        // steps t = 0 .. (y1 - y0) + 1: bin rows y0-1 .. y1, count rows y0 .. y1-1
        const int nsteps = c.y1 - c.y0 + 2;
        for (int t = 0; t < nsteps; t += 3) {
            ystep<T, CONN4, 0, DM>(c, win, t);
            if (t + 1 < nsteps) ystep<T, CONN4, 1, DM>(c, win, t + 1);
            if (t + 2 < nsteps) ystep<T, CONN4, 2, DM>(c, win, t + 2);
        }
    }
    if (c.sh_hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < p.nd * L; i += kThreads) {
            const int v = c.sh_hist[i];
            if (v) atomicAdd((unsigned long long *)&p.hist[i], (unsigned long long)(long long)v);
        }
    }
}

template <typename T, bool CONN4, int DM = 0>
static int launch_t(const Params &p, size_t smem, int num_sms, int items, int grid_override, cudaStream_t s)
{
    auto kern = k_pixel2d_fast<T, CONN4, DM>;
    EC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    EC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem));
    if (occ < 1) { set_error("fast 2D kernel does not fit (%zu B shared)", smem); return EC_ERR_UNSUPPORTED; }
    int grid = grid_override > 0 ? grid_override : num_sms * occ;
    grid = grid > items ? items : grid;
    kern<<<grid, kThreads, smem, s>>>(p);
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

template <typename T>
static int launch_dt(const Params &p, uint32_t desc, size_t smem, int num_sms, int items, int grid, cudaStream_t s)
{
    if (p.smem_hist && !p.conn4) {
        if (desc == 1u) return launch_t<T, false, 1>(p, smem, num_sms, items, grid, s);
        if (desc == 7u) return launch_t<T, false, 7>(p, smem, num_sms, items, grid, s);
    }
    return p.conn4 ? launch_t<T, true>(p, smem, num_sms, items, grid, s)
                   : launch_t<T, false>(p, smem, num_sms, items, grid, s);
}

}  // namespace fast2d

int launch_uniform_check(const float *thr, int32_t L, int *uni, cudaStream_t s);

int launch_fast_2d(const void *field, const int64_t dims[2], const BinArgs &ba, const HistArgs &ha, int connectivity,
                   int grid_override, int num_sms, int *err_flag, cudaStream_t s)
{
    using namespace fast2d;
    if (ba.L > 32767 || dims[0] > INT32_MAX / 2 || dims[1] > INT32_MAX / 2) return EC_ERR_UNSUPPORTED;
    Params p{};
    p.field = field;
    p.H = dims[0];
    p.W = dims[1];
    p.nstrips = (int)((p.W + SW - 1) / SW);
    // rows per work item: enough items to fill the GPU, at most 128 rows
    const int64_t target = (int64_t)num_sms * 6;
    int64_t ry = (p.H * p.nstrips + target - 1) / target;
    ry = ry < 8 ? 8 : (ry > 128 ? 128 : ry);
    p.ry = (int)ry;
    p.nrows_items = (int)((p.H + ry - 1) / ry);
    const int64_t items64 = (int64_t)p.nstrips * p.nrows_items;
    if (items64 > INT32_MAX) return EC_ERR_UNSUPPORTED;
    p.L = ba.L;
    p.thr = ba.thr;
    p.hist = ha.hist;
    uint32_t desc = 0;
    for (int i = 0; i < kMaxDesc; i++) {
        p.rows[i] = ha.rows.row[i];
        if (ha.rows.row[i] >= 0) desc |= 1u << i;
    }
    p.nd = ha.rows.nd;
    p.smem_hist = ha.smem_hist;
    p.conn4 = connectivity == 4 ? 1 : 0;
    p.uni = nullptr;
    if (ba.dtype == EC_F32) {
        p.uni = err_flag + 2;
        int rc = launch_uniform_check((const float *)ba.thr, ba.L, err_flag + 2, s);
        if (rc) return rc;
    }
    const int dsz = ba.dtype == EC_F32 ? 4 : (ba.dtype == EC_U16 ? 2 : 1);
    size_t smem = (size_t)NR * RWORDS * 4;
    if (p.smem_hist) smem += ((size_t)p.nd * p.L * 4 + 15) & ~(size_t)15;
    if (dsz == 1) smem += 512;
    else if (ba.thr && p.L <= kThrSmem) smem += ((size_t)p.L * dsz + 15) & ~(size_t)15;
    const int items = (int)items64;
    switch (ba.dtype) {
    case EC_F32: return launch_dt<float>(p, desc, smem, num_sms, items, grid_override, s);
    case EC_U16: return launch_dt<uint16_t>(p, desc, smem, num_sms, items, grid_override, s);
    case EC_U8: return launch_dt<uint8_t>(p, desc, smem, num_sms, items, grid_override, s);
    }
    return EC_ERR_DTYPE;
}

}  // namespace ec

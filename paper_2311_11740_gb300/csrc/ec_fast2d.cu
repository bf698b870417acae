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

#include "ec_fast2d.cuh"

namespace ec {

namespace fast2d {

// Row staging of the 2D kernel: per-pixel loads one row ahead, or cp.async
// rows three rows ahead (whole 16-byte aligned rows, or 16-byte covers).
enum { ROWS_LOADS = 0, ROWS_ALIGNED = 1, ROWS_COVER = 2 };

template <typename T, bool CONN4, int DM, int ROWS>
__global__ void __launch_bounds__(kThreads, 3) k_pixel2d_fast(Params p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // layout: [key ring NR*RWORDS*4] [raw rows NRAW*raw_bytes (ASYNC)] [hist nd*(L+1)*4] [thresholds / byte table]
    Ctx2<T> c;
    c.p = p;
    c.ring = (uint32_t *)smem;
    unsigned char *tail = smem + (size_t)NR * RWORDS * 4;
    c.raw = tail;
    if (ROWS != ROWS_LOADS) tail += (size_t)NRAW * raw_bytes<T>();
    const int L = p.L;
    c.sh_hist = nullptr;
    const int slots = hist_slots2<DM>(p.nd);
    if (p.smem_hist) {
        c.sh_hist = (int *)tail;
        for (int i = threadIdx.x; i < slots * (L + 1); i += kThreads) c.sh_hist[i] = 0;
        tail += ((size_t)slots * (L + 1) * 4 + 15) & ~(size_t)15;
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
        c.fb.lm1 = (float)(L - 1);
        c.fb.off = 0.f;
        c.fb.uniform = 0;
        if (p.uni && p.uni[0]) {
            c.fb.uniform = 1;
            c.fb.inv = __int_as_float(p.uni[1]);
            c.fb.off = __int_as_float(p.uni[2]);
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
        // a strip whose counted columns reach past the field leaves out the
        // pixels at level L (the generic descriptor path always does)
        if (DM != 0 && c.x0 + SW > p.W) {
            if constexpr (ROWS == ROWS_ALIGNED) walk_item_2d_async<T, CONN4, DM, fast3d::STG_ALIGNED, false, true>(c, win);
            else if constexpr (ROWS == ROWS_COVER) walk_item_2d_async<T, CONN4, DM, fast3d::STG_COVER, false, true>(c, win);
            else walk_item_2d<T, CONN4, DM, true>(c, win);
        } else {
            if constexpr (ROWS == ROWS_ALIGNED) walk_item_2d_async<T, CONN4, DM, fast3d::STG_ALIGNED>(c, win);
            else if constexpr (ROWS == ROWS_COVER) walk_item_2d_async<T, CONN4, DM, fast3d::STG_COVER>(c, win);
            else walk_item_2d<T, CONN4, DM>(c, win);
        }
    }
    if (c.sh_hist) {
        if constexpr (DM == 7) {
            __syncthreads();
            exchange_packed2(c.sh_hist, L);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < p.nd * L; i += kThreads) {
            // global rows are [nd][L]; compile-time rows are interleaved [L+1][slots]
            // (DM 7: EC, packed, perimeter, area, spare)
            int v;
            if constexpr (DM != 0) {
                const int r = i / L, k = i - r * L;
                v = c.sh_hist[k * slots + (DM == 7 && r > 0 ? r + 1 : r)];
            } else {
                v = c.sh_hist[i];
            }
            if (v) atomicAdd((unsigned long long *)&p.hist[i], (unsigned long long)(long long)v);
        }
    }
}

template <typename T, bool CONN4, int DM = 0>
static int launch_t(const Params &p, size_t smem, int num_sms, int items, int grid_override, int rows,
                    cudaStream_t s)
{
    auto kern = rows == ROWS_ALIGNED ? k_pixel2d_fast<T, CONN4, DM, ROWS_ALIGNED>
                : rows == ROWS_COVER ? k_pixel2d_fast<T, CONN4, DM, ROWS_COVER>
                                     : k_pixel2d_fast<T, CONN4, DM, ROWS_LOADS>;
    if (rows != ROWS_LOADS) smem += (size_t)NRAW * raw_bytes<T>();
    int occ = 0;
    if (const int orc = kernel_occupancy((const void *)kern, kThreads, smem, &occ)) return orc;
    if (occ < 1) { set_error("fast 2D kernel does not fit (%zu B shared)", smem); return EC_ERR_UNSUPPORTED; }
    int grid = grid_override > 0 ? grid_override : num_sms * occ;
    grid = grid > items ? items : grid;
    kern<<<grid, kThreads, smem, s>>>(p);
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

template <typename T>
static int launch_dt(const Params &p, uint32_t desc, size_t smem, int num_sms, int items, int grid, int rows,
                     cudaStream_t s)
{
    if (p.smem_hist && !p.conn4) {
        if (desc == 1u) return launch_t<T, false, 1>(p, smem, num_sms, items, grid, rows, s);
        if (desc == 7u && (size_t)5 * ((size_t)p.L + 1) * 4 <= kSmemHistBudget) {
            // five words per level instead of the three rows
            const size_t extra = (((size_t)5 * (p.L + 1) * 4 + 15) & ~(size_t)15) -
                                 (((size_t)3 * (p.L + 1) * 4 + 15) & ~(size_t)15);
            return launch_t<T, false, 7>(p, smem + extra, num_sms, items, grid, rows, s);
        }
    }
    return p.conn4 ? launch_t<T, true>(p, smem, num_sms, items, grid, rows, s)
                   : launch_t<T, false>(p, smem, num_sms, items, grid, rows, s);
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
    if (p.smem_hist) smem += ((size_t)p.nd * (p.L + 1) * 4 + 15) & ~(size_t)15;
    if (dsz == 1) smem += 512;
    else if (ba.thr && p.L <= kThrSmem) smem += ((size_t)p.L * dsz + 15) & ~(size_t)15;
    const int items = (int)items64;
    // rows copied with cp.async when the field starts 16-byte aligned: whole
    // rows if every row starts aligned too, else their 16-byte covers
    const bool cover = ((uintptr_t)field % 16) == 0;
    const int rows = !cover ? ROWS_LOADS : (((size_t)p.W * dsz) % 16 == 0 ? ROWS_ALIGNED : ROWS_COVER);
    switch (ba.dtype) {
    case EC_F32: return launch_dt<float>(p, desc, smem, num_sms, items, grid_override, rows, s);
    case EC_U16: return launch_dt<uint16_t>(p, desc, smem, num_sms, items, grid_override, rows, s);
    case EC_U8: return launch_dt<uint8_t>(p, desc, smem, num_sms, items, grid_override, rows, s);
    }
    return EC_ERR_DTYPE;
}

}  // namespace ec

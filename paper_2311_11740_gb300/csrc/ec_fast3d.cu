// ec_fast3d.cu -- the fast per-voxel 3D histogram kernel for sm_103a.
//
// One block owns a 64 x 16 column of voxels and walks it along z in work
// items of `tz` planes.  Per plane:
//   * float32 fields: the Tensor Memory Accelerator copies a 72 x 18 box of
//     the plane (x from x0-4 so the start is 16-byte aligned, y from y0-1)
//     into an 8-deep shared-memory ring, tracked by mbarriers, about six
//     planes ahead of use.  Out-of-bounds elements arrive as NaN, which bins
//     to the never-active level, exactly what cells outside the field are.
//     Other dtypes (or unaligned float32 fields) are read with plain loads.
//   * every thread bins pairs of values of the staged plane to 16-bit levels
//     (a guess from the uniform spacing, checked against the thresholds and
//     corrected by binary search when it misses) into a 4-deep ring of key
//     planes;
//   * every thread then handles 4 consecutive voxels of its row: it keeps the
//     3 x 3 x 6 key window in registers (sliding along z), compares pairs of
//     voxels per instruction (ec_swar.h) and adds each voxel's contribution
//     change at its level to the block's shared-memory histogram.
// The rings are ordered by one __syncthreads per two planes on the TMA path
// (two planes binned per barrier, three planes ahead of their count) and one
// per plane with plain loads.  Waits on mbarriers are bounded: a wait that
// gives up sets an error flag and the block returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "ec_internal.h"
#include "ec_rules.h"
#include "ec_swar.h"

#include "ec_fast3d.cuh"

namespace ec {

namespace fast3d {

// Decide whether bin_guess is always the true bin or one below it, for every
// float (guess_ok_for_level on every level 0..L).  Writes uni[0] (1 = fast
// path exact) and uni[1], uni[2] (the guess's scale and offset, float bits).
__global__ void k_uniform_check(const float *t, int L, int *uni)
{
    __shared__ int ok;
    float inv, off;
    guess_params(t[0], t[L - 1], L, inv, off);
    if (threadIdx.x == 0) ok = 1;
    __syncthreads();
    for (int k = threadIdx.x; k <= L; k += blockDim.x)
        if (!guess_ok_for_level(t, L, k, inv, off)) ok = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        uni[0] = ok;
        uni[1] = __float_as_int(inv);
        uni[2] = __float_as_int(off);
    }
}

#ifndef EC_FAST_MIN_BLOCKS
#define EC_FAST_MIN_BLOCKS 3
#endif

// Staging modes of the fast 3D kernel.
// MODE_ASYNC: cp.async 16-byte chunks, rows start 16-byte aligned;
// MODE_COVER: cp.async 16-byte chunks covering rows of any width (field
// start 16-byte aligned).
enum { MODE_PLAIN = 0, MODE_TMA = 1, MODE_ASYNC = 2, MODE_COVER = 3 };

template <typename T>
constexpr size_t stage_bytes(int mode)
{
    return mode == MODE_TMA      ? (size_t)NS * FSTRIDE * sizeof(float)
           : (mode == MODE_ASYNC || mode == MODE_COVER) ? ((size_t)NRAWP2 * rplane_bytes<T>() + 127) / 128 * 128
                                                         : 0;
}

// SLICE: count with the planar form of ec_slice.h (two planes in registers)
// instead of the 26-neighbour form (three planes); same staging and schedule.
template <typename T, int MODE, bool PER, int DM, int SCHED = 0, bool SLICE = false>
__global__ void __launch_bounds__(kThreads, EC_FAST_MIN_BLOCKS)
k_voxel3d_fast(const __grid_constant__ CUtensorMap tmap, Params p)
{
    constexpr bool TMA = MODE == MODE_TMA;
    extern __shared__ __align__(128) unsigned char smem[];
    // layout: [float ring NS*FSTRIDE*4 (TMA) | raw plane ring (ASYNC)] [key ring NK*KWORDS*4] [mbar NS*8]
    //         [abort 16] [hist nd*(L+1)*4] [thresholds / byte table]
    Ctx<T> c;
    c.p = p;
    const size_t fbytes = stage_bytes<T>(MODE);
    c.fring = (float *)smem;
    c.raw = smem;
    c.kring = (uint32_t *)(smem + fbytes);
    c.bars = (uint64_t *)(smem + fbytes + (size_t)NK * KWORDS * 4);
    c.abort_flag = (volatile int *)(c.bars + NS);
    unsigned char *tail = (unsigned char *)(c.bars + NS) + 16;
    const int L = p.L;
    c.sh_hist = nullptr;
    if (p.smem_hist) {
        c.sh_hist = (int *)tail;
        for (int i = threadIdx.x; i < p.nd * (L + 1); i += kThreads) c.sh_hist[i] = 0;
        tail += ((size_t)p.nd * (L + 1) * 4 + 15) & ~(size_t)15;
        c.pw1 = c.pw2 = nullptr;
        c.pstride = ((L + 31) & ~31) + 1;
        if (p.pairs) {
            c.pw1 = (uint32_t *)tail;
            c.pw2 = c.pw1 + 2 * c.pstride;
            for (int i = threadIdx.x; i < 4 * c.pstride; i += kThreads) c.pw1[i] = 0u;
            tail += ((size_t)4 * c.pstride * 4 + 15) & ~(size_t)15;
        }
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
    if (TMA && threadIdx.x == 0) {
        for (int i = 0; i < NS; i++) mbar_init(&c.bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x == 0) *c.abort_flag = 0;
    __syncthreads();

    c.tr = threadIdx.x >> 4;
    c.tc = threadIdx.x & 15;
    c.bin3 = bin3_offsets(threadIdx.x);
    c.parity = 0;
    c.inflight = 0;
    uint32_t seq = 0;
    const int nitems = p.nbx * p.nby * p.nbz;
    uint32_t win[3][3][5];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++)
#pragma unroll
            for (int e = 0; e < 5; e++) win[a][b][e] = 0;

    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % p.nbx, by = (item / p.nbx) % p.nby, bz = item / (p.nbx * p.nby);
        c.x0 = bx * TXF;
        c.y0 = by * TYF;
        c.z0 = p.zc0 + bz * p.tz;
        c.z1 = min(c.z0 + p.tz, p.zc1);
        c.interior = c.x0 >= 4 && c.x0 + TXF + 4 <= p.W;
        c.skip = c.x0 + TXF > p.W || c.y0 + TYF > p.H;
        __syncthreads();   // the previous item is done with both rings
        c.base = seq;
        if constexpr (SLICE) {
            if constexpr (TMA) {
                if (threadIdx.x == 0) {
                    for (int q = 0; q < NS - 2; q++) {
                        const int pz = c.z0 - 1 + q;
                        if (pz > c.z1) break;
                        const uint32_t slot = (c.base + q) % NS;
                        mbar_expect_tx(&c.bars[slot], BX * BY * 4);
                        tma_load_plane(c.fring + slot * FSTRIDE, &tmap, c.x0 - 4, c.y0 - 1, pz, &c.bars[slot]);
                        c.inflight |= 1u << slot;
                    }
                }
                if (!walk_slice_tma<T, PER, DM>(c, &tmap)) return;
            } else if constexpr (MODE == MODE_ASYNC || MODE == MODE_COVER) {
                constexpr int STG = MODE == MODE_ASYNC ? STG_ALIGNED : STG_COVER;
                if (!walk_slice_async2<T, PER, DM, STG>(c)) return;
            } else {
                if (!walk_slice_plain<T, PER, DM>(c)) return;
            }
        } else if constexpr (TMA) {
            // planes z0-1 .. z0+NS-4 now; the barrier steps request the rest
            if (threadIdx.x == 0) {
                for (int q = 0; q < NS - 2; q++) {
                    const int pz = c.z0 - 1 + q;
                    if (pz > c.z1) break;
                    const uint32_t slot = (c.base + q) % NS;
                    mbar_expect_tx(&c.bars[slot], BX * BY * 4);
                    tma_load_plane(c.fring + slot * FSTRIDE, &tmap, c.x0 - 4, c.y0 - 1, pz, &c.bars[slot]);
                    c.inflight |= 1u << slot;
                }
            }
            const int nsteps = c.z1 - c.z0 + 4;
            for (int t = 0; t < nsteps; t += 3) {
                if (!zstep_tma<T, PER, 0, DM, SCHED>(c, &tmap, win, t)) return;
                if (t + 1 < nsteps && !zstep_tma<T, PER, 1, DM, SCHED>(c, &tmap, win, t + 1)) return;
                if (t + 2 < nsteps && !zstep_tma<T, PER, 2, DM, SCHED>(c, &tmap, win, t + 2)) return;
            }
        } else if constexpr (MODE == MODE_ASYNC || MODE == MODE_COVER) {
            constexpr int STG = MODE == MODE_ASYNC ? STG_ALIGNED : STG_COVER;
            if (!walk_item_async2<T, PER, DM, SCHED, STG>(c, win)) return;
        } else {
            const int nsteps = c.z1 - c.z0 + 3;
            for (int t = 0; t < nsteps; t += 3) {
                if (!zstep<T, PER, 0, DM, SCHED>(c, win, t)) return;
                if (t + 1 < nsteps && !zstep<T, PER, 1, DM, SCHED>(c, win, t + 1)) return;
                if (t + 2 < nsteps && !zstep<T, PER, 2, DM, SCHED>(c, win, t + 2)) return;
            }
        }
        if (TMA) seq += (uint32_t)(c.z1 - c.z0 + 2);
    }
    if (c.sh_hist && p.pairs) {
        __syncthreads();
        for (int k = threadIdx.x; k < L; k += kThreads) {
            int lo, hi;
            for (int cpy = 0; cpy < 2; cpy++) {
                pair_decode(c.pw1[cpy * c.pstride + k], lo, hi);
                if (p.rows[0] >= 0) c.sh_hist[p.rows[0] * L + k] += lo;
                if (p.rows[3] >= 0) c.sh_hist[p.rows[3] * L + k] += hi;
                pair_decode(c.pw2[cpy * c.pstride + k], lo, hi);
                if (p.rows[2] >= 0) c.sh_hist[p.rows[2] * L + k] += lo;
                if (p.rows[1] >= 0) c.sh_hist[p.rows[1] * L + k] += hi;
            }
        }
    }
    if (c.sh_hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < p.nd * L; i += kThreads) {
            // global rows are [nd][L]; level L of the interleaved layout is dropped
            int v;
            if constexpr (SLICE || interleaved_hist<DM, SCHED>()) {
                const int r = i / L, k = i - r * L;
                v = c.sh_hist[k * (DM ? dm_nd<DM>() : p.nd) + r];
            } else {
                v = c.sh_hist[i];
            }
            if (v) atomicAdd((unsigned long long *)&p.hist[i], (unsigned long long)(long long)v);
        }
    }
}

// ------------------------------------------------------------------- host

}  // namespace fast3d

namespace fast3d {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();
}

int launch_uniform_check(const float *thr, int32_t L, int *uni, cudaStream_t s)
{
    fast3d::k_uniform_check<<<1, 256, 0, s>>>(thr, L, uni);
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

void *tma_encode_fn()
{
    return (void *)fast3d::encode_fn();
}

namespace fast3d {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
        else
            cudaGetLastError();
    }
    return fn;
}

template <typename T>
static size_t smem_bytes(int mode, int dtype_size, int nd, int L, bool smem_hist, bool has_thr, bool pairs)
{
    size_t b = stage_bytes<T>(mode);
    b += (size_t)NK * KWORDS * 4 + NS * 8 + 16;
    if (smem_hist) b += ((size_t)nd * (L + 1) * 4 + 15) & ~(size_t)15;
    if (smem_hist && pairs) b += ((size_t)4 * (((L + 31) & ~31) + 1) * 4 + 15) & ~(size_t)15;
    if (dtype_size == 1) b += 512;
    else if (has_thr && L <= kThrSmem) b += ((size_t)L * dtype_size + 15) & ~(size_t)15;
    return b;
}

template <typename T, int MODE, bool PER, int DM = 0, int SCHED = 0, bool SLICE = false>
static int launch_t(const CUtensorMap &map, const Params &p, size_t smem, int num_sms, int items, int grid_override,
                    cudaStream_t s)
{
    auto kern = k_voxel3d_fast<T, MODE, PER, DM, SCHED, SLICE>;
    int occ = 0;
    if (const int orc = kernel_occupancy((const void *)kern, kThreads, smem, &occ)) return orc;
    if (occ < 1) { set_error("fast 3D kernel does not fit (%zu B shared)", smem); return EC_ERR_UNSUPPORTED; }
    int grid = grid_override > 0 ? grid_override : num_sms * occ;
    grid = grid > items ? items : grid;
    kern<<<grid, kThreads, smem, s>>>(map, p);
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

// Planar-form launches (shared-memory histogram): compile-time histogram rows
// for the common descriptor sets, run-time rows otherwise.
template <typename T, int MODE>
static int launch_slice(const CUtensorMap &map, const Params &p, uint32_t desc, bool per, size_t smem, int num_sms,
                        int items, int grid_override, cudaStream_t s)
{
    if (desc == 1u) return launch_t<T, MODE, false, 1, 0, true>(map, p, smem, num_sms, items, grid_override, s);
    if (desc == 13u) return launch_t<T, MODE, false, 13, 0, true>(map, p, smem, num_sms, items, grid_override, s);
    if (desc == 15u) return launch_t<T, MODE, true, 15, 0, true>(map, p, smem, num_sms, items, grid_override, s);
    return per ? launch_t<T, MODE, true, 0, 0, true>(map, p, smem, num_sms, items, grid_override, s)
               : launch_t<T, MODE, false, 0, 0, true>(map, p, smem, num_sms, items, grid_override, s);
}

// Plain-load and cp.async modes: compile-time histogram rows for the common
// descriptor sets on the cp.async path, run-time rows otherwise.
template <typename T, int MODE>
static int launch_loads(const CUtensorMap &map, const Params &p, uint32_t desc, bool per, size_t smem, int num_sms,
                        int items, int grid_override, cudaStream_t s)
{
    if (p.smem_hist && p.planar) return launch_slice<T, MODE>(map, p, desc, per, smem, num_sms, items, grid_override, s);
    if constexpr (MODE == MODE_ASYNC || MODE == MODE_COVER) {
        if (p.smem_hist) {
            if (desc == 1u) return launch_t<T, MODE, false, 1>(map, p, smem, num_sms, items, grid_override, s);
            if (desc == 13u) return launch_t<T, MODE, false, 13>(map, p, smem, num_sms, items, grid_override, s);
            if (desc == 15u) return launch_t<T, MODE, true, 15>(map, p, smem, num_sms, items, grid_override, s);
        }
    }
    return per ? launch_t<T, MODE, true>(map, p, smem, num_sms, items, grid_override, s)
               : launch_t<T, MODE, false>(map, p, smem, num_sms, items, grid_override, s);
}

}  // namespace fast3d

// Returns EC_ERR_UNSUPPORTED (without launching) when the request does not fit
// this kernel (more than kMaxFastL3 levels, or dims beyond 32-bit tile indices).
int launch_fast_3d(const void *field, const int64_t dims[3], const BinArgs &ba, const HistArgs &ha, int tile_z,
                   int grid_override, int num_sms, int *err_flag, cudaStream_t s, const int zrange[4])
{
    using namespace fast3d;
    if (ha.planar && ha.schedule <= 1) {
        // float32 TMA fields with up to 1024 levels: two stacked quads per thread
        const int rc = launch_planar_3d(field, dims, ba, ha, tile_z, grid_override, num_sms, err_flag, s, zrange);
        if (rc != EC_ERR_UNSUPPORTED) return rc;
    }
    if (ba.L > kMaxFastL3 || dims[0] > INT32_MAX / 2 || dims[1] > INT32_MAX / 2 || dims[2] > INT32_MAX / 2)
        return EC_ERR_UNSUPPORTED;
    Params p{};
    p.field = field;
    p.D = dims[0]; p.H = dims[1]; p.W = dims[2];
    p.tz = tile_z > 0 ? tile_z : 64;
    p.zc0 = zrange ? zrange[0] : 0;
    p.zc1 = zrange ? zrange[1] : (int)p.D;
    p.zv0 = zrange ? zrange[2] : 0;
    p.zv1 = zrange ? zrange[3] : (int)p.D;
    p.nbx = (int)((p.W + TXF - 1) / TXF);
    p.nby = (int)((p.H + TYF - 1) / TYF);
    p.nbz = (p.zc1 - p.zc0 + p.tz - 1) / p.tz;
    if (p.nbz < 1) return EC_OK;
    const int64_t items64 = (int64_t)p.nbx * p.nby * p.nbz;
    if (items64 > INT32_MAX) return EC_ERR_UNSUPPORTED;
    p.L = ba.L;
    p.thr = ba.thr;
    p.hist = ha.hist;
    for (int i = 0; i < kMaxDesc; i++) p.rows[i] = ha.rows.row[i];
    p.nd = ha.rows.nd;
    p.smem_hist = ha.smem_hist;
    p.err = err_flag;
    p.agg = ha.schedule == 2 ? 1 : 0;
    p.pairs = 0;
    p.uni = nullptr;
    if (ba.dtype == EC_F32) {
        p.uni = err_flag + 2;
        if (!ba.uni_ready) {
            k_uniform_check<<<1, 256, 0, s>>>((const float *)ba.thr, ba.L, err_flag + 2);
            EC_CUDA(cudaGetLastError());
        }
    }
    const bool per = ha.rows.row[1] >= 0;
    uint32_t desc = 0;
    for (int i = 0; i < kMaxDesc; i++)
        if (ha.rows.row[i] >= 0) desc |= 1u << i;
    const int dsz = ba.dtype == EC_F32 ? 4 : (ba.dtype == EC_U16 ? 2 : 1);

    CUtensorMap map;
    memset(&map, 0, sizeof map);
    bool tma = false;
    if (ba.dtype == EC_F32 && (p.W % 4) == 0 && ((uintptr_t)field % 16) == 0) {
        PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
        if (enc) {
            cuuint64_t gdim[3] = {(cuuint64_t)p.W, (cuuint64_t)p.H, (cuuint64_t)p.D};
            cuuint64_t gstride[2] = {(cuuint64_t)p.W * 4, (cuuint64_t)p.W * p.H * 4};
            cuuint32_t box[3] = {(cuuint32_t)BX, (cuuint32_t)BY, 1};
            cuuint32_t estr[3] = {1, 1, 1};
            CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(field), gdim, gstride, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA);
            tma = r == CUDA_SUCCESS;
        }
    }
    if (ha.schedule == 3 && ha.smem_hist && tma && (desc == 13u || desc == 15u)) p.pairs = 1;
    // the planar form needs the block histogram and the one-atomic schedule
    p.planar = ha.planar && ha.smem_hist && !p.agg && !p.pairs ? 1 : 0;
    // without TMA, rows are staged with 16-byte cp.async chunks when the field
    // starts 16-byte aligned: whole rows if every row does too, else the
    // aligned cover of each row
    const bool cover = ((uintptr_t)field % 16) == 0;
    const bool async = cover && ((size_t)p.W * dsz) % 16 == 0;
    const int mode = tma ? MODE_TMA : (async ? MODE_ASYNC : (cover ? MODE_COVER : MODE_PLAIN));
    const int items = (int)items64;
    switch (ba.dtype) {
    case EC_F32: {
        const size_t smem = smem_bytes<float>(mode, dsz, p.nd, p.L, p.smem_hist != 0, ba.thr != nullptr, p.pairs != 0);
        if (tma && p.smem_hist && p.planar)
            return launch_slice<float, MODE_TMA>(map, p, desc, per, smem, num_sms, items, grid_override, s);
        if (tma && p.smem_hist && !p.agg) {
            // descriptor sets with compile-time histogram rows
            if (p.pairs) {
                if (desc == 13u) return launch_t<float, MODE_TMA, false, 13, 3>(map, p, smem, num_sms, items, grid_override, s);
                if (desc == 15u) return launch_t<float, MODE_TMA, true, 15, 3>(map, p, smem, num_sms, items, grid_override, s);
            }
            if (desc == 1u) return launch_t<float, MODE_TMA, false, 1>(map, p, smem, num_sms, items, grid_override, s);
            if (desc == 13u) return launch_t<float, MODE_TMA, false, 13>(map, p, smem, num_sms, items, grid_override, s);
            if (desc == 15u) return launch_t<float, MODE_TMA, true, 15>(map, p, smem, num_sms, items, grid_override, s);
        }
        if (tma && p.agg)
            return per ? launch_t<float, MODE_TMA, true, 0, 2>(map, p, smem, num_sms, items, grid_override, s)
                       : launch_t<float, MODE_TMA, false, 0, 2>(map, p, smem, num_sms, items, grid_override, s);
        if (tma) return per ? launch_t<float, MODE_TMA, true>(map, p, smem, num_sms, items, grid_override, s)
                            : launch_t<float, MODE_TMA, false>(map, p, smem, num_sms, items, grid_override, s);
        if (async) return launch_loads<float, MODE_ASYNC>(map, p, desc, per, smem, num_sms, items, grid_override, s);
        if (cover) return launch_loads<float, MODE_COVER>(map, p, desc, per, smem, num_sms, items, grid_override, s);
        return launch_loads<float, MODE_PLAIN>(map, p, desc, per, smem, num_sms, items, grid_override, s);
    }
    case EC_U16: {
        const size_t smem = smem_bytes<uint16_t>(mode, dsz, p.nd, p.L, p.smem_hist != 0, ba.thr != nullptr, false);
        if (async) return launch_loads<uint16_t, MODE_ASYNC>(map, p, desc, per, smem, num_sms, items, grid_override, s);
        if (cover) return launch_loads<uint16_t, MODE_COVER>(map, p, desc, per, smem, num_sms, items, grid_override, s);
        return launch_loads<uint16_t, MODE_PLAIN>(map, p, desc, per, smem, num_sms, items, grid_override, s);
    }
    case EC_U8: {
        const size_t smem = smem_bytes<uint8_t>(mode, dsz, p.nd, p.L, p.smem_hist != 0, ba.thr != nullptr, false);
        if (async) return launch_loads<uint8_t, MODE_ASYNC>(map, p, desc, per, smem, num_sms, items, grid_override, s);
        if (cover) return launch_loads<uint8_t, MODE_COVER>(map, p, desc, per, smem, num_sms, items, grid_override, s);
        return launch_loads<uint8_t, MODE_PLAIN>(map, p, desc, per, smem, num_sms, items, grid_override, s);
    }
    }
    return EC_ERR_DTYPE;
}

}  // namespace ec

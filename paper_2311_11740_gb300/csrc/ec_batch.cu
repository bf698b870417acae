// ec_batch.cu -- curves of many uneven fields in one persistent launch.
//
// Sec. 4 of the paper notes that small images gain little from parallelising
// one image at a time.  Here every field of a batch is cut into work items
// (64 x 16 x 64 voxel tiles for 3D fields, 1024 x 64 pixel tiles for 2D
// fields); one persistent kernel pulls items from a global counter, so
// fields of any size and mix share the whole GPU.  Per item a block:
//   1. loads the item's field parameters and binning tables into shared
//      memory (thresholds, byte-value table, uniform-spacing check);
//   2. walks the tile exactly like the single-field kernels (the 3D path is
//      the fast paired-comparison code of ec_fast3d.cuh with plain loads);
//   3. adds its shared-memory histogram into the field's int64 histogram;
//   4. counts the item as done; the block that completes a field's last item
//      computes that field's running sums into its output.
// Nothing waits on another block.  The launch sequence (table upload, reset,
// kernel) is captured once into a CUDA graph and later calls update and
// relaunch the instantiated graph.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "ec_fast2d.cuh"

namespace ec {

namespace batch {

using namespace fast3d;

struct BField {
    const void *field;
    int64_t dims[3];      // 3D: {D, H, W}; 2D: {1, H, W}
    const void *thr;
    long long *hist;      // int64 [nd][L]
    int64_t *out;
    int ndim, dtype, L, conn4, nd, nitems;
    int rows[kMaxDesc];
    int smem_hist;
    int done_idx;
};

struct BItem {
    int f;
    int x0, y0, z0, z1;   // 2D: z0..z1 are the item's rows; y0 > 1: that many row bands (banded strip)
};

constexpr int kThrMaxB = 4096;

struct Shared {
    uint32_t *kring;
    unsigned char *raw;    // raw plane ring of the cp.async staging (3D items)
    volatile int *abort_flag;
    int *sh_hist;          // may be too small for a field: then nullptr for that field
    size_t hist_cap;       // ints
    unsigned char *thr;    // thresholds / byte table
    int *item_bcast;
};

// Binning tables of a field into shared memory; returns the uniform flag for
// float32 (1 = the spacing guess is exact for every value).
__device__ int load_binning(const BField &F, const Shared &S, FBin &fb)
{
    const int L = F.L;
    if (F.dtype == EC_F32) {
        const float *gt = (const float *)F.thr;
        const float *t = gt;
        if (L <= kThrMaxB) {
            float *s = (float *)S.thr;
            for (int k = threadIdx.x; k < L; k += blockDim.x) s[k] = gt[k];
            t = s;
        }
        fb.t = t;
        fb.L = L;
        fb.t0 = gt[0];
        fb.tl = gt[L - 1];
        guess_params(fb.t0, fb.tl, L, fb.inv, fb.off);
        fb.lm1 = (float)(L - 1);
        // same per-level test as k_uniform_check
        int ok = 1;
        for (int k = threadIdx.x; k <= L; k += blockDim.x)
            if (!guess_ok_for_level(gt, L, k, fb.inv, fb.off)) ok = 0;
        fb.uniform = __syncthreads_and(ok);
        return fb.uniform;
    }
    if (F.dtype == EC_U16) {
        if (F.thr && L <= kThrMaxB) {
            uint16_t *s = (uint16_t *)S.thr;
            const uint16_t *gt = (const uint16_t *)F.thr;
            for (int k = threadIdx.x; k < L; k += blockDim.x) s[k] = gt[k];
        }
    } else {
        uint16_t *tab = (uint16_t *)S.thr;
        const uint8_t *gt = (const uint8_t *)F.thr;
        for (int v = threadIdx.x; v < 256; v += blockDim.x) {
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
    }
    __syncthreads();
    return 0;
}

template <typename T>
__device__ IBin<T> make_ibin(const BField &F, const Shared &S)
{
    IBin<T> ib{};
    ib.L = F.L;
    if constexpr (sizeof(T) == 1) {
        ib.table = (const uint16_t *)S.thr;
    } else {
        ib.t = (const T *)F.thr;
        if (F.thr && F.L <= kThrMaxB) ib.t = (const T *)S.thr;
    }
    return ib;
}

template <typename T, bool PER, int DM = 0>
__device__ void item_3d(const BField &F, const BItem &it, const Shared &S, const FBin &fb, int *err)
{
    Ctx<T> c;
    c.p = Params{};
    c.p.field = F.field;
    c.p.D = F.dims[0]; c.p.H = F.dims[1]; c.p.W = F.dims[2];
    c.p.tz = 64;
    c.p.zc0 = 0; c.p.zc1 = (int)F.dims[0];
    c.p.zv0 = 0; c.p.zv1 = (int)F.dims[0];
    c.p.L = F.L;
    c.p.thr = F.thr;
    c.p.hist = F.hist;
    for (int i = 0; i < kMaxDesc; i++) c.p.rows[i] = F.rows[i];
    c.p.nd = F.nd;
    c.p.smem_hist = F.smem_hist;
    c.p.err = err;
    c.p.agg = 0;
    c.fring = nullptr;
    c.raw = S.raw;
    c.kring = S.kring;
    c.bars = nullptr;
    c.abort_flag = S.abort_flag;
    c.sh_hist = F.smem_hist ? S.sh_hist : nullptr;
    c.fb = fb;
    c.ib = make_ibin<T>(F, S);
    c.tr = threadIdx.x >> 4;
    c.tc = threadIdx.x & 15;
    c.bin3 = ~0u;
    c.x0 = it.x0; c.y0 = it.y0; c.z0 = it.z0; c.z1 = it.z1;
    c.interior = c.x0 >= 4 && c.x0 + TXF + 4 <= c.p.W;
    c.skip = c.x0 + TXF > c.p.W || c.y0 + TYF > c.p.H;
    c.base = 0;
    c.parity = 0;
    c.inflight = 0;
    uint32_t win[3][3][5];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++)
#pragma unroll
            for (int e = 0; e < 5; e++) win[a][b][e] = 0;
    const int nsteps = c.z1 - c.z0 + 3;
    if (((uintptr_t)F.field & 15u) == 0) {
        // planes staged with 16-byte cp.async chunks covering each row, KAP planes ahead
        for (int q = 0; q < KAP; q++) copy_plane<T, STG_COVER, NRAWP>(c, c.z0 - 1 + q, c.z0 - 1 + q <= c.z1);
        for (int t = 0; t < nsteps; t += 3) {
            zstep_async<T, PER, 0, DM, 0, STG_COVER>(c, win, t);
            if (t + 1 < nsteps) zstep_async<T, PER, 1, DM, 0, STG_COVER>(c, win, t + 1);
            if (t + 2 < nsteps) zstep_async<T, PER, 2, DM, 0, STG_COVER>(c, win, t + 2);
        }
        cp_async_wait<0>();
    } else {
        for (int t = 0; t < nsteps; t += 3) {
            zstep<T, PER, 0, DM>(c, win, t);
            if (t + 1 < nsteps) zstep<T, PER, 1, DM>(c, win, t + 1);
            if (t + 2 < nsteps) zstep<T, PER, 2, DM>(c, win, t + 2);
        }
    }
}

template <typename T>
__device__ __forceinline__ uint32_t bin2(T v, const FBin &fb, const IBin<T> &ib)
{
    if constexpr (sizeof(T) == 4) return fb.uniform ? fbin_uniform(v, fb) : fbin(v, fb);
    else return ib(v);
}

// One 2D item: a 1024-column strip (x0) over rows [z0, z1), with the fast
// 2D row walk of ec_fast2d.cuh.
template <typename T, bool CONN4>
__device__ void item_2d(const BField &F, const BItem &it, const Shared &S, const FBin &fb)
{
    fast2d::Ctx2<T> c;
    c.p = fast2d::Params{};
    c.p.field = F.field;
    c.p.H = F.dims[1];
    c.p.W = F.dims[2];
    c.p.L = F.L;
    c.p.thr = F.thr;
    c.p.hist = F.hist;
    for (int i = 0; i < kMaxDesc; i++) c.p.rows[i] = F.rows[i];
    c.p.nd = F.nd;
    c.p.smem_hist = F.smem_hist;
    c.p.conn4 = CONN4 ? 1 : 0;
    c.ring = S.kring;
    c.sh_hist = F.smem_hist ? S.sh_hist : nullptr;
    c.fb = fb;
    c.ib = make_ibin<T>(F, S);
    c.x0 = it.x0;
    c.y0 = it.z0;
    c.y1 = it.z1;
    c.interior = c.x0 >= 2 && c.x0 + fast2d::SW + 2 <= c.p.W;
    if (it.y0 > 1) {
        // banded strip: virtual rows 0 .. min(kBandRows, rows) of nb bands
        c.nb = it.y0;
        c.yb0 = it.z0;
        c.y0 = 0;
        c.y1 = min(fast2d::kBandRows, it.z1 - it.z0);
        c.interior = false;
    }
    uint32_t win[3][5];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int e = 0; e < 5; e++) win[a][e] = 0;
    if (((uintptr_t)F.field & 15u) == 0) {
        c.raw = S.raw;   // rows staged with 16-byte cp.async covers, three rows ahead
        if (c.nb > 1) fast2d::walk_item_2d_async<T, CONN4, 0, STG_COVER, true>(c, win);
        else fast2d::walk_item_2d_async<T, CONN4, 0, STG_COVER, false>(c, win);
    } else {
        fast2d::walk_item_2d<T, CONN4, 0>(c, win);
    }
}

// Running sums of one field's histogram into its output (one block).
__device__ void scan_field(const BField &F)
{
    __shared__ long long warp_tot[32];
    const int L = F.L;
    for (int row = 0; row < F.nd; row++) {
        const long long *h = F.hist + (size_t)row * L;
        int64_t *o = F.out + (size_t)row * L;
        const int per = (L + blockDim.x - 1) / blockDim.x;
        const int beg = min((int)threadIdx.x * per, L), end = min(beg + per, L);
        long long s = 0;
        for (int k = beg; k < end; k++) s += ((volatile const long long *)h)[k];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        long long incl = s;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int nw = blockDim.x >> 5;
            long long w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const long long t = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += t;
            }
            if (lane < nw) warp_tot[lane] = w;
        }
        __syncthreads();
        long long run = incl - s + (wid > 0 ? warp_tot[wid - 1] : 0);
        for (int k = beg; k < end; k++) {
            run += ((volatile const long long *)h)[k];
            o[k] = run;
        }
        __syncthreads();
    }
}

// Shared memory of k_batch: [key ring] [abort, item broadcast 16] [hist hist_cap ints]
// [thresholds kThrMaxB words] [raw plane ring (float32 size, 128-byte aligned)].
// Compile-time descriptor rows of a field (0: none), as in the single-field kernel.
__device__ __forceinline__ int batch_dm(const BField &F)
{
    uint32_t desc = 0;
    for (int i = 0; i < kMaxDesc; i++)
        if (F.rows[i] >= 0) desc |= 1u << i;
    return (desc == 1u || desc == 13u || desc == 15u) ? (int)desc : 0;
}

__host__ __device__ constexpr size_t batch_raw_offset(size_t hist_cap)
{
    return ((size_t)NK * KWORDS * 4 + 16 + hist_cap * 4 + (size_t)kThrMaxB * 4 + 127) / 128 * 128;
}
__host__ __device__ constexpr size_t batch_smem_bytes(size_t hist_cap)
{
    return batch_raw_offset(hist_cap) + (size_t)NRAWP * rplane_bytes<float>();
}

__global__ void __launch_bounds__(kThreads, 2)
k_batch(const BField *__restrict__ fields, const BItem *__restrict__ items, int nitems, int *counters, int *err,
        size_t hist_cap)
{
    extern __shared__ __align__(128) unsigned char smem[];
    Shared S;
    S.kring = (uint32_t *)smem;
    S.abort_flag = (volatile int *)(smem + (size_t)NK * KWORDS * 4);
    S.item_bcast = (int *)(smem + (size_t)NK * KWORDS * 4 + 8);
    S.sh_hist = (int *)(smem + (size_t)NK * KWORDS * 4 + 16);
    S.hist_cap = hist_cap;
    S.thr = (unsigned char *)(S.sh_hist + hist_cap);
    S.raw = smem + batch_raw_offset(hist_cap);
    if (threadIdx.x == 0) *S.abort_flag = 0;
    int loaded_f = -1;   // field whose binning tables are in shared memory
    FBin fb{};
    int *next_item = counters;          // counters[0]: item counter; counters[1 + f]: items done per field
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) *S.item_bcast = atomicAdd(next_item, 1);
        __syncthreads();
        const int i = *S.item_bcast;
        if (i >= nitems) break;
        const BItem it = items[i];
        const BField F = fields[it.f];
        // float32 3D items with the common descriptor sets use compile-time
        // rows: their shared histogram is interleaved per level, [L+1][nd]
        const int dm = (F.ndim == 3 && F.dtype == EC_F32 && F.smem_hist) ? batch_dm(F) : 0;
        const int hn = dm ? F.nd * (F.L + 1) : F.nd * F.L;
        if (F.smem_hist)
            for (int k = threadIdx.x; k < hn; k += blockDim.x) S.sh_hist[k] = 0;
        if (it.f != loaded_f) {
            load_binning(F, S, fb);   // ends with a barrier
            loaded_f = it.f;
        } else {
            __syncthreads();
        }
        if (F.ndim == 3) {
            const bool per = F.rows[1] >= 0;
            switch (F.dtype) {
            case EC_F32:
                if (dm == 15) item_3d<float, true, 15>(F, it, S, fb, err);
                else if (dm == 13) item_3d<float, false, 13>(F, it, S, fb, err);
                else if (dm == 1) item_3d<float, false, 1>(F, it, S, fb, err);
                else per ? item_3d<float, true>(F, it, S, fb, err) : item_3d<float, false>(F, it, S, fb, err);
                break;
            case EC_U16: per ? item_3d<uint16_t, true>(F, it, S, fb, err) : item_3d<uint16_t, false>(F, it, S, fb, err); break;
            default: per ? item_3d<uint8_t, true>(F, it, S, fb, err) : item_3d<uint8_t, false>(F, it, S, fb, err); break;
            }
        } else {
            if (F.conn4) {
                switch (F.dtype) {
                case EC_F32: item_2d<float, true>(F, it, S, fb); break;
                case EC_U16: item_2d<uint16_t, true>(F, it, S, fb); break;
                default: item_2d<uint8_t, true>(F, it, S, fb); break;
                }
            } else {
                switch (F.dtype) {
                case EC_F32: item_2d<float, false>(F, it, S, fb); break;
                case EC_U16: item_2d<uint16_t, false>(F, it, S, fb); break;
                default: item_2d<uint8_t, false>(F, it, S, fb); break;
                }
            }
        }
        __syncthreads();
        if (F.smem_hist)
            for (int k = threadIdx.x; k < F.nd * F.L; k += blockDim.x) {
                int v;
                if (dm) {
                    const int r = k / F.L, lv = k - r * F.L;
                    v = S.sh_hist[lv * F.nd + r];
                } else {
                    v = S.sh_hist[k];
                }
                if (v) atomicAdd((unsigned long long *)&F.hist[k], (unsigned long long)(long long)v);
            }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) *S.item_bcast = (atomicAdd(&counters[1 + F.done_idx], 1) == F.nitems - 1);
        __syncthreads();
        if (*S.item_bcast) {
            __threadfence();
            scan_field(F);
        }
    }
}

}  // namespace batch

}  // namespace ec

using namespace ec;
using namespace ec::batch;

namespace {

constexpr int kPlanarBranches = 4;

struct BatchState {
    void *dev = nullptr;
    size_t dev_bytes = 0;
    void *staging = nullptr;   // pinned
    size_t staging_bytes = 0;
    cudaEvent_t staged_free = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t fork = nullptr;                   // capture-time branches of the planar launches (kPlanarBranches)
    cudaEvent_t join[4] = {nullptr, nullptr, nullptr, nullptr};
};

}  // namespace

// Launch plan of one batch: z planes per 3D item, rows per ordinary 2D item,
// blocks per launch (0 = as many as fit on every SM).
struct BatchPlan {
    int tz3 = 64;
    int rows2d = 64;
    int grid = 0;
    int64_t planar_min = int64_t(1) << 21;   // 3D fields of at least this many voxels that the planar
                                             // kernel takes get its own launches (a graph branch)
};

static int batch_run(ec_ctx *ctx, const ec_field_desc *fields, int32_t n, cudaStream_t s, const BatchPlan &plan);

// Mix class of a batch for the autotuner: total cells (factor-4 buckets)
// and share of 3D cells (quarters).
static std::string batch_class_key(ec_ctx *ctx, const ec_field_desc *fields, int32_t n)
{
    double cells = 0, cells3 = 0;
    for (int i = 0; i < n; i++) {
        const ec_field_desc &d = fields[i];
        const double c = d.ndim == 3 ? (double)d.dims[0] * d.dims[1] * d.dims[2] : (double)d.dims[0] * d.dims[1];
        cells += c;
        if (d.ndim == 3) cells3 += c;
    }
    char buf[96];
    snprintf(buf, sizeof buf, "batch_sm%d_c%d_f%d", ctx->num_sms, (int)std::floor(std::log2(cells + 1) / 2),
             (int)std::lround(4.0 * cells3 / std::max(cells, 1.0)));
    return buf;
}

// Time one plan on the batch itself (one warm-up run, then the best of two).
static int time_plan(ec_ctx *ctx, const ec_field_desc *fields, int32_t n, cudaStream_t s, const BatchPlan &p,
                     double &us)
{
    cudaEvent_t e0, e1;
    EC_CUDA(cudaEventCreate(&e0));
    EC_CUDA(cudaEventCreate(&e1));
    us = 1e30;
    int rc = EC_OK;
    for (int rep = 0; rep < 3 && rc == EC_OK; rep++) {
        cudaEventRecord(e0, s);
        rc = batch_run(ctx, fields, n, s, p);
        cudaEventRecord(e1, s);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = EC_ERR_CUDA; break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) us = std::min(us, (double)ms * 1e3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// Autotuner (EC_OPT_AUTOTUNE) for ec_batch: the first batch of a mix class
// times candidate plans on itself by coordinate descent (3D item depth
// 16 / 32 / 64, then 2D item rows 32 / 64 / 128, then one or all resident
// blocks per SM), keeps the fastest per class with the single-field plans
// (and in EC_AUTOTUNE_CACHE when set); later batches of the class use it.
// Each candidate runs the whole batch, so the outputs end up written by the
// last run as usual.
// Every plan computes the same curves.
static int tuned_batch_plan(ec_ctx *ctx, const ec_field_desc *fields, int32_t n, cudaStream_t s, BatchPlan &plan)
{
    const std::string key = batch_class_key(ctx, fields, n);
    int v[3];
    if (tune_lookup(ctx, key, v)) {
        plan.tz3 = v[0];
        plan.grid = v[1];
        plan.rows2d = v[2];
        return EC_OK;
    }
    BatchPlan best = plan;
    double best_us = 1e30;
    auto consider = [&](BatchPlan p) -> int {
        double us = 0;
        const int rc = time_plan(ctx, fields, n, s, p, us);
        if (rc == EC_OK && us < best_us) { best_us = us; best = p; }
        return rc;
    };
    int rc = EC_OK;
    for (int tz : {64, 32, 16}) {
        BatchPlan p = best;
        p.tz3 = tz;
        if ((rc = consider(p))) return rc;
    }
    for (int rows : {32, 128}) {
        BatchPlan p = best;
        p.rows2d = rows;
        if ((rc = consider(p))) return rc;
    }
    {
        BatchPlan p = best;
        p.grid = ctx->num_sms;
        if ((rc = consider(p))) return rc;
    }
    plan = best;
    const int w[3] = {best.tz3, best.grid, best.rows2d};
    tune_store(ctx, key, w, best_us);
    return EC_OK;
}

extern "C" int ec_batch_tuned_plan(ec_ctx *ctx, const ec_field_desc *fields, int32_t n, int32_t out[3])
{
    clear_error();
    if (!ctx || !fields || n < 1 || !out) { set_error("bad arguments"); return EC_ERR_ARG; }
    std::lock_guard<std::mutex> lock(ctx->mu);
    int v[3];
    if (!tune_lookup(ctx, batch_class_key(ctx, fields, n), v)) {
        set_error("no tuned plan for this mix class yet");
        return EC_ERR_ARG;
    }
    for (int i = 0; i < 3; i++) out[i] = v[i];
    return EC_OK;
}

extern "C" int ec_batch(ec_ctx *ctx, const ec_field_desc *fields, int32_t n, void *stream)
{
    clear_error();
    if (!ctx || (n > 0 && !fields) || n < 0) { set_error("bad batch arguments"); return EC_ERR_ARG; }
    for (int i = 0; i < n; i++) {
        const ec_field_desc &d = fields[i];
        if (d.ndim != 2 && d.ndim != 3) { set_error("field %d: ndim must be 2 or 3", i); return EC_ERR_ARG; }
        const int rc = validate_request(d.ndim, d.field, d.dims, d.dtype, d.thresholds, d.L, d.connectivity,
                                        d.descriptors, d.out);
        if (rc) {
            const std::string msg = ec_last_error();
            set_error("field %d: %s", i, msg.c_str());
            return rc;
        }
    }
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    BatchPlan plan;
    plan.grid = ctx->grid;
    if (ctx->autotune && n > 0) {
        const int rc = tuned_batch_plan(ctx, fields, n, s, plan);
        if (rc) return rc;
    }
    return batch_run(ctx, fields, n, s, plan);
}

static int batch_run(ec_ctx *ctx, const ec_field_desc *fields, int32_t n, cudaStream_t s, const BatchPlan &plan)
{
    // ---- host tables: fields (largest first for scheduling) and items
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    auto vox = [&](int i) {
        const ec_field_desc &d = fields[i];
        return d.ndim == 3 ? d.dims[0] * d.dims[1] * d.dims[2] : d.dims[0] * d.dims[1];
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return vox(a) > vox(b); });
    std::vector<BField> bf;
    std::vector<BItem> items;
    std::vector<int> separate;   // 3D fields with more levels than 16-bit comparison lanes hold, or 6-connected
    std::vector<int> planar;     // large 3D fields the planar kernel takes: own launches, a graph branch
    size_t hist_entries = 0, max_smem_entries = 0;
    for (int oi = 0; oi < n; oi++) {
        const ec_field_desc &d = fields[order[oi]];
        if (d.L == 0) continue;
        if (d.ndim == 3 && (d.L > kMaxFastL3 || d.connectivity == 6)) {
            separate.push_back(order[oi]);
            continue;
        }
        if (d.ndim == 3 && vox(order[oi]) >= plan.planar_min &&
            planar_3d_supported(d.field, d.dims, d.dtype, d.thresholds, d.L, d.descriptors)) {
            planar.push_back(order[oi]);
            continue;
        }
        BField F{};
        F.field = d.field;
        F.ndim = d.ndim;
        F.dtype = d.dtype;
        F.L = d.L;
        F.thr = d.thresholds;
        F.out = d.out;
        F.conn4 = d.connectivity == 4;
        const RowMap rm = row_map(d.descriptors);
        F.nd = rm.nd;
        for (int k = 0; k < kMaxDesc; k++) F.rows[k] = rm.row[k];
        F.smem_hist = use_smem_hist(rm.nd, d.L) ? 1 : 0;
        if (F.smem_hist) max_smem_entries = std::max(max_smem_entries, (size_t)rm.nd * ((size_t)d.L + 1));
        F.hist = (long long *)(uintptr_t)hist_entries;   // offset, fixed up below
        hist_entries += (size_t)rm.nd * d.L;
        F.done_idx = (int)bf.size();
        const int f = (int)bf.size();
        int cnt = 0;
        if (d.ndim == 3) {
            F.dims[0] = d.dims[0]; F.dims[1] = d.dims[1]; F.dims[2] = d.dims[2];
            for (int64_t z = 0; z < d.dims[0]; z += plan.tz3)
                for (int64_t y = 0; y < d.dims[1]; y += TYF)
                    for (int64_t x = 0; x < d.dims[2]; x += TXF) {
                        items.push_back(BItem{f, (int)x, (int)y, (int)z,
                                              (int)std::min<int64_t>(z + plan.tz3, d.dims[0])});
                        cnt++;
                    }
        } else {
            F.dims[0] = 1; F.dims[1] = d.dims[0]; F.dims[2] = d.dims[1];
            // narrow fields (cover staging) share a strip between 2 or 4 row bands
            int nb = 1;
            if (((uintptr_t)d.field & 15u) == 0) {
                const int w4 = d.dtype == EC_F32 ? fast2d::band_max_width<float>(4)
                               : d.dtype == EC_U16 ? fast2d::band_max_width<uint16_t>(4)
                                                   : fast2d::band_max_width<uint8_t>(4);
                const int w2 = d.dtype == EC_F32 ? fast2d::band_max_width<float>(2)
                               : d.dtype == EC_U16 ? fast2d::band_max_width<uint16_t>(2)
                                                   : fast2d::band_max_width<uint8_t>(2);
                // 1, 2 or 4 bands (segments of 1024, 512 or 256 pixels); a band
                // past the field's last row is all invalid pixels
                const int64_t bands = (d.dims[0] + fast2d::kBandRows - 1) / fast2d::kBandRows;
                if (d.dims[1] <= w4 && bands >= 3) nb = 4;
                else if (d.dims[1] <= w2 && bands >= 2) nb = 2;
            }
            if (nb > 1) {
                const int64_t rows = (int64_t)nb * fast2d::kBandRows;
                for (int64_t y = 0; y < d.dims[0]; y += rows) {
                    items.push_back(BItem{f, 0, nb, (int)y, (int)std::min<int64_t>(y + rows, d.dims[0])});
                    cnt++;
                }
            } else {
                for (int64_t y = 0; y < d.dims[0]; y += plan.rows2d)
                    for (int64_t x = 0; x < d.dims[1]; x += fast2d::SW) {
                        items.push_back(BItem{f, (int)x, 0, (int)y,
                                              (int)std::min<int64_t>(y + plan.rows2d, d.dims[0])});
                        cnt++;
                    }
            }
        }
        F.nitems = cnt;
        bf.push_back(F);
    }
    for (int i : separate) {
        // one ordinary launch sequence per such field, on the batch's stream
        const ec_field_desc &d = fields[i];
        int rc = ensure_scratch(ctx, curve_scratch_bytes(d.descriptors, d.L));
        if (rc) return rc;
        CurvePlan cp;
        cp.algo = ALGO_VOXEL;
        cp.num_sms = ctx->num_sms;
        rc = enqueue_curve(cp, 3, d.field, d.dims, d.dtype, d.thresholds, d.L, d.connectivity, d.descriptors, d.out,
                           ctx->ws, s);
        if (rc) return rc;
    }
    // the planar fields' launch sequences on up to kPlanarBranches parallel
    // branches (fields, largest first, to the branch with the fewest voxels
    // so far), each with its own part of the context's scratch (sized first:
    // none is allocated while a graph is captured) and half the GPU's blocks
    // per launch, so that two fields share the GPU with deeper work items
    const int nbr = (int)std::min<size_t>(kPlanarBranches, planar.size());
    std::vector<std::vector<int>> branch(nbr);
    {
        std::vector<int64_t> load(nbr, 0);
        for (int i : planar) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            branch[k].push_back(i);
            load[k] += vox(i);
        }
    }
    size_t planar_scratch = 0;
    for (int i : planar)
        planar_scratch = std::max(planar_scratch, curve_scratch_bytes(fields[i].descriptors, fields[i].L));
    planar_scratch = (planar_scratch + 255) & ~(size_t)255;
    if (!planar.empty()) {
        const int rc = ensure_scratch(ctx, (size_t)nbr * planar_scratch);
        if (rc) return rc;
    }
    auto enqueue_branch = [&](int k, cudaStream_t st) -> int {
        for (int i : branch[k]) {
            const ec_field_desc &d = fields[i];
            CurvePlan cp;
            cp.algo = ALGO_PLANAR;
            cp.num_sms = ctx->num_sms;
            cp.grid = nbr > 1 ? ctx->num_sms : 0;
            const int rc = enqueue_curve(cp, 3, d.field, d.dims, d.dtype, d.thresholds, d.L, d.connectivity,
                                         d.descriptors, d.out, (char *)ctx->ws + (size_t)k * planar_scratch, st);
            if (rc) return rc;
        }
        return EC_OK;
    };
    if (bf.empty() && planar.empty()) return EC_OK;
    if (items.size() > (size_t)INT32_MAX) { set_error("batch too large"); return EC_ERR_UNSUPPORTED; }

    // ---- device layout: [flags 256][fields][items][counters][hist]
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t fb_bytes = al(bf.size() * sizeof(BField)), it_bytes = al(items.size() * sizeof(BItem));
    const size_t ct_bytes = al((bf.size() + 1) * sizeof(int)), hs_bytes = hist_entries * sizeof(long long);
    const size_t total = 256 + fb_bytes + it_bytes + ct_bytes + hs_bytes;
    if (!ctx->batch_state) ctx->batch_state = new BatchState();
    BatchState &st = *(BatchState *)ctx->batch_state;
    if (st.staged_free) EC_CUDA(cudaEventSynchronize(st.staged_free));   // previous batch done with staging
    if (st.dev_bytes < total) {
        if (st.dev) { EC_CUDA(cudaDeviceSynchronize()); cudaFree(st.dev); st.dev = nullptr; }
        if (st.exec) { cudaGraphExecDestroy(st.exec); st.exec = nullptr; }
        const size_t want = std::max(total, (size_t)4 << 20);
        if (cudaMalloc(&st.dev, want) != cudaSuccess) { cudaGetLastError(); set_error("batch scratch allocation failed"); return EC_ERR_OOM; }
        st.dev_bytes = want;
    }
    const size_t table_bytes = fb_bytes + it_bytes;
    if (st.staging_bytes < table_bytes) {
        if (st.staging) cudaFreeHost(st.staging);
        if (st.exec) { cudaGraphExecDestroy(st.exec); st.exec = nullptr; }
        const size_t want = std::max(table_bytes, (size_t)1 << 20);
        if (cudaMallocHost(&st.staging, want) != cudaSuccess) { cudaGetLastError(); set_error("batch staging allocation failed"); return EC_ERR_OOM; }
        st.staging_bytes = want;
    }
    if (!st.staged_free) EC_CUDA(cudaEventCreateWithFlags(&st.staged_free, cudaEventDisableTiming));
    if (!st.fork) EC_CUDA(cudaEventCreateWithFlags(&st.fork, cudaEventDisableTiming));
    for (int k = 0; k < kPlanarBranches; k++)
        if (!st.join[k]) EC_CUDA(cudaEventCreateWithFlags(&st.join[k], cudaEventDisableTiming));
    char *base = (char *)st.dev;
    int *flags = (int *)base;
    BField *d_fields = (BField *)(base + 256);
    BItem *d_items = (BItem *)(base + 256 + fb_bytes);
    int *d_counters = (int *)(base + 256 + fb_bytes + it_bytes);
    long long *d_hist = (long long *)(base + 256 + fb_bytes + it_bytes + ct_bytes);
    for (auto &F : bf) F.hist = d_hist + (size_t)(uintptr_t)F.hist;
    if (!bf.empty()) memcpy(st.staging, bf.data(), bf.size() * sizeof(BField));
    if (!items.empty()) memcpy((char *)st.staging + fb_bytes, items.data(), items.size() * sizeof(BItem));

    // ---- launch configuration
    const size_t hist_cap = std::max<size_t>(max_smem_entries, 1);
    const size_t smem = batch_smem_bytes(hist_cap);
    int occ = 0;
    if (const int orc = kernel_occupancy((const void *)k_batch, kThreads, smem, &occ)) return orc;
    if (occ < 1) { set_error("batch kernel does not fit (%zu B shared)", smem); return EC_ERR_UNSUPPORTED; }
    int grid = plan.grid > 0 ? std::min(plan.grid, ctx->num_sms * occ) : ctx->num_sms * occ;
    grid = std::min<int>(grid, (int)items.size());

    // ---- capture the sequence into a graph; update the cached executable if possible
    // the planar fields run on further branches of the same graph, beside
    // the persistent kernel
    cudaStream_t cap = nullptr, capb[kPlanarBranches] = {};
    EC_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    for (int k = 0; k < nbr; k++)
        if (cudaStreamCreateWithFlags(&capb[k], cudaStreamNonBlocking) != cudaSuccess) {
            for (int j = 0; j < k; j++) cudaStreamDestroy(capb[j]);
            cudaStreamDestroy(cap);
            return cuda_fail(cudaGetLastError(), "batch stream creation");
        }
    cudaGraph_t graph = nullptr;
    int prc = EC_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (nbr > 0) cudaEventRecord(st.fork, cap);
        for (int k = 0; k < nbr; k++) {
            cudaStreamWaitEvent(capb[k], st.fork, 0);
            if (!prc) prc = enqueue_branch(k, capb[k]);
            cudaEventRecord(st.join[k], capb[k]);
        }
        if (!items.empty()) {
            cudaMemcpyAsync(d_fields, st.staging, table_bytes, cudaMemcpyHostToDevice, cap);
            cudaMemsetAsync(flags, 0, 256, cap);
            cudaMemsetAsync(d_counters, 0, ct_bytes + hs_bytes, cap);
            k_batch<<<grid, kThreads, smem, cap>>>(d_fields, d_items, (int)items.size(), d_counters, flags,
                                                   hist_cap);
        }
        for (int k = 0; k < nbr; k++) cudaStreamWaitEvent(cap, st.join[k], 0);
        e = cudaStreamEndCapture(cap, &graph);
    }
    cudaStreamDestroy(cap);
    for (int k = 0; k < nbr; k++) cudaStreamDestroy(capb[k]);
    if (prc) { if (graph) cudaGraphDestroy(graph); return prc; }
    if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "batch graph capture"); }
    bool updated = false;
    if (st.exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(st.exec, graph, &info) == cudaSuccess) updated = true;
        else {
            cudaGetLastError();
            cudaGraphExecDestroy(st.exec);
            st.exec = nullptr;
        }
    }
    if (!updated) {
        e = cudaGraphInstantiate(&st.exec, graph, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(graph); st.exec = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    }
    cudaGraphDestroy(graph);
    if (ctx->profile && prof_begin(ctx, s)) return EC_ERR_CUDA;
    EC_CUDA(cudaGraphLaunch(st.exec, s));
    if (ctx->profile && prof_end(ctx, s)) return EC_ERR_CUDA;
    EC_CUDA(cudaEventRecord(st.staged_free, s));
    return EC_OK;
}

// Release the batch state of a context (called by ec_ctx_destroy).
void ec::batch_release(ec_ctx *ctx)
{
    BatchState *st = (BatchState *)ctx->batch_state;
    if (!st) return;
    if (st->exec) cudaGraphExecDestroy(st->exec);
    if (st->staged_free) cudaEventDestroy(st->staged_free);
    if (st->fork) cudaEventDestroy(st->fork);
    for (int k = 0; k < 4; k++)
        if (st->join[k]) cudaEventDestroy(st->join[k]);
    if (st->dev) cudaFree(st->dev);
    if (st->staging) cudaFreeHost(st->staging);
    delete st;
    ctx->batch_state = nullptr;
}

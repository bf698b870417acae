// ec_typemap.cu -- the vertex-contribution type map and weighted curves.
//
// The paper's output is not only the EC curve but the number of vertices of
// each contribution type at each level (Sec. 2, Algorithm 1 and Table 1;
// Sec. 2.2, Algorithm 3 and Table 2); any descriptor that is a weighted sum
// of vertex contributions, for any connectivity, follows from that map by
// changing the weights (Sec. 4).  ec_type_map computes the map on the
// device (histogram of type transitions per level, running sums, empty type
// from the number of vertices); ec_apply_weights turns a map into curves.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "ec_internal.h"
#include "ec_rules.h"

using namespace ec;

namespace {

constexpr size_t kFlagBytes = 256;
constexpr int kMaxWeightRows = 16;

// Running sum over levels of one type's transition row (block = type 1..T-1).
__global__ void __launch_bounds__(1024) k_type_scan(const long long *__restrict__ hist, int L,
                                                    int64_t *__restrict__ counts)
{
    __shared__ long long warp_tot[32];
    const int row = blockIdx.x;   // type row + 1
    const long long *h = hist + (size_t)row * L;
    int64_t *o = counts + (size_t)(row + 1) * L;
    const int per = (L + blockDim.x - 1) / blockDim.x;
    const int beg = min((int)threadIdx.x * per, L), end = min(beg + per, L);
    long long s = 0;
    for (int k = beg; k < end; k++) s += h[k];
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
        run += h[k];
        o[k] = run;
    }
}

// Empty type (row 0): the vertices of no other type.
__global__ void k_type_empty(int64_t *__restrict__ counts, int nt, int L, long long nvert)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L) return;
    long long s = 0;
    for (int t = 1; t < nt; t++) s += counts[(size_t)t * L + k];
    counts[k] = nvert - s;
}

struct Weights {
    int32_t w[kMaxWeightRows][kTypes3];
    int32_t scale[kMaxWeightRows];
};

// out[d][k] = sum_t w[d][t] counts[t][k] / scale[d], accumulated in 128 bits;
// a sum that leaves int64 or is not a multiple of its scale poisons its
// entry with INT64_MIN and sets flag bit 0.
__global__ void k_apply_weights(const int64_t *__restrict__ counts, int nt, int L, Weights W,
                                int64_t *__restrict__ out, int *flag)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
    if (k >= L) return;
    __int128 acc = 0;
    for (int t = 0; t < nt; t++) acc += (__int128)W.w[d][t] * (__int128)counts[(size_t)t * L + k];
    const __int128 lo = (__int128)INT64_MIN, hi = (__int128)INT64_MAX;
    int64_t r = INT64_MIN;
    bool ok = acc >= lo && acc <= hi;
    if (ok) {
        const long long a = (long long)acc, sc = W.scale[d];
        const long long q = a / sc;
        ok = q * sc == a;
        if (ok) r = q;
    }
    if (!ok) atomicOr(flag, 1);
    out[(size_t)d * L + k] = r;
}

}  // namespace

extern "C" {

int ec_type_table(int32_t ndim, int32_t *out)
{
    clear_error();
    if (!out) { set_error("out is NULL"); return EC_ERR_ARG; }
    if (ndim == 2) {
        constexpr TypeTable2D t = make_type_table_2d();
        for (int m = 0; m < 16; m++) out[m] = t.t[m];
        return EC_OK;
    }
    if (ndim == 3) {
        constexpr TypeTable3D t = make_type_table_3d();
        for (int m = 0; m < 256; m++) out[m] = t.t[m];
        return EC_OK;
    }
    set_error("ndim must be 2 or 3 (got %d)", ndim);
    return EC_ERR_ARG;
}

int ec_type_map(ec_ctx *ctx, int32_t ndim, const void *field_dev, const int64_t *dims, int dtype,
                const void *thresholds_dev, int32_t L, int64_t *counts_dev, void *stream)
{
    clear_error();
    if (!ctx) { set_error("ctx is NULL"); return EC_ERR_ARG; }
    if (ndim != 2 && ndim != 3) { set_error("ndim must be 2 or 3 (got %d)", ndim); return EC_ERR_ARG; }
    int rc = validate_request(ndim, field_dev, dims, dtype, thresholds_dev, L, ndim == 2 ? 8 : 26, EC_DESC_EC,
                              counts_dev);
    if (rc) return rc;
    if (L == 0) return EC_OK;
    const int nt = ndim == 2 ? kTypes2 : kTypes3;
    long long nvert = 1;
    for (int i = 0; i < ndim; i++) {
        if (dims[i] + 1 > (int64_t)1 << 40 || nvert > ((long long)1 << 62) / (dims[i] + 1)) {
            set_error("field too large");
            return EC_ERR_ARG;
        }
        nvert *= dims[i] + 1;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    const size_t hist_bytes = (size_t)(nt - 1) * L * sizeof(long long);
    rc = ensure_scratch(ctx, kFlagBytes + hist_bytes);
    if (rc) return rc;
    int *flags = (int *)ctx->ws;
    long long *hist = (long long *)((char *)ctx->ws + kFlagBytes);
    EC_CUDA(cudaMemsetAsync(ctx->ws, 0, kFlagBytes + hist_bytes, s));
    if (ctx->validate && thresholds_dev) {
        rc = launch_check_sorted(thresholds_dev, dtype, L, flags + 1, s);
        if (rc) return rc;
        EC_CUDA(cudaMemcpyAsync(ctx->host_flag, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        EC_CUDA(cudaStreamSynchronize(s));
        if (*ctx->host_flag) { set_error("thresholds are not non-decreasing"); return EC_ERR_ARG; }
    }
    BinArgs ba{L, dtype, thresholds_dev};
    if (ctx->profile && (rc = prof_begin(ctx, s))) return rc;
    rc = launch_type_map(ndim, field_dev, dims, ba, hist, ctx->tile_z, ctx->grid, ctx->num_sms, s);
    if (rc) return rc;
    if (ctx->profile && (rc = prof_end(ctx, s))) return rc;
    k_type_scan<<<nt - 1, 1024, 0, s>>>(hist, L, counts_dev);
    EC_CUDA(cudaGetLastError());
    k_type_empty<<<(L + 255) / 256, 256, 0, s>>>(counts_dev, nt, L, nvert);
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

int ec_apply_weights(ec_ctx *ctx, int32_t ntypes, const int64_t *counts_dev, int32_t L, int32_t nd,
                     const int32_t *weights_host, const int32_t *scales_host, int64_t *out_dev, void *stream)
{
    clear_error();
    if (!ctx) { set_error("ctx is NULL"); return EC_ERR_ARG; }
    if (ntypes < 1 || ntypes > kTypes3) { set_error("ntypes must be in [1, %d] (got %d)", kTypes3, ntypes); return EC_ERR_ARG; }
    if (nd < 1 || nd > kMaxWeightRows) { set_error("nd must be in [1, %d] (got %d)", kMaxWeightRows, nd); return EC_ERR_ARG; }
    if (L < 0 || L > 65535) { set_error("L = %d outside [0, 65535]", L); return EC_ERR_ARG; }
    if (!weights_host) { set_error("weights is NULL"); return EC_ERR_ARG; }
    if (L == 0) return EC_OK;
    if (!counts_dev || !out_dev) { set_error("counts or out is NULL"); return EC_ERR_ARG; }
    Weights W;
    memset(&W, 0, sizeof W);
    for (int d = 0; d < nd; d++) {
        for (int t = 0; t < ntypes; t++) W.w[d][t] = weights_host[(size_t)d * ntypes + t];
        W.scale[d] = scales_host ? scales_host[d] : 1;
        if (W.scale[d] < 1) { set_error("scale[%d] = %d < 1", d, W.scale[d]); return EC_ERR_ARG; }
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    int rc = ensure_scratch(ctx, kFlagBytes);
    if (rc) return rc;
    int *flags = (int *)ctx->ws;
    EC_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), s));
    dim3 grid((unsigned)((L + 255) / 256), (unsigned)nd);
    k_apply_weights<<<grid, 256, 0, s>>>(counts_dev, ntypes, L, W, out_dev, flags);
    EC_CUDA(cudaGetLastError());
    if (ctx->validate) {
        EC_CUDA(cudaMemcpyAsync(ctx->host_flag, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        EC_CUDA(cudaStreamSynchronize(s));
        if (*ctx->host_flag) {
            set_error("a weighted sum is not a multiple of its scale or leaves int64");
            return EC_ERR_ARG;
        }
    }
    return EC_OK;
}

}  // extern "C"

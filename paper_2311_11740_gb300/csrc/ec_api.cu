// ec_api.cu -- C ABI: contexts, argument validation, curve requests.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <thread>
#include <vector>

#include "ec_internal.h"
#include "ec_rules.h"
#include "ec_types.h"
#include "ec_slice.h"
#include "ec_swar.h"

namespace ec {

static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}
void clear_error() { g_err.clear(); }
int cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return EC_ERR_CUDA;
}

const Table2D &host_table_2d();
const Table3D &host_table_3d();

}  // namespace ec

using namespace ec;

namespace {

constexpr size_t kFlagBytes = 256;

// The planar per-voxel form (ec_slice.h) on random small grids with many tied
// levels, walked the way the kernels walk a column (one quad of four voxels
// along x, or two stacked quads; start state from the plane below the first,
// planes outside the field never active), summed per level and compared with the vertex tables
// summed over every vertex of the grid (8 EC, 2 perimeter, 4 area, 8 volume).
// Returns the number of mismatching (trial, level, descriptor) entries.
int64_t selfcheck_planar(const Table3D &t3)
{
    uint64_t rs = 0xD1B54A32D192ED03ull;
    auto rnd = [&rs]() {
        rs ^= rs << 13; rs ^= rs >> 7; rs ^= rs << 17;
        return rs;
    };
    int64_t bad = 0;
    for (int trial = 0; trial < 3000; trial++) {
        const int D = 1 + (int)(rnd() % 5), H = 1 + (int)(rnd() % 5), W = 1 + (int)(rnd() % 10);
        const int L = trial % 4 == 0 ? 2 : (trial % 4 == 1 ? 4 : (trial % 4 == 2 ? 9 : 300));
        // level of every voxel; L (never active) outside the field
        std::vector<int> lev((size_t)D * H * W);
        for (auto &v : lev) v = (int)(rnd() % (uint64_t)(L + 1));
        auto key = [&](int z, int y, int x) -> uint32_t {
            if (z < 0 || z >= D || y < 0 || y >= H || x < 0 || x >= W) return (uint32_t)L;
            return (uint32_t)lev[((size_t)z * H + y) * W + x];
        };
        auto pair = [&](int z, int y, int x) { return key(z, y, x) | (key(z, y, x + 1) << 16); };
        auto row5 = [&](int z, int y, int x) {
            return Row5{pair(z, y, x - 1), pair(z, y, x), pair(z, y, x + 1), pair(z, y, x + 2), pair(z, y, x + 3)};
        };
        std::vector<int64_t> h((size_t)(L + 1) * 4, 0);
        std::vector<int64_t> h2((size_t)(L + 1) * 4, 0);
        // the two-row form (stacked quads, area as free faces)
        for (int y = 0; y < H; y += 2)
            for (int x = 0; x < W; x += 4) {
                Row5 P[4], Q[4];
                for (int r = 0; r < 4; r++) {
                    P[r] = row5(-1, y - 1 + r, x);
                    Q[r] = row5(0, y - 1 + r, x);
                }
                SliceState sa{}, sb{};
                slice_pair_begin<true>(P, Q, sa, sb);
                for (int z = 0; z < D; z++) {
                    for (int r = 0; r < 4; r++) {
                        P[r] = Q[r];
                        Q[r] = row5(z + 1, y - 1 + r, x);
                    }
                    SliceOut oa, ob;
                    slice_pair<AREA_FREE_FACES, true>(P, Q, sa, sb, oa, ob);
                    for (int half = 0; half < 2; half++) {
                        const SliceOut &o = half ? ob : oa;
                        for (int v = 0; v < 4; v++) {
                            const uint32_t k = key(z, y + half, x + v);
                            const int sh = 8 * v;
                            h2[k * 4 + 0] += (int8_t)(uint8_t)(o.ec >> sh);
                            h2[k * 4 + 1] += (int8_t)(uint8_t)(o.per >> sh);
                            h2[k * 4 + 2] += 2 * (int)((o.area >> sh) & 0xFFu) - 6;
                            h2[k * 4 + 3] += 1;
                        }
                    }
                }
            }
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x += 4) {
                Row5 P[3], Q[3];
                for (int dy = 0; dy < 3; dy++) {
                    P[dy] = row5(-1, y - 1 + dy, x);
                    Q[dy] = row5(0, y - 1 + dy, x);
                }
                SliceState st{};
                slice_begin<true>(P, Q, st);
                for (int z = 0; z < D; z++) {
                    for (int dy = 0; dy < 3; dy++) {
                        P[dy] = Q[dy];
                        Q[dy] = row5(z + 1, y - 1 + dy, x);
                    }
                    const SliceOut o = slice_quad<true, true>(P, Q, st);
                    for (int v = 0; v < 4; v++) {
                        const uint32_t k = key(z, y, x + v);
                        const int sh = 8 * v;
                        h[k * 4 + 0] += (int8_t)(uint8_t)(o.ec >> sh);
                        h[k * 4 + 1] += (int8_t)(uint8_t)(o.per >> sh);
                        h[k * 4 + 2] += (int8_t)(uint8_t)(o.area >> sh);
                        h[k * 4 + 3] += 1;
                    }
                }
            }
        int64_t run[4] = {0, 0, 0, 0}, run2[4] = {0, 0, 0, 0};
        for (int k = 0; k < L; k++) {
            int64_t want[4] = {0, 0, 0, 0};
            for (int z = 0; z <= D; z++)
                for (int y = 0; y <= H; y++)
                    for (int x = 0; x <= W; x++) {
                        unsigned m = 0;
                        for (unsigned b = 0; b < 8; b++)
                            if ((int)key(z - 1 + (int)(b >> 2), y - 1 + (int)((b >> 1) & 1), x - 1 + (int)(b & 1)) <= k)
                                m |= 1u << b;
                        for (int d = 0; d < 4; d++) want[d] += t3.v[m][d];
                    }
            const int scale[4] = {8, 2, 4, 8};
            for (int d = 0; d < 4; d++) {
                run[d] += h[(size_t)k * 4 + d];
                run2[d] += h2[(size_t)k * 4 + d];
                bad += run[d] * scale[d] != want[d];
                bad += run2[d] * scale[d] != want[d];
            }
        }
    }
    return bad;
}

}  // namespace

int ec::kernel_occupancy(const void *kern, int threads, size_t smem, int *occ)
{
    int dev = 0;
    EC_CUDA(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    static std::map<std::pair<int, const void *>, size_t> limit;   // dynamic shared bytes allowed so far
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, kern, threads, smem);
    const auto it = cache.find(key);
    if (it != cache.end()) {
        *occ = it->second;
        return EC_OK;
    }
    size_t &lim = limit[std::make_pair(dev, kern)];
    if (smem > lim) {
        EC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        lim = smem;
    }
    EC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, threads, smem));
    cache[key] = *occ;
    return EC_OK;
}

int ec::ensure_scratch(ec_ctx *ctx, size_t bytes)
{
    if (ctx->ws_bytes >= bytes) return EC_OK;
    if (ctx->ws) {
        EC_CUDA(cudaDeviceSynchronize());   // the old buffer may still be in use by queued work
        EC_CUDA(cudaFree(ctx->ws));
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cannot allocate %zu bytes of scratch: %s", want, cudaGetErrorString(e));
        return EC_ERR_OOM;
    }
    ctx->ws_bytes = want;
    return EC_OK;
}

int ec::validate_request(int ndim, const void *field, const int64_t *dims, int dtype, const void *thr, int32_t L,
                    int connectivity, uint32_t descriptors, const int64_t *out)
{
    if (dtype != EC_U8 && dtype != EC_U16 && dtype != EC_F32) {
        set_error("unknown dtype %d", dtype);
        return EC_ERR_DTYPE;
    }
    if (dtype == EC_F32 && !thr && L > 0) {
        set_error("float32 fields need thresholds");
        return EC_ERR_DTYPE;
    }
    if (!dims) { set_error("dims is NULL"); return EC_ERR_ARG; }
    for (int i = 0; i < ndim; i++)
        if (dims[i] < 1) { set_error("dims[%d] = %lld < 1", i, (long long)dims[i]); return EC_ERR_ARG; }
    if (L < 0 || L > 65535) { set_error("L = %d outside [0, 65535]", L); return EC_ERR_ARG; }
    const uint32_t allowed = ndim == 2 ? 0x7u : 0xFu;
    if (descriptors == 0 || (descriptors & ~allowed)) {
        set_error("descriptors 0x%x not valid for %dD", descriptors, ndim);
        return EC_ERR_ARG;
    }
    if (ndim == 2 && connectivity != 8 && connectivity != 4) {
        set_error("2D connectivity must be 8 or 4 (got %d)", connectivity);
        return EC_ERR_ARG;
    }
    if (ndim == 3 && connectivity != 26 && connectivity != 6) {
        set_error("3D connectivity must be 26 or 6 (got %d)", connectivity);
        return EC_ERR_ARG;
    }
    if (L > 0 && (!field || !out)) { set_error("field or out is NULL"); return EC_ERR_ARG; }
    return EC_OK;
}

namespace {

int run_curve(ec_ctx *ctx, int ndim, const void *field, const int64_t *dims, int dtype, const void *thr,
              int32_t L, int connectivity, uint32_t descriptors, int64_t *out, cudaStream_t s)
{
    int rc = validate_request(ndim, field, dims, dtype, thr, L, connectivity, descriptors, out);
    if (rc) return rc;
    if (L == 0) return EC_OK;
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    rc = ensure_scratch(ctx, curve_scratch_bytes(descriptors, L));
    if (rc) return rc;
    int *flags = (int *)ctx->ws;
    if (ctx->validate && thr) {
        EC_CUDA(cudaMemsetAsync(flags, 0, kFlagBytes, s));
        rc = launch_check_sorted(thr, dtype, L, flags + 1, s);
        if (rc) return rc;
        EC_CUDA(cudaMemcpyAsync(ctx->host_flag, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        EC_CUDA(cudaStreamSynchronize(s));
        if (*ctx->host_flag) { set_error("thresholds are not non-decreasing"); return EC_ERR_ARG; }
    }
    CurvePlan plan;
    plan.algo = ctx->algo;
    plan.hist_schedule = ctx->hist_schedule;
    plan.tile_z = ctx->tile_z;
    plan.grid = ctx->grid;
    plan.num_sms = ctx->num_sms;
    plan.prof = ctx->profile ? ctx : nullptr;
    plan.test_give_up = ctx->test_give_up;
    if (ctx->autotune && plan.algo != ALGO_VERTEX) {
        rc = tuned_plan(ctx, ndim, field, dims, dtype, thr, L, connectivity, descriptors, out, s, plan);
        if (rc) return rc;
    }
    rc = enqueue_curve(plan, ndim, field, dims, dtype, thr, L, connectivity, descriptors, out, ctx->ws, s);
    if (rc) return rc;
    if (ctx->validate) {
        EC_CUDA(cudaMemcpyAsync(ctx->host_flag, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        EC_CUDA(cudaStreamSynchronize(s));
        if (*ctx->host_flag & 4) { set_error("a bounded device wait gave up"); return EC_ERR_TIMEOUT; }
        if (*ctx->host_flag) { set_error("histogram did not divide by its scale"); return EC_ERR_OVERFLOW; }
    }
    return EC_OK;
}

}  // namespace

size_t ec::curve_scratch_bytes(uint32_t descriptors, int32_t L)
{
    return kFlagBytes + (size_t)row_map(descriptors).nd * (size_t)(L > 0 ? L : 0) * sizeof(long long);
}

// Stream-ordered launch sequence of one validated curve request on the given
// scratch (curve_scratch_bytes): reset, histogram kernel(s), scan.
int ec::enqueue_curve(const CurvePlan &plan, int ndim, const void *field, const int64_t *dims, int dtype,
                      const void *thr, int32_t L, int connectivity, uint32_t descriptors, int64_t *out,
                      void *scratch, cudaStream_t s)
{
    const RowMap rows = row_map(descriptors);
    int *flags = (int *)scratch;
    long long *hist = (long long *)((char *)scratch + kFlagBytes);
    EC_CUDA(cudaMemsetAsync(scratch, 0, curve_scratch_bytes(descriptors, L), s));
    const int algo = plan.algo == ALGO_VERTEX ? ALGO_VERTEX : ALGO_VOXEL;
    BinArgs ba{L, dtype, thr};
    HistArgs ha{rows, hist, use_smem_hist(rows.nd, L) ? 1 : 0, plan.hist_schedule};
    ha.planar = plan.algo == ALGO_AUTO || plan.algo == ALGO_PLANAR;
    ha.test_give_up = plan.test_give_up;
    int rc;
    if (plan.prof && (rc = prof_begin(plan.prof, s))) return rc;
    if (ndim == 3) {
        // 6-connectivity runs on the generic kernels (the EC row from the AND
        // counterparts of the covers, or the 6-connected vertex table)
        const int conn6 = connectivity == 6 ? 1 : 0;
        rc = EC_ERR_UNSUPPORTED;
        if (algo == ALGO_VOXEL && !conn6)
            rc = launch_fast_3d(field, dims, ba, ha, plan.tile_z, plan.grid, plan.num_sms, flags, s);
        if (rc == EC_ERR_UNSUPPORTED)
            rc = launch_curve_3d(field, dims, ba, ha, algo, plan.tile_z, plan.grid, plan.num_sms, s, nullptr, conn6);
    } else {
        rc = EC_ERR_UNSUPPORTED;
        if (algo == ALGO_VOXEL)
            rc = launch_fast_2d(field, dims, ba, ha, connectivity, plan.grid, plan.num_sms, flags, s);
        if (rc == EC_ERR_UNSUPPORTED)
            rc = launch_curve_2d(field, dims, ba, ha, connectivity, algo, plan.grid, plan.num_sms, s);
    }
    if (rc) return rc;
    if (plan.prof && (rc = prof_end(plan.prof, s))) return rc;
    int32_t scale[kMaxDesc];
    row_scales(ndim, algo, descriptors, scale);
    return launch_scan(hist, rows.nd, L, scale, out, flags, s);
}

int ec::prof_begin(ec_ctx *ctx, cudaStream_t s)
{
    if (ctx->prof_used + 2 > ctx->prof_events.size()) {
        for (int i = 0; i < 256; i++) {
            cudaEvent_t e;
            EC_CUDA(cudaEventCreate(&e));
            ctx->prof_events.push_back(e);
        }
    }
    EC_CUDA(cudaEventRecord(ctx->prof_events[ctx->prof_used], s));
    return EC_OK;
}

int ec::prof_end(ec_ctx *ctx, cudaStream_t s)
{
    EC_CUDA(cudaEventRecord(ctx->prof_events[ctx->prof_used + 1], s));
    ctx->prof_used += 2;
    return EC_OK;
}

extern "C" {

int ec_ctx_profile_read(ec_ctx *ctx, double *kernel_ms, int64_t *launches)
{
    clear_error();
    if (!ctx || !kernel_ms || !launches) { set_error("NULL argument"); return EC_ERR_ARG; }
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    double tot = 0;
    for (size_t i = 0; i + 1 < ctx->prof_used; i += 2) {
        EC_CUDA(cudaEventSynchronize(ctx->prof_events[i + 1]));
        float ms = 0;
        EC_CUDA(cudaEventElapsedTime(&ms, ctx->prof_events[i], ctx->prof_events[i + 1]));
        tot += ms;
    }
    *kernel_ms = tot;
    *launches = (int64_t)(ctx->prof_used / 2);
    ctx->prof_used = 0;
    return EC_OK;
}


const char *ec_last_error(void) { return g_err.c_str(); }

int ec_ctx_create(ec_ctx **out, int device)
{
    clear_error();
    if (!out) { set_error("ctx is NULL"); return EC_ERR_ARG; }
    int ndev = 0;
    EC_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) { set_error("device %d not present (%d devices)", device, ndev); return EC_ERR_ARG; }
    ec_ctx *ctx = new ec_ctx();
    ctx->device = device;
    DeviceGuard dg(device);
    cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->host_flag, sizeof(int) * 4);
    if (e != cudaSuccess) {
        delete ctx;
        return cuda_fail(e, "ec_ctx_create");
    }
    *out = ctx;
    return EC_OK;
}

int ec_ctx_destroy(ec_ctx *ctx)
{
    clear_error();
    if (!ctx) return EC_OK;
    {
        DeviceGuard dg(ctx->device);
        cudaDeviceSynchronize();
        if (ctx->ws) cudaFree(ctx->ws);
        if (ctx->host_flag) cudaFreeHost(ctx->host_flag);
        for (cudaEvent_t e : ctx->prof_events) cudaEventDestroy(e);
        batch_release(ctx);
        tune_release(ctx);
        stream_release(ctx);
    }
    delete ctx;
    return EC_OK;
}

int ec_ctx_set_option(ec_ctx *ctx, int option, int64_t value)
{
    clear_error();
    if (!ctx) { set_error("ctx is NULL"); return EC_ERR_ARG; }
    switch (option) {
    case EC_OPT_ALGO:
        if (value < 0 || value > 3) { set_error("bad algo %lld", (long long)value); return EC_ERR_ARG; }
        ctx->algo = (int)value;
        return EC_OK;
    case EC_OPT_VALIDATE: ctx->validate = value ? 1 : 0; return EC_OK;
    case EC_OPT_TILE_Z:
        if (value < 0 || value > 4096) { set_error("bad tile_z"); return EC_ERR_ARG; }
        ctx->tile_z = (int)value;
        return EC_OK;
    case EC_OPT_GRID:
        if (value < 0 || value > (1 << 20)) { set_error("bad grid"); return EC_ERR_ARG; }
        ctx->grid = (int)value;
        return EC_OK;
    case EC_OPT_AUTOTUNE: ctx->autotune = value ? 1 : 0; return EC_OK;
    case EC_OPT_HIST_SCHEDULE:
        if (value < 0 || value > 3) { set_error("bad histogram schedule"); return EC_ERR_ARG; }
        ctx->hist_schedule = (int)value;
        return EC_OK;
    case EC_OPT_TEST_GIVE_UP: ctx->test_give_up = value ? 1 : 0; return EC_OK;
    case EC_OPT_PROFILE: {
        std::lock_guard<std::mutex> lock(ctx->mu);
        ctx->profile = value ? 1 : 0;
        ctx->prof_used = 0;
        return EC_OK;
    }
    }
    set_error("unknown option %d", option);
    return EC_ERR_ARG;
}

int ec_curve_2d(ec_ctx *ctx, const void *field_dev, const int64_t dims[2], int dtype, const void *thresholds_dev,
                int32_t L, int connectivity, uint32_t descriptors, int64_t *out_dev, void *stream)
{
    clear_error();
    if (!ctx) { set_error("ctx is NULL"); return EC_ERR_ARG; }
    return run_curve(ctx, 2, field_dev, dims, dtype, thresholds_dev, L, connectivity, descriptors, out_dev,
                     (cudaStream_t)stream);
}

int ec_curve_3d(ec_ctx *ctx, const void *field_dev, const int64_t dims[3], int dtype, const void *thresholds_dev,
                int32_t L, int connectivity, uint32_t descriptors, int64_t *out_dev, void *stream)
{
    clear_error();
    if (!ctx) { set_error("ctx is NULL"); return EC_ERR_ARG; }
    return run_curve(ctx, 3, field_dev, dims, dtype, thresholds_dev, L, connectivity, descriptors, out_dev,
                     (cudaStream_t)stream);
}

size_t ec_workspace_bytes(int dtype, int32_t ndim, const int64_t *dims, int32_t L, uint32_t descriptors)
{
    (void)dtype; (void)ndim; (void)dims;
    return curve_scratch_bytes(descriptors, L);
}

int ec_vertex_table_2d(int32_t *out)
{
    if (!out) return EC_ERR_ARG;
    memcpy(out, host_table_2d().v, sizeof(host_table_2d().v));
    return EC_OK;
}

int ec_vertex_table_3d_ec6(int32_t *out)
{
    static constexpr Table3D6 t6 = make_table_3d_ec6();
    if (!out) return EC_ERR_ARG;
    memcpy(out, t6.v, sizeof(t6.v));
    return EC_OK;
}

int ec_vertex_table_3d(int32_t *out)
{
    if (!out) return EC_ERR_ARG;
    memcpy(out, host_table_3d().v, sizeof(host_table_3d().v));
    return EC_OK;
}

int64_t ec_selfcheck_rules(void)
{
    const Table2D &t2 = host_table_2d();
    const Table3D &t3 = host_table_3d();
    static constexpr Table3D6 t6 = make_table_3d_ec6();
    int64_t bad = 0;
    // 2D: all 2^8 precedence patterns of the 8 neighbours
    for (uint32_t i = 0; i < 256; i++) {
        const uint32_t P = (i & 0xFu) | ((i >> 4) << 5);
        int sum[4] = {0, 0, 0, 0};
        for (int v = 0; v < 4; v++) {
            const int vx = v & 1, vy = v >> 1;
            unsigned m = 0, cbit = 0;
            for (int o = 0; o < 4; o++) {
                const int ox = o & 1, oy = o >> 1;
                const int pos = (vx + ox) + 3 * (vy + oy);
                if (pos == 4) cbit = (unsigned)o;
                else if (P >> pos & 1u) m |= 1u << o;
            }
            for (int k = 0; k < 4; k++) sum[k] += t2.v[m | (1u << cbit)][k] - t2.v[m][k];
        }
        const Delta2 d = pixel_delta_2d(P);
        if (sum[0] != 4 * d.ec8 || sum[1] != 4 * d.ec4 || sum[2] != 2 * d.per || sum[3] != 4) bad++;
    }
    // 3D: all 2^26 precedence patterns, split across threads
    unsigned nthr = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<int64_t> part(nthr, 0);
    std::vector<std::thread> th;
    const uint32_t total = 1u << 26;
    for (unsigned t = 0; t < nthr; t++) {
        th.emplace_back([&, t]() {
            int64_t b = 0;
            for (uint32_t i = t; i < total; i += nthr) {
                const uint32_t P = (i & 0x1FFFu) | ((i >> 13) << 14);
                int s0 = 0, s1 = 0, s2 = 0, s3 = 0;
                for (int v = 0; v < 8; v++) {
                    const int vx = v & 1, vy = (v >> 1) & 1, vz = v >> 2;
                    const int base = vx + 3 * vy + 9 * vz;
                    const uint32_t q = P >> base;
                    const unsigned m = (q & 3u) | (((q >> 3) & 3u) << 2) | (((q >> 9) & 3u) << 4) |
                                       (((q >> 12) & 3u) << 6);
                    const unsigned cbit = (unsigned)((1 - vx) + 2 * (1 - vy) + 4 * (1 - vz));
                    const unsigned mc = m | (1u << cbit);
                    s0 += t3.v[mc][0] - t3.v[m][0];
                    s1 += t3.v[mc][1] - t3.v[m][1];
                    s2 += t3.v[mc][2] - t3.v[m][2];
                    s3 += t3.v[mc][3] - t3.v[m][3];
                }
                const Delta3 d = voxel_delta_3d(P);
                if (s0 != 8 * d.ec || s1 != 2 * d.per || s2 != 4 * d.area || s3 != 8) b++;
                // 6-connectivity: the same telescoping with the 6-connected table
                int s6 = 0;
                for (int v = 0; v < 8; v++) {
                    const int vx = v & 1, vy = (v >> 1) & 1, vz = v >> 2;
                    const uint32_t q = P >> (vx + 3 * vy + 9 * vz);
                    const unsigned m = (q & 3u) | (((q >> 3) & 3u) << 2) | (((q >> 9) & 3u) << 4) |
                                       (((q >> 12) & 3u) << 6);
                    const unsigned cbit = (unsigned)((1 - vx) + 2 * (1 - vy) + 4 * (1 - vz));
                    s6 += t6.v[m | (1u << cbit)] - t6.v[m];
                }
                if (s6 != 8 * voxel_delta_3d6(P)) b++;
            }
            part[t] = b;
        });
    }
    for (auto &x : th) x.join();
    for (auto v : part) bad += v;
    // planar per-voxel form (ec_slice.h) against the vertex tables
    bad += selfcheck_planar(t3);
    // four-pixel byte-mask evaluation (fast 2D kernel) against the scalar closed form
    {
        uint64_t r2 = 0x2545F4914F6CDD1Dull;
        auto rnd2 = [&r2]() {
            r2 ^= r2 << 13; r2 ^= r2 >> 7; r2 ^= r2 << 17;
            return r2;
        };
        for (int trial = 0; trial < 200000; trial++) {
            const uint32_t span = (trial % 3 == 0) ? 2u : (trial % 3 == 1 ? 5u : (uint32_t)kMaxFastL3 + 1u);
            uint32_t k[4][9];
            for (int v = 0; v < 4; v++)
                for (int i = 0; i < 9; i++) k[v][i] = (uint32_t)(rnd2() % span);
            uint32_t n0[9], n1[9];
            for (int i = 0; i < 9; i++) {
                n0[i] = k[0][i] | (k[1][i] << 16);
                n1[i] = k[2][i] | (k[3][i] << 16);
            }
            const Quad2 q8 = quad_delta_2d<false>(n0, n0[4], n1, n1[4]);
            const Quad2 q4 = quad_delta_2d<true>(n0, n0[4], n1, n1[4]);
            const int e8[4] = {sbyte<0>(q8.ec), sbyte<1>(q8.ec), sbyte<2>(q8.ec), sbyte<3>(q8.ec)};
            const int e4[4] = {sbyte<0>(q4.ec), sbyte<1>(q4.ec), sbyte<2>(q4.ec), sbyte<3>(q4.ec)};
            const int pe[4] = {sbyte<0>(q8.per), sbyte<1>(q8.per), sbyte<2>(q8.per), sbyte<3>(q8.per)};
            for (int v = 0; v < 4; v++) {
                uint32_t P = 0;
                for (int i = 0; i < 9; i++) {
                    if (i == 4) continue;
                    const bool prec = i < 4 ? k[v][i] <= k[v][4] : k[v][i] < k[v][4];
                    P |= (uint32_t)prec << i;
                }
                const Delta2 d = pixel_delta_2d(P);
                if (e8[v] != d.ec8 || e4[v] != d.ec4 || pe[v] != d.per) bad++;
            }
        }
    }
    // four-voxel byte-mask evaluation (fast kernel) against the scalar closed form
    uint64_t rs = 0x9E3779B97F4A7C15ull;
    auto rnd = [&rs]() {
        rs ^= rs << 13; rs ^= rs >> 7; rs ^= rs << 17;
        return rs;
    };
    for (int trial = 0; trial < 200000; trial++) {
        const uint32_t span = (trial % 3 == 0) ? 3u : (trial % 3 == 1 ? 40u : (uint32_t)kMaxFastL3 + 1u);
        uint32_t k[4][27];
        for (int v = 0; v < 4; v++)
            for (int i = 0; i < 27; i++) k[v][i] = (uint32_t)(rnd() % span);
        uint32_t n0[27], n1[27];
        for (int i = 0; i < 27; i++) {
            n0[i] = k[0][i] | (k[1][i] << 16);
            n1[i] = k[2][i] | (k[3][i] << 16);
        }
        const QuadDelta q = quad_delta<true>(n0, n0[13], n1, n1[13]);
        const int ec[4] = {sbyte<0>(q.ec), sbyte<1>(q.ec), sbyte<2>(q.ec), sbyte<3>(q.ec)};
        const int pe[4] = {sbyte<0>(q.per), sbyte<1>(q.per), sbyte<2>(q.per), sbyte<3>(q.per)};
        const int ar[4] = {sbyte<0>(q.area), sbyte<1>(q.area), sbyte<2>(q.area), sbyte<3>(q.area)};
        for (int v = 0; v < 4; v++) {
            uint32_t P = 0;
            for (int i = 0; i < 27; i++) {
                if (i == 13) continue;
                const bool prec = i < 13 ? k[v][i] <= k[v][13] : k[v][i] < k[v][13];
                P |= (uint32_t)prec << i;
            }
            const Delta3 d = voxel_delta_3d(P);
            if (ec[v] != d.ec || pe[v] != d.per || ar[v] != d.area) bad++;
        }
    }
    // vertex types: every mask has a row, and the per-mask contributions are
    // the same for every mask of a type (the tables' premise)
    {
        constexpr TypeTable2D tt2 = make_type_table_2d();
        constexpr TypeTable3D tt3 = make_type_table_3d();
        for (unsigned m = 0; m < 16; m++) {
            if (tt2.t[m] >= kTypes2) { bad++; continue; }
            const unsigned r = kTable1Reps[tt2.t[m]];
            for (int k = 0; k < 4; k++) bad += t2.v[m][k] != t2.v[r][k];
        }
        for (unsigned m = 0; m < 256; m++) {
            if (tt3.t[m] >= kTypes3) { bad++; continue; }
            const unsigned r = kTable2Reps[tt3.t[m]];
            for (int k = 0; k < 4; k++) bad += t3.v[m][k] != t3.v[r][k];
        }
    }
    return bad;
}

}  // extern "C"

// ec_tune.cu -- autotuner for the curve kernels.
//
// A request's launch plan (z planes per work item, blocks per launch,
// shared-memory update schedule) is picked per shape class by timing the
// candidates on the request itself the first time the class is seen, with
// CUDA events on the request's stream.  Results are cached in the context and,
// when the environment variable EC_AUTOTUNE_CACHE names a file, kept in that
// JSON file (one object: class key -> [tile_z, grid, schedule, microseconds])
// across processes.  A server's slot contexts share the tuned plans of the
// context the server was created on.  Every candidate computes the same
// curves, so tuning changes only speed.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ec_internal.h"

using namespace ec;

namespace {

struct TunedPlan {
    int tile_z, grid, schedule;
    double us;
};

struct TuneCache {
    std::mutex mu;   // guards plans and refs (contexts sharing a cache have separate locks)
    std::map<std::string, TunedPlan> plans;
    bool loaded = false;
    int refs = 1;
};

std::string class_key(int device_sms, int ndim, int dtype, int32_t L, uint32_t desc, const int64_t *dims)
{
    int64_t n = 1;
    for (int i = 0; i < ndim; i++) n *= dims[i];
    const int size_class = (int)std::floor(std::log2((double)std::max<int64_t>(n, 1)));
    const int l_class = (int)std::ceil(std::log2((double)std::max(L, 1)));
    char buf[128];
    snprintf(buf, sizeof buf, "sm%d_d%d_t%d_L%d_D%u_n%d_w%d", device_sms, ndim, dtype, l_class, desc, size_class,
             (int)(dims[ndim - 1] % 4 == 0));
    return buf;
}

void load_file(TuneCache &tc)
{
    tc.loaded = true;
    const char *path = getenv("EC_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    std::string s;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, n);
    fclose(f);
    // entries look like  "key": [tile_z, grid, schedule, us]
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {
        const size_t end = s.find('"', pos + 1);
        if (end == std::string::npos) break;
        const std::string key = s.substr(pos + 1, end - pos - 1);
        TunedPlan tp{};
        if (sscanf(s.c_str() + end + 1, " : [ %d , %d , %d , %lf ]", &tp.tile_z, &tp.grid, &tp.schedule, &tp.us) == 4)
            tc.plans[key] = tp;
        pos = end + 1;
    }
}

void save_file(const TuneCache &tc)
{
    const char *path = getenv("EC_AUTOTUNE_CACHE");
    if (!path) return;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (const auto &kv : tc.plans) {
        fprintf(f, "  \"%s\": [%d, %d, %d, %.2f]%s\n", kv.first.c_str(), kv.second.tile_z, kv.second.grid,
                kv.second.schedule, kv.second.us, ++i < tc.plans.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

// The context's cache, created on first use (under ctx->mu); lock tc.mu
// before touching its plans.
TuneCache &cache_of(ec_ctx *ctx)
{
    if (!ctx->tune_cache) ctx->tune_cache = new TuneCache();
    TuneCache &tc = *(TuneCache *)ctx->tune_cache;
    std::lock_guard<std::mutex> g(tc.mu);
    if (!tc.loaded) load_file(tc);
    return tc;
}

}  // namespace

// Pick (and remember) the plan for a request.  Called with ctx->mu held and
// the context's scratch large enough for the request.
int ec::tuned_plan(ec_ctx *ctx, int ndim, const void *field, const int64_t *dims, int dtype, const void *thr,
                   int32_t L, int connectivity, uint32_t desc, int64_t *out, cudaStream_t s, CurvePlan &plan)
{
    TuneCache &tc = cache_of(ctx);
    const std::string key = class_key(ctx->num_sms, ndim, dtype, L, desc, dims);
    {
        std::lock_guard<std::mutex> g(tc.mu);
        auto it = tc.plans.find(key);
        if (it != tc.plans.end()) {
            plan.tile_z = it->second.tile_z;
            plan.grid = it->second.grid;
            plan.hist_schedule = it->second.schedule;
            return EC_OK;
        }
    }
    std::vector<TunedPlan> cands;
    if (ndim == 3) {
        const int64_t nb = ((dims[2] + 63) / 64) * ((dims[1] + 15) / 16);   // fast-kernel columns
        for (int tz : {16, 32, 64})
            for (int g : {0, 2 * ctx->num_sms})
                for (int sch : {1, 3}) {
                    if (g && nb * ((dims[0] + tz - 1) / tz) < g) continue;
                    cands.push_back({tz, g, sch, 0});
                }
    } else {
        for (int g : {0, ctx->num_sms, 4 * ctx->num_sms}) cands.push_back({0, g, 1, 0});
    }
    cudaEvent_t e0, e1;
    EC_CUDA(cudaEventCreate(&e0));
    EC_CUDA(cudaEventCreate(&e1));
    TunedPlan best{0, 0, 1, 1e30};
    int rc = EC_OK;
    for (auto &c : cands) {
        CurvePlan p = plan;
        p.tile_z = c.tile_z;
        p.grid = c.grid;
        p.hist_schedule = c.schedule;
        p.prof = nullptr;
        float best_ms = 1e30f;
        for (int rep = 0; rep < 3 && rc == EC_OK; rep++) {
            cudaEventRecord(e0, s);
            rc = enqueue_curve(p, ndim, field, dims, dtype, thr, L, connectivity, desc, out, ctx->ws, s);
            cudaEventRecord(e1, s);
            if (rc) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = EC_ERR_CUDA; break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best_ms) best_ms = ms;   // first run warms up
        }
        if (rc) break;
        c.us = best_ms * 1e3;
        if (c.us < best.us) best = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> g(tc.mu);
        tc.plans[key] = best;
        save_file(tc);
    }
    plan.tile_z = best.tile_z;
    plan.grid = best.grid;
    plan.hist_schedule = best.schedule;
    return EC_OK;
}

bool ec::tune_lookup(ec_ctx *ctx, const std::string &key, int out[3])
{
    TuneCache &tc = cache_of(ctx);
    std::lock_guard<std::mutex> g(tc.mu);
    auto it = tc.plans.find(key);
    if (it == tc.plans.end()) return false;
    out[0] = it->second.tile_z;
    out[1] = it->second.grid;
    out[2] = it->second.schedule;
    return true;
}

void ec::tune_store(ec_ctx *ctx, const std::string &key, const int v[3], double us)
{
    TuneCache &tc = cache_of(ctx);
    std::lock_guard<std::mutex> g(tc.mu);
    tc.plans[key] = TunedPlan{v[0], v[1], v[2], us};
    save_file(tc);
}

void ec::tune_share(ec_ctx *from, ec_ctx *to)
{
    TuneCache &tc = cache_of(from);
    std::lock_guard<std::mutex> g(tc.mu);
    tc.refs++;
    to->tune_cache = &tc;
}

void ec::tune_release(ec_ctx *ctx)
{
    TuneCache *tc = (TuneCache *)ctx->tune_cache;
    ctx->tune_cache = nullptr;
    if (!tc) return;
    bool last;
    {
        std::lock_guard<std::mutex> g(tc->mu);
        last = --tc->refs == 0;
    }
    if (last) delete tc;
}

extern "C" int ec_tuned_plan(ec_ctx *ctx, int32_t ndim, int dtype, int32_t L, uint32_t descriptors,
                             const int64_t *dims, int32_t out[3])
{
    clear_error();
    if (!ctx || !dims || !out || (ndim != 2 && ndim != 3)) { set_error("bad arguments"); return EC_ERR_ARG; }
    std::lock_guard<std::mutex> lock(ctx->mu);
    TuneCache &tc = cache_of(ctx);
    std::lock_guard<std::mutex> g(tc.mu);
    auto it = tc.plans.find(class_key(ctx->num_sms, ndim, dtype, L, descriptors, dims));
    if (it == tc.plans.end()) { set_error("no tuned plan for this class yet"); return EC_ERR_ARG; }
    out[0] = it->second.tile_z;
    out[1] = it->second.grid;
    out[2] = it->second.schedule;
    return EC_OK;
}

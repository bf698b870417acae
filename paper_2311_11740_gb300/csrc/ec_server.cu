// ec_server.cu -- request loop with continuous batching.
//
// The paper motivates real-time use (Sec. 4: a liquid-crystal sensor whose
// 36 grid squares must be processed at video rate).  The server turns a
// stream of independent requests into overlapping, batched GPU work:
//   * submit() queues a request (FIFO) and returns a ticket at once;
//   * a worker thread admits, whenever a slot (a CUDA stream with its own
//     context) is free, the run of queued requests at the head of the queue
//     whose device bytes fit in the budget (at most kGroupRequests requests
//     and kGroupBytes of fields, or one larger request), even while earlier
//     groups are still running.  Under light load a group is one request;
//     under load groups grow and the per-request launch cost disappears;
//   * an admitted group gets stream-ordered device memory from the server's
//     own pool (which keeps up to the budget mapped), its fields and thresholds are copied
//     in, all its curves are computed by one persistent batched launch
//     (ec_batch on the slot's context), and every result is copied back to
//     its caller's host buffer;
//   * the worker notices completion through an event, frees the memory and
//     the slot, stamps the latencies and admits the next group.
// Results are identical to standalone calls: every request has its own
// histogram and the curves are exact integers.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ec_internal.h"

using namespace ec;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int dsize(int dtype) { return dtype == EC_F32 ? 4 : (dtype == EC_U16 ? 2 : 1); }

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Req {
    uint64_t ticket = 0;
    ec_field_desc d{};
    bool field_on_device = false;
    size_t field_bytes = 0, thr_bytes = 0, out_bytes = 0, scratch_bytes = 0, total = 0;
    int state = 0;   // 0 queued, 3 being started, 1 running, 2 done
    int status = EC_OK;
    double t_submit = 0, t_done = 0;
    int slot = -1;
    void *dmem = nullptr;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    ec_ctx *bctx = nullptr;    // batch tables and graph of this slot's groups
    std::vector<Req *> group;  // admitted requests (empty = free)
    size_t group_total = 0;    // their budgeted bytes
    void *dmem = nullptr;
    bool running = false;
    // page-locked staging of the group's thresholds (in) and outputs (out):
    // one copy each way per group instead of one per request
    char *stage_in = nullptr, *stage_out = nullptr;
    size_t stage_in_bytes = 0, stage_out_bytes = 0;
    std::vector<size_t> out_off;   // each request's output offset in stage_out
};

// Grow a page-locked staging buffer to at least `need` bytes.
int ensure_pinned(char *&buf, size_t &have, size_t need)
{
    if (have >= need) return EC_OK;
    if (buf) cudaFreeHost(buf);
    buf = nullptr;
    have = 0;
    const size_t want = std::max(need, (size_t)1 << 20);
    if (cudaMallocHost((void **)&buf, want) != cudaSuccess) {
        cudaGetLastError();
        buf = nullptr;
        set_error("server staging allocation failed");
        return EC_ERR_OOM;
    }
    have = want;
    return EC_OK;
}

constexpr size_t kGroupRequests = 256;
constexpr size_t kGroupBytes = (size_t)64 << 20;

}  // namespace

struct ec_server {
    ec_ctx *ctx = nullptr;
    cudaMemPool_t pool = nullptr;   // the server's own stream-ordered pool; keeps up to `budget` mapped
    size_t budget = 0;
    size_t used = 0;
    std::vector<Slot> slots;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    std::mutex mu;
    std::condition_variable wake, done_cv;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t max_queue = 1u << 16;
    std::vector<double> latencies;
    double first_submit = -1, last_done = 0;
};

namespace {

// Enqueue one admitted group on its slot's stream (worker thread, server lock
// released): device memory, input copies, one batched launch, output copies.
// Device layout: [thresholds][outputs][fields], each piece 256-byte aligned.
int start_group(ec_server *sv, Slot &sl)
{
    const size_t n = sl.group.size();
    size_t thr_bytes = 0, out_bytes = 0, field_bytes = 0;
    for (Req *r : sl.group) {
        thr_bytes += round256(r->thr_bytes);
        out_bytes += round256(r->out_bytes);
        field_bytes += r->field_on_device ? 0 : round256(r->field_bytes);
    }
    int rc = ensure_pinned(sl.stage_in, sl.stage_in_bytes, thr_bytes);
    if (!rc) rc = ensure_pinned(sl.stage_out, sl.stage_out_bytes, out_bytes);
    if (rc) return rc;
    cudaError_t e =
        cudaMallocFromPoolAsync(&sl.dmem, std::max<size_t>(thr_bytes + out_bytes + field_bytes, 256), sv->pool, sl.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sl.dmem = nullptr;
        set_error("request allocation failed: %s", cudaGetErrorString(e));
        return EC_ERR_OOM;
    }
    char *thr_dev = (char *)sl.dmem, *out_dev = thr_dev + thr_bytes, *field_dev = out_dev + out_bytes;
    std::vector<ec_field_desc> descs(n);
    sl.out_off.resize(n);
    size_t to = 0, oo = 0, fo = 0;
    for (size_t i = 0; i < n; i++) {
        Req *r = sl.group[i];
        ec_field_desc &d = descs[i];
        d = r->d;
        if (r->d.thresholds) {
            memcpy(sl.stage_in + to, r->d.thresholds, r->thr_bytes);
            d.thresholds = thr_dev + to;
            to += round256(r->thr_bytes);
        }
        sl.out_off[i] = oo;
        d.out = (int64_t *)(out_dev + oo);
        oo += round256(r->out_bytes);
        if (!r->field_on_device) {
            EC_CUDA(cudaMemcpyAsync(field_dev + fo, r->d.field, r->field_bytes, cudaMemcpyHostToDevice, sl.stream));
            d.field = field_dev + fo;
            fo += round256(r->field_bytes);
        }
    }
    if (to) EC_CUDA(cudaMemcpyAsync(thr_dev, sl.stage_in, to, cudaMemcpyHostToDevice, sl.stream));
    rc = ec_batch(sl.bctx, descs.data(), (int32_t)n, (void *)sl.stream);
    if (rc) return rc;
    EC_CUDA(cudaMemcpyAsync(sl.stage_out, out_dev, oo, cudaMemcpyDeviceToHost, sl.stream));
    EC_CUDA(cudaEventRecord(sl.done, sl.stream));
    return EC_OK;
}

void finish_request(ec_server *sv, Req *r, int status)
{
    r->status = status;
    r->state = 2;
    r->t_done = now_s();
    sv->latencies.push_back(r->t_done - r->t_submit);
    sv->last_done = std::max(sv->last_done, r->t_done);
}

void worker_loop(ec_server *sv)
{
    DeviceGuard dg(sv->ctx->device);
    std::unique_lock<std::mutex> lock(sv->mu);
    std::vector<Slot *> admitted;
    for (;;) {
        bool progress = false;
        // completions (event queries do not block); outputs leave the staging
        // buffer without the lock held
        for (auto &sl : sv->slots) {
            if (!sl.running) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            int st = EC_OK;
            if (q != cudaSuccess) {
                st = EC_ERR_CUDA;
                cudaGetLastError();
            }
            if (sl.dmem) cudaFreeAsync(sl.dmem, sl.stream);
            sl.dmem = nullptr;
            sl.running = false;
            if (st == EC_OK) {
                lock.unlock();
                for (size_t i = 0; i < sl.group.size(); i++)
                    memcpy(sl.group[i]->d.out, sl.stage_out + sl.out_off[i], sl.group[i]->out_bytes);
                lock.lock();
            }
            sv->used -= sl.group_total;
            for (Req *r : sl.group) finish_request(sv, r, st);
            sl.group.clear();
            sl.group_total = 0;
            progress = true;
        }
        if (progress) sv->done_cv.notify_all();
        // admissions in arrival order: reserve memory and a slot under the lock
        admitted.clear();
        for (auto &sl : sv->slots) {
            if (sv->queue.empty()) break;
            if (!sl.group.empty()) continue;
            size_t field_bytes = 0;
            while (!sv->queue.empty() && sl.group.size() < kGroupRequests) {
                Req *r = sv->queue.front();
                if (sv->used + r->total > sv->budget) break;
                if (!sl.group.empty() && field_bytes + r->field_bytes > kGroupBytes) break;
                sv->queue.pop_front();
                sv->used += r->total;
                sl.group_total += r->total;
                field_bytes += r->field_bytes;
                r->state = 3;   // being started
                sl.group.push_back(r);
            }
            if (sl.group.empty()) break;   // the head does not fit yet
            admitted.push_back(&sl);
        }
        if (!admitted.empty()) {
            // copies from pageable host memory block: start groups without the lock
            lock.unlock();
            for (Slot *sl : admitted) {
                const int rc = start_group(sv, *sl);
                if (rc != EC_OK) {
                    cudaStreamSynchronize(sl->stream);
                    cudaGetLastError();
                    if (sl->dmem) cudaFreeAsync(sl->dmem, sl->stream);
                    sl->dmem = nullptr;
                }
                lock.lock();
                if (rc != EC_OK) {
                    sv->used -= sl->group_total;
                    for (Req *r : sl->group) finish_request(sv, r, rc);
                    sl->group.clear();
                    sl->group_total = 0;
                    sv->done_cv.notify_all();
                } else {
                    for (Req *r : sl->group) r->state = 1;
                    sl->running = true;
                }
                lock.unlock();
            }
            lock.lock();
            progress = true;
        }
        bool busy = false;
        for (auto &sl : sv->slots) busy |= !sl.group.empty();
        if (sv->stop && !busy) break;
        if (!progress) {
            if (busy) sv->wake.wait_for(lock, std::chrono::microseconds(50));
            else sv->wake.wait_for(lock, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace

extern "C" {

int ec_server_create(ec_ctx *ctx, size_t device_mem_budget, int32_t max_slots, ec_server **out)
{
    clear_error();
    if (!ctx || !out || max_slots < 1 || max_slots > 256 || device_mem_budget == 0) {
        set_error("bad server arguments");
        return EC_ERR_ARG;
    }
    DeviceGuard dg(ctx->device);
    auto sv = std::make_unique<ec_server>();
    sv->ctx = ctx;
    sv->budget = device_mem_budget;
    sv->slots.resize(max_slots);
    int rc = EC_OK;
    {
        // a pool of its own whose freed memory stays mapped up to the budget, so
        // groups reuse it instead of mapping fresh memory each time
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        uint64_t keep = device_mem_budget;
        if (cudaMemPoolCreate(&sv->pool, &props) != cudaSuccess ||
            cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaGetLastError();
            if (sv->pool) cudaMemPoolDestroy(sv->pool);
            set_error("server memory pool creation failed");
            return EC_ERR_CUDA;
        }
    }
    for (auto &sl : sv->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            set_error("server stream creation failed");
            rc = EC_ERR_CUDA;
            break;
        }
        if ((rc = ec_ctx_create(&sl.bctx, ctx->device)) != EC_OK) break;
        if (ctx->autotune) {
            // the slots tune their groups' mix classes into the creator's plans
            std::lock_guard<std::mutex> lock(ctx->mu);
            sl.bctx->autotune = ctx->autotune;
            tune_share(ctx, sl.bctx);
        }
    }
    if (rc != EC_OK) {
        for (auto &sl : sv->slots) {
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.bctx) ec_ctx_destroy(sl.bctx);
        }
        cudaMemPoolDestroy(sv->pool);
        return rc;
    }
    ec_server *raw = sv.release();
    raw->worker = std::thread(worker_loop, raw);
    *out = raw;
    return EC_OK;
}

}  // extern "C"

namespace {

// Validate one request and size it (no lock held).
int make_req(const ec_field_desc *req, std::unique_ptr<Req> &out)
{
    if (req->ndim != 2 && req->ndim != 3) { set_error("ndim must be 2 or 3"); return EC_ERR_ARG; }
    int rc = validate_request(req->ndim, req->field, req->dims, req->dtype, req->thresholds, req->L,
                              req->connectivity, req->descriptors, req->out);
    if (rc) return rc;
    auto r = std::make_unique<Req>();
    r->d = *req;
    int64_t n = 1;
    for (int i = 0; i < req->ndim; i++) n *= req->dims[i];
    r->field_bytes = (size_t)n * dsize(req->dtype);
    r->thr_bytes = req->thresholds ? (size_t)req->L * dsize(req->dtype) : 0;
    r->out_bytes = (size_t)row_map(req->descriptors).nd * (size_t)req->L * sizeof(int64_t);
    r->scratch_bytes = curve_scratch_bytes(req->descriptors, req->L);
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, req->field) == cudaSuccess && attr.type == cudaMemoryTypeDevice)
        r->field_on_device = true;
    cudaGetLastError();
    r->total = round256(r->scratch_bytes) + round256(r->out_bytes) + round256(r->thr_bytes) +
               (r->field_on_device ? 0 : round256(r->field_bytes));
    out = std::move(r);
    return EC_OK;
}

// Queue validated requests under the server lock, all or none.
int enqueue(ec_server *sv, std::vector<std::unique_ptr<Req>> &rs, uint64_t *tickets)
{
    std::lock_guard<std::mutex> lock(sv->mu);
    for (size_t i = 0; i < rs.size(); i++)
        if (rs[i]->total > sv->budget) {
            set_error("request %zu needs %zu device bytes, above the server budget of %zu", i, rs[i]->total,
                      sv->budget);
            return EC_ERR_OOM;
        }
    if (sv->queue.size() + rs.size() > sv->max_queue) { set_error("request queue full"); return EC_ERR_BUSY; }
    if (sv->stop) { set_error("server is shutting down"); return EC_ERR_BUSY; }
    const double t = now_s();
    if (sv->first_submit < 0) sv->first_submit = t;
    for (size_t i = 0; i < rs.size(); i++) {
        Req *r = rs[i].get();
        r->ticket = sv->next_ticket++;
        r->t_submit = t;
        tickets[i] = r->ticket;
        sv->queue.push_back(r);
        sv->reqs[r->ticket] = std::move(rs[i]);
    }
    sv->wake.notify_one();
    return EC_OK;
}

}  // namespace

extern "C" {

int ec_server_submit(ec_server *sv, const ec_field_desc *req, uint64_t *ticket)
{
    clear_error();
    if (!sv || !req || !ticket) { set_error("NULL argument"); return EC_ERR_ARG; }
    std::vector<std::unique_ptr<Req>> rs(1);
    int rc = make_req(req, rs[0]);
    if (rc) return rc;
    return enqueue(sv, rs, ticket);
}

int ec_server_submit_many(ec_server *sv, const ec_field_desc *reqs, int32_t n, uint64_t *tickets)
{
    clear_error();
    if (!sv || n < 0 || (n > 0 && (!reqs || !tickets))) { set_error("bad arguments"); return EC_ERR_ARG; }
    std::vector<std::unique_ptr<Req>> rs(n);
    for (int32_t i = 0; i < n; i++) {
        const int rc = make_req(&reqs[i], rs[i]);
        if (rc) {
            const std::string msg = ec_last_error();
            set_error("request %d: %s", i, msg.c_str());
            return rc;
        }
    }
    return enqueue(sv, rs, tickets);
}

int ec_server_poll(ec_server *sv, uint64_t ticket, int *done, int32_t *status)
{
    clear_error();
    if (!sv || !done || !status) { set_error("NULL argument"); return EC_ERR_ARG; }
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) { set_error("unknown ticket"); return EC_ERR_ARG; }
    *done = it->second->state == 2;
    *status = it->second->status;
    return EC_OK;
}

int ec_server_wait(ec_server *sv, uint64_t ticket, int64_t timeout_ms, int32_t *status)
{
    clear_error();
    if (!sv || !status) { set_error("NULL argument"); return EC_ERR_ARG; }
    std::unique_lock<std::mutex> lock(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) { set_error("unknown ticket"); return EC_ERR_ARG; }
    Req *r = it->second.get();
    const bool ok = sv->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                         [r] { return r->state == 2; });
    if (!ok) { set_error("request %llu not done after %lld ms", (unsigned long long)ticket, (long long)timeout_ms); return EC_ERR_TIMEOUT; }
    *status = r->status;
    return EC_OK;
}

int ec_server_stats(ec_server *sv, double out[5])
{
    clear_error();
    if (!sv || !out) { set_error("NULL argument"); return EC_ERR_ARG; }
    std::lock_guard<std::mutex> lock(sv->mu);
    std::vector<double> l = sv->latencies;
    std::sort(l.begin(), l.end());
    const size_t n = l.size();
    out[0] = (double)n;
    out[1] = n ? l[(size_t)(0.50 * (n - 1))] * 1e6 : 0;
    out[2] = n ? l[(size_t)(0.99 * (n - 1))] * 1e6 : 0;
    double s = 0;
    for (double v : l) s += v;
    out[3] = n ? s / n * 1e6 : 0;
    out[4] = n ? (sv->last_done - sv->first_submit) * 1e6 : 0;
    return EC_OK;
}

int ec_server_wait_all(ec_server *sv, int64_t timeout_ms)
{
    clear_error();
    if (!sv) { set_error("NULL argument"); return EC_ERR_ARG; }
    std::unique_lock<std::mutex> lock(sv->mu);
    const bool ok = sv->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [sv] {
        if (!sv->queue.empty()) return false;
        for (auto &sl : sv->slots)
            if (!sl.group.empty()) return false;
        return true;
    });
    if (!ok) { set_error("requests still pending after %lld ms", (long long)timeout_ms); return EC_ERR_TIMEOUT; }
    return EC_OK;
}

int ec_server_reset_stats(ec_server *sv)
{
    clear_error();
    if (!sv) { set_error("NULL argument"); return EC_ERR_ARG; }
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->latencies.clear();
    sv->first_submit = -1;
    sv->last_done = 0;
    return EC_OK;
}

int ec_server_destroy(ec_server *sv)
{
    clear_error();
    if (!sv) return EC_OK;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        // requests not yet admitted are cancelled
        for (Req *r : sv->queue) {
            r->status = EC_ERR_BUSY;
            r->state = 2;
        }
        sv->queue.clear();
    }
    sv->wake.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    {
        DeviceGuard dg(sv->ctx->device);
        for (auto &sl : sv->slots) {
            if (sl.stream) cudaStreamSynchronize(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.bctx) ec_ctx_destroy(sl.bctx);
            if (sl.stage_in) cudaFreeHost(sl.stage_in);
            if (sl.stage_out) cudaFreeHost(sl.stage_out);
        }
        if (sv->pool) cudaMemPoolDestroy(sv->pool);
    }
    delete sv;
    return EC_OK;
}

}  // extern "C"

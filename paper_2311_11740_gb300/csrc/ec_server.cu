// ec_server.cu -- request loop with continuous admission.
//
// The paper motivates real-time use (Sec. 4: a liquid-crystal sensor whose
// 36 grid squares must be processed at video rate).  The server turns a
// stream of independent requests into overlapping GPU work:
//   * submit() queues a request (FIFO) and returns a ticket at once;
//   * a worker thread admits the head of the queue as soon as a slot (a CUDA
//     stream) is free and the request's device bytes fit in the budget, even
//     while earlier requests are still running;
//   * an admitted request gets stream-ordered device memory (cudaMallocAsync
//     from the device's default pool), its field and thresholds are copied
//     in, its curves are computed into its own histogram, and the result is
//     copied back to the caller's host buffer;
//   * the worker notices completion through an event, frees the memory and
//     the slot, stamps the latency and admits the next request.
// Results are identical to standalone calls: every request has its own
// scratch and the curves are exact integers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
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
    Req *req = nullptr;
};

}  // namespace

struct ec_server {
    ec_ctx *ctx = nullptr;
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

// Enqueue one admitted request on its slot's stream (worker thread, server lock released).
int start_request(ec_server *sv, Req *r, Slot &sl)
{
    cudaError_t e = cudaMallocAsync(&r->dmem, r->total, sl.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        r->dmem = nullptr;
        set_error("request allocation failed: %s", cudaGetErrorString(e));
        return EC_ERR_OOM;
    }
    char *p = (char *)r->dmem;
    void *scratch = p;
    p += round256(r->scratch_bytes);
    int64_t *out_dev = (int64_t *)p;
    p += round256(r->out_bytes);
    void *thr_dev = nullptr;
    if (r->d.thresholds) {
        thr_dev = p;
        p += round256(r->thr_bytes);
        EC_CUDA(cudaMemcpyAsync(thr_dev, r->d.thresholds, r->thr_bytes, cudaMemcpyHostToDevice, sl.stream));
    }
    const void *field_dev = r->d.field;
    if (!r->field_on_device) {
        EC_CUDA(cudaMemcpyAsync(p, r->d.field, r->field_bytes, cudaMemcpyHostToDevice, sl.stream));
        field_dev = p;
    }
    CurvePlan plan;
    plan.algo = ALGO_VOXEL;
    plan.num_sms = sv->ctx->num_sms;
    int rc = enqueue_curve(plan, r->d.ndim, field_dev, r->d.dims, r->d.dtype, thr_dev, r->d.L, r->d.connectivity,
                           r->d.descriptors, out_dev, scratch, sl.stream);
    if (rc) return rc;
    EC_CUDA(cudaMemcpyAsync(r->d.out, out_dev, r->out_bytes, cudaMemcpyDeviceToHost, sl.stream));
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
    std::vector<std::pair<Req *, Slot *>> admitted;
    for (;;) {
        bool progress = false;
        // completions (event queries do not block)
        for (size_t i = 0; i < sv->slots.size(); i++) {
            Slot &sl = sv->slots[i];
            if (!sl.req || sl.req->state != 1) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            Req *r = sl.req;
            int st = EC_OK;
            if (q != cudaSuccess) {
                st = EC_ERR_CUDA;
                cudaGetLastError();
            }
            if (r->dmem) cudaFreeAsync(r->dmem, sl.stream);
            r->dmem = nullptr;
            sv->used -= r->total;
            finish_request(sv, r, st);
            sl.req = nullptr;
            progress = true;
        }
        if (progress) sv->done_cv.notify_all();
        // admissions in arrival order: reserve memory and a slot under the lock
        admitted.clear();
        while (!sv->queue.empty()) {
            Req *r = sv->queue.front();
            if (sv->used + r->total > sv->budget) break;
            Slot *free_slot = nullptr;
            for (auto &sl : sv->slots)
                if (!sl.req) { free_slot = &sl; break; }
            if (!free_slot) break;
            sv->queue.pop_front();
            sv->used += r->total;
            r->state = 3;   // being started
            free_slot->req = r;
            admitted.emplace_back(r, free_slot);
        }
        if (!admitted.empty()) {
            // copies from pageable host memory block: start requests without the lock
            lock.unlock();
            for (auto &rs : admitted) {
                Req *r = rs.first;
                Slot *sl = rs.second;
                const int rc = start_request(sv, r, *sl);
                if (rc != EC_OK) {
                    cudaStreamSynchronize(sl->stream);
                    cudaGetLastError();
                    if (r->dmem) cudaFreeAsync(r->dmem, sl->stream);
                    r->dmem = nullptr;
                }
                lock.lock();
                if (rc != EC_OK) {
                    sv->used -= r->total;
                    finish_request(sv, r, rc);
                    sl->req = nullptr;
                    sv->done_cv.notify_all();
                } else {
                    r->state = 1;
                }
                lock.unlock();
            }
            lock.lock();
            progress = true;
        }
        bool busy = false;
        for (auto &sl : sv->slots) busy |= sl.req != nullptr;
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
    for (auto &sl : sv->slots) {
        EC_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
        EC_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    }
    ec_server *raw = sv.release();
    raw->worker = std::thread(worker_loop, raw);
    *out = raw;
    return EC_OK;
}

int ec_server_submit(ec_server *sv, const ec_field_desc *req, uint64_t *ticket)
{
    clear_error();
    if (!sv || !req || !ticket) { set_error("NULL argument"); return EC_ERR_ARG; }
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
    std::lock_guard<std::mutex> lock(sv->mu);
    if (r->total > sv->budget) {
        set_error("request needs %zu device bytes, above the server budget of %zu", r->total, sv->budget);
        return EC_ERR_OOM;
    }
    if (sv->queue.size() >= sv->max_queue) { set_error("request queue full"); return EC_ERR_BUSY; }
    if (sv->stop) { set_error("server is shutting down"); return EC_ERR_BUSY; }
    r->ticket = sv->next_ticket++;
    r->t_submit = now_s();
    if (sv->first_submit < 0) sv->first_submit = r->t_submit;
    *ticket = r->ticket;
    sv->queue.push_back(r.get());
    sv->reqs[r->ticket] = std::move(r);
    sv->wake.notify_one();
    return EC_OK;
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
        }
    }
    delete sv;
    return EC_OK;
}

}  // extern "C"

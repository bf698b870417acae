// ec_stream.cu -- low-memory 3D processing by z-slabs (Sec. 2.3).
//
// The paper's low-memory mode reads only the values a vertex needs straight
// from the file.  On the GPU the same idea becomes streaming: the field is
// cut into slabs of S planes; each slab is brought into a device buffer
// together with one halo plane on each side (a voxel's contribution change
// depends on its 26 neighbours), while the previous slab is being counted.
// Every slab adds into one shared int64 histogram, so the result does not
// depend on the slab height: histograms are additive and every voxel is
// counted in exactly one slab.  Halo planes that fall outside the field read
// as never active.
//
// Two streams: the side stream fills buffer b (pinned-host copy or the
// caller's producer), the compute stream waits for it, counts the slab and
// releases the buffer with an event.  With a host field, a slab's two lower
// planes (the previous slab's top two) are copied on the device from the
// previous buffer, so every plane crosses the host link once.  The memory
// cap bounds the number and height of the buffers.
#include <cuda_runtime.h>
#include <errno.h>
#include <fcntl.h>
#include <stdint.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "ec_internal.h"

using namespace ec;

namespace {

int dtype_size(int dtype) { return dtype == EC_F32 ? 4 : (dtype == EC_U16 ? 2 : 1); }

// Reader threads kept in the context for raw-file streaming: each slab's
// byte range is split into nthr contiguous parts read in parallel
// (page-cache copies are bound by per-core memory bandwidth, so more readers
// read faster).
struct ReaderPool {
    std::vector<std::thread> th;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::function<void(int)> job;
    uint64_t gen = 0;
    int pending = 0;
    bool stop = false;
    explicit ReaderPool(int n)
    {
        for (int t = 1; t < n; t++)
            th.emplace_back([this, t]() {
                uint64_t seen = 0;
                for (;;) {
                    std::function<void(int)> fn;
                    {
                        std::unique_lock<std::mutex> lk(mu);
                        cv.wait(lk, [&] { return stop || gen != seen; });
                        if (stop) return;
                        seen = gen;
                        fn = job;
                    }
                    fn(t);
                    std::lock_guard<std::mutex> lk(mu);
                    if (--pending == 0) done_cv.notify_one();
                }
            });
    }
    int size() const { return (int)th.size() + 1; }
    // run fn(0 .. size()-1), part 0 on the calling thread
    void run(const std::function<void(int)> &fn)
    {
        {
            std::lock_guard<std::mutex> lk(mu);
            job = fn;
            pending = (int)th.size();
            gen++;
        }
        cv.notify_all();
        fn(0);
        std::unique_lock<std::mutex> lk(mu);
        done_cv.wait(lk, [&] { return pending == 0; });
    }
    ~ReaderPool()
    {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv.notify_all();
        for (auto &x : th) x.join();
    }
};

// Page-locked staging of raw-file streaming, kept in the context between
// calls (grown when a call needs more; used only inside the streaming call,
// which holds the context's lock): two buffers, an event per buffer marking
// the copy that last read it, and the reader pool.
struct FileStaging {
    void *pinned[2] = {nullptr, nullptr};
    size_t cap = 0;
    cudaEvent_t copied[2] = {nullptr, nullptr};
    ReaderPool *pool = nullptr;
    ~FileStaging()
    {
        delete pool;
        for (int i = 0; i < 2; i++) {
            if (copied[i]) { cudaEventSynchronize(copied[i]); cudaEventDestroy(copied[i]); }
            if (pinned[i]) cudaFreeHost(pinned[i]);
        }
    }
};

// Streams, events and device memory of the streaming path, kept in the
// context between calls (the memory is reallocated when a call needs more, or
// when it would not fit the call's cap).
struct StreamRes {
    void *mem = nullptr;
    size_t bytes = 0;
    cudaStream_t comp = nullptr, side = nullptr;
    cudaEvent_t filled[3] = {nullptr, nullptr, nullptr}, freed[3] = {nullptr, nullptr, nullptr};
    FileStaging *file = nullptr;
    ~StreamRes()
    {
        delete file;
        if (comp) cudaStreamSynchronize(comp);
        if (side) cudaStreamSynchronize(side);
        for (int i = 0; i < 3; i++) {
            if (filled[i]) cudaEventDestroy(filled[i]);
            if (freed[i]) cudaEventDestroy(freed[i]);
        }
        if (comp) cudaStreamDestroy(comp);
        if (side) cudaStreamDestroy(side);
        if (mem) cudaFree(mem);
    }
};

int stream_setup(StreamRes &res)
{
    if (res.comp) return EC_OK;
    EC_CUDA(cudaStreamCreateWithFlags(&res.comp, cudaStreamNonBlocking));
    EC_CUDA(cudaStreamCreateWithFlags(&res.side, cudaStreamNonBlocking));
    for (int i = 0; i < 3; i++) {
        EC_CUDA(cudaEventCreateWithFlags(&res.filled[i], cudaEventDisableTiming));
        EC_CUDA(cudaEventCreateWithFlags(&res.freed[i], cudaEventDisableTiming));
    }
    return EC_OK;
}

}  // namespace

void ec::stream_release(ec_ctx *ctx)
{
    delete (StreamRes *)ctx->stream_state;
    ctx->stream_state = nullptr;
}

extern "C" int ec_curve_3d_stream(ec_ctx *ctx, const void *host_field, ec_slab_fn producer, void *user,
                                  const int64_t dims[3], int dtype, const void *thresholds_host, int32_t L,
                                  int connectivity, uint32_t descriptors, int64_t slab_planes, size_t device_mem_cap,
                                  int64_t *out_host)
{
    clear_error();
    if (!ctx) { set_error("ctx is NULL"); return EC_ERR_ARG; }
    const void *any_field = host_field ? host_field : (const void *)producer;
    int rc = validate_request(3, any_field, dims, dtype, thresholds_host, L, connectivity, descriptors, out_host);
    if (rc) return rc;
    if (!host_field && !producer) { set_error("need a host field or a producer"); return EC_ERR_ARG; }
    if (slab_planes < 1) { set_error("slab_planes must be >= 1"); return EC_ERR_ARG; }
    if (L == 0) return EC_OK;
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);

    const int64_t d = dims[0], h = dims[1], w = dims[2];
    const int dsz = dtype_size(dtype);
    const RowMap rows = row_map(descriptors);
    const size_t plane = (size_t)h * w * dsz;
    const size_t fixed = 256 + ((size_t)L * dsz + 255) / 256 * 256 + 2 * (size_t)rows.nd * L * sizeof(long long);
    const int nbuf = 2 + (host_field ? 1 : 0);
    int64_t S = std::min<int64_t>(slab_planes, d);
    if (device_mem_cap > 0) {
        if (device_mem_cap <= fixed) { set_error("memory cap below the fixed scratch (%zu B)", fixed); return EC_ERR_OOM; }
        const int64_t fit = (int64_t)((device_mem_cap - fixed) / ((size_t)nbuf * plane)) - 2;
        if (fit < 1) { set_error("memory cap too small for a one-plane slab"); return EC_ERR_OOM; }
        S = std::min(S, fit);
    }
    if (S > INT32_MAX / 4) S = INT32_MAX / 4;
    const size_t buf_bytes = (size_t)(S + 2) * plane;
    const size_t total = fixed + (size_t)nbuf * buf_bytes;

    if (!ctx->stream_state) ctx->stream_state = new StreamRes();
    StreamRes &res = *(StreamRes *)ctx->stream_state;
    rc = stream_setup(res);
    if (rc) return rc;
    if (res.mem && (res.bytes < total || (device_mem_cap > 0 && res.bytes > device_mem_cap))) {
        EC_CUDA(cudaStreamSynchronize(res.comp));
        EC_CUDA(cudaStreamSynchronize(res.side));
        cudaFree(res.mem);
        res.mem = nullptr;
        res.bytes = 0;
    }
    if (!res.mem) {
        cudaError_t e = cudaMalloc(&res.mem, total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            res.mem = nullptr;
            set_error("cannot allocate %zu bytes for streaming", total);
            return EC_ERR_OOM;
        }
        res.bytes = total;
    }
    char *base = (char *)res.mem;
    int *flags = (int *)base;
    void *thr_dev = thresholds_host ? (void *)(base + 256) : nullptr;
    long long *hist = (long long *)(base + 256 + ((size_t)L * dsz + 255) / 256 * 256);
    int64_t *out_dev = (int64_t *)(hist + (size_t)rows.nd * L);
    char *bufs = base + fixed;
    EC_CUDA(cudaMemsetAsync(base, 0, fixed, res.comp));
    if (thresholds_host)
        EC_CUDA(cudaMemcpyAsync(thr_dev, thresholds_host, (size_t)L * dsz, cudaMemcpyHostToDevice, res.comp));

    BinArgs ba{L, dtype, thr_dev};
    if (dtype == EC_F32 && L <= kMaxFastL3) {
        // one spacing check per call, not per slab
        rc = launch_uniform_check((const float *)thr_dev, L, flags + 2, res.comp);
        if (rc) return rc;
        ba.uni_ready = 1;
    }
    HistArgs ha{rows, hist, use_smem_hist(rows.nd, L) ? 1 : 0, ctx->hist_schedule};
    ha.planar = ctx->algo == ALGO_AUTO || ctx->algo == ALGO_PLANAR;
    const int64_t nslabs = (d + S - 1) / S;
    for (int64_t i = 0; i < nslabs; i++) {
        const int b = (int)(i % nbuf);
        char *buf = bufs + (size_t)b * buf_bytes;
        const int64_t z0 = i * S, z1 = std::min(z0 + S, d);
        const int64_t n = z1 - z0;   // planes counted; the buffer holds planes z0-1 .. z1
        if (i >= nbuf) EC_CUDA(cudaStreamWaitEvent(res.side, res.freed[b], 0));
        if (host_field) {
            int64_t a = std::max<int64_t>(z0 - 1, 0);
            const int64_t c = std::min<int64_t>(z1 + 1, d);
            if (i > 0) {
                // planes z0-1 and z0 sit at positions S and S+1 of the previous buffer
                const char *prev = bufs + (size_t)((i - 1) % nbuf) * buf_bytes;
                EC_CUDA(cudaMemcpyAsync(buf, prev + (size_t)S * plane, 2 * plane, cudaMemcpyDeviceToDevice, res.side));
                a = z0 + 1;
            }
            if (c > a) {
                const char *src = (const char *)host_field + (size_t)a * plane;
                EC_CUDA(cudaMemcpyAsync(buf + (size_t)(a - (z0 - 1)) * plane, src, (size_t)(c - a) * plane,
                                        cudaMemcpyHostToDevice, res.side));
            }
        } else {
            const int prc = producer(user, z0 - 1, z1 + 1, buf, (void *)res.side);
            if (prc != 0) { set_error("slab producer failed (%d)", prc); return EC_ERR_ARG; }
        }
        EC_CUDA(cudaEventRecord(res.filled[b], res.side));
        EC_CUDA(cudaStreamWaitEvent(res.comp, res.filled[b], 0));
        const int64_t bdims[3] = {n + 2, h, w};
        const int zr[4] = {1, (int)(n + 1), z0 == 0 ? 1 : 0, z1 == d ? (int)(n + 1) : (int)(n + 2)};
        if (ctx->profile && (rc = prof_begin(ctx, res.comp))) return rc;
        rc = EC_ERR_UNSUPPORTED;
        if (connectivity != 6)
            rc = launch_fast_3d(buf, bdims, ba, ha, ctx->tile_z, ctx->grid, ctx->num_sms, flags, res.comp, zr);
        if (rc == EC_ERR_UNSUPPORTED)
            rc = launch_curve_3d(buf, bdims, ba, ha, ALGO_VOXEL, ctx->tile_z, ctx->grid, ctx->num_sms, res.comp, zr,
                                 connectivity == 6 ? 1 : 0);
        if (rc) return rc;
        if (ctx->profile && (rc = prof_end(ctx, res.comp))) return rc;
        EC_CUDA(cudaEventRecord(res.freed[b], res.comp));
    }
    int32_t scale[kMaxDesc];
    row_scales(3, ALGO_VOXEL, descriptors, scale);
    rc = launch_scan(hist, rows.nd, L, scale, out_dev, flags, res.comp);
    if (rc) return rc;
    EC_CUDA(cudaMemcpyAsync(out_host, out_dev, (size_t)rows.nd * L * sizeof(int64_t), cudaMemcpyDeviceToHost,
                            res.comp));
    int hflags[2] = {0, 0};
    EC_CUDA(cudaMemcpyAsync(hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, res.comp));
    EC_CUDA(cudaStreamSynchronize(res.comp));
    if (hflags[0] & 4) { set_error("a bounded device wait gave up"); return EC_ERR_TIMEOUT; }
    return EC_OK;
}

// ------------------------------------------------------------ raw files
//
// Algorithm 1 starts from a raw data file and the low-memory mode of
// Sec. 2.3 reads only what a vertex needs from it.  ec_curve_3d_file streams
// z-slabs straight from such a file: the streaming path above asks for the
// planes of each slab (with its halo planes), the producer below reads them
// with pread into one of two page-locked staging buffers and enqueues their
// copy to the device on the side stream.  A staging buffer is reused only
// after the copy that last read it has finished (an event per buffer), so
// the host reads slab i+1 while the GPU counts slab i.

namespace {

struct FileSlabs {
    int fd = -1;
    int64_t offset = 0, d = 0;
    size_t plane = 0, cap = 0;          // bytes per plane, bytes a staging buffer needs
    FileStaging *st = nullptr;          // the context's staging
    int next = 0;
    int64_t bad_plane = -1;             // first plane whose read failed
    int bad_errno = 0;
    bool staging_failed = false;
    ~FileSlabs()
    {
        if (fd >= 0) close(fd);
    }
};

// Staging of at least f.cap bytes per buffer, events and readers (inside the
// streaming call, under the context's lock).
int file_staging_ready(FileSlabs &f)
{
    FileStaging &st = *f.st;
    for (int i = 0; i < 2; i++)
        if (!st.copied[i] && cudaEventCreateWithFlags(&st.copied[i], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            st.copied[i] = nullptr;
            return 1;
        }
    if (st.cap < f.cap) {
        for (int i = 0; i < 2; i++) {
            if (cudaEventSynchronize(st.copied[i]) != cudaSuccess) return 1;
            if (st.pinned[i]) cudaFreeHost(st.pinned[i]);
            st.pinned[i] = nullptr;
        }
        st.cap = 0;
        for (int i = 0; i < 2; i++)
            if (cudaMallocHost(&st.pinned[i], f.cap) != cudaSuccess) {
                cudaGetLastError();
                st.pinned[i] = nullptr;
                return 1;
            }
        st.cap = f.cap;
    }
    if (!st.pool) st.pool = new ReaderPool((int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
    return 0;
}

int file_producer(void *user, int64_t z0, int64_t z1, void *dst_dev, void *stream)
{
    FileSlabs &f = *(FileSlabs *)user;
    const int64_t a = std::max<int64_t>(z0, 0), b = std::min<int64_t>(z1, f.d);   // halo planes outside are ignored
    if (b <= a) return 0;
    const size_t bytes = (size_t)(b - a) * f.plane;
    if (bytes > f.cap) return 1;
    if (file_staging_ready(f)) { f.staging_failed = true; return 6; }
    FileStaging &st = *f.st;
    const int i = f.next;
    f.next ^= 1;
    if (cudaEventSynchronize(st.copied[i]) != cudaSuccess) return 2;
    // the slab's bytes in equal contiguous parts, one per reader (parts of at
    // least 1 MiB)
    const int nthr = (int)std::max<size_t>(1, std::min<size_t>((size_t)st.pool->size(), bytes >> 20));
    const int64_t base_off = f.offset + a * (int64_t)f.plane;
    std::vector<int64_t> bad(nthr, -1);
    std::vector<int> bad_err(nthr, 0);
    auto read_part = [&](int t) {
        if (t >= nthr) return;
        const size_t b0 = bytes * (size_t)t / (size_t)nthr, b1 = bytes * (size_t)(t + 1) / (size_t)nthr;
        char *p = (char *)st.pinned[i] + b0;
        off_t off = (off_t)(base_off + (int64_t)b0);
        size_t left = b1 - b0;
        while (left > 0) {
            const ssize_t r = pread(f.fd, p, left, off);
            if (r < 0 && errno == EINTR) continue;
            if (r <= 0) {
                bad[t] = a + (int64_t)((b1 - left) / f.plane);
                bad_err[t] = r < 0 ? errno : 0;
                return;
            }
            p += r;
            off += r;
            left -= (size_t)r;
        }
    };
    if (nthr == 1) read_part(0);
    else st.pool->run(read_part);
    for (int t = 0; t < nthr; t++)
        if (bad[t] >= 0) {
            f.bad_plane = bad[t];
            f.bad_errno = bad_err[t];
            return 3;
        }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync((char *)dst_dev + (size_t)(a - z0) * f.plane, st.pinned[i], bytes, cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        return 4;
    if (cudaEventRecord(st.copied[i], s) != cudaSuccess) return 5;
    return 0;
}

}  // namespace

extern "C" int ec_curve_3d_file(ec_ctx *ctx, const char *path, int64_t offset, const int64_t dims[3], int dtype,
                                const void *thresholds_host, int32_t L, int connectivity, uint32_t descriptors,
                                int64_t slab_planes, size_t device_mem_cap, int64_t *out_host)
{
    clear_error();
    if (!ctx) { set_error("ctx is NULL"); return EC_ERR_ARG; }
    if (!path) { set_error("path is NULL"); return EC_ERR_ARG; }
    int rc = validate_request(3, path, dims, dtype, thresholds_host, L, connectivity, descriptors, out_host);
    if (rc) return rc;
    if (offset < 0) { set_error("offset < 0"); return EC_ERR_ARG; }
    if (slab_planes < 1) { set_error("slab_planes must be >= 1"); return EC_ERR_ARG; }
    if (L == 0) return EC_OK;
    FileSlabs f;
    f.fd = open(path, O_RDONLY);
    if (f.fd < 0) { set_error("cannot open %s: %s", path, strerror(errno)); return EC_ERR_ARG; }
    struct stat st;
    if (fstat(f.fd, &st) != 0) { set_error("cannot stat %s: %s", path, strerror(errno)); return EC_ERR_ARG; }
    f.offset = offset;
    f.d = dims[0];
    f.plane = (size_t)dims[1] * (size_t)dims[2] * (size_t)dtype_size(dtype);
    const int64_t need = offset + (int64_t)f.plane * dims[0];
    if ((int64_t)st.st_size < need) {
        set_error("%s holds %lld bytes, the field needs %lld from offset %lld", path, (long long)st.st_size,
                  (long long)need, (long long)offset);
        return EC_ERR_ARG;
    }
    // a slab asks for at most min(slab_planes, d) + 2 planes (halo planes outside the file are not read)
    f.cap = (size_t)(std::min<int64_t>(slab_planes, dims[0]) + 2) * f.plane;
    {
        // the context's staging holder (its buffers are sized inside the call)
        std::lock_guard<std::mutex> lock(ctx->mu);
        if (!ctx->stream_state) ctx->stream_state = new StreamRes();
        StreamRes &res = *(StreamRes *)ctx->stream_state;
        if (!res.file) res.file = new FileStaging();
        f.st = res.file;
    }
    rc = ec_curve_3d_stream(ctx, nullptr, file_producer, &f, dims, dtype, thresholds_host, L, connectivity,
                            descriptors, slab_planes, device_mem_cap, out_host);
    if (rc && f.staging_failed) {
        set_error("cannot allocate %zu bytes of page-locked staging", f.cap);
        return EC_ERR_OOM;
    }
    if (rc && f.bad_plane >= 0) {
        set_error("reading plane %lld of %s failed: %s", (long long)f.bad_plane, path,
                  f.bad_errno ? strerror(f.bad_errno) : "end of file");
        return EC_ERR_ARG;
    }
    return rc;
}


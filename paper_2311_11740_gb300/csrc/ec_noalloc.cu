// ec_noalloc.cu -- ec_curve_3d_noalloc: 3D curves without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs under a memory planner
// which owns every byte of the device (a framework's caching allocator, an
// embedded real-time sensor loop with a fixed budget), or code that must not
// trigger the implicit device synchronisation an allocation can cause in the
// middle of a latency-critical loop.  This entry point gives them the 3D curve
// with no ec_ctx and no allocation: the only scratch it needs (error flags and
// the int64 level histogram) lives in a fixed file-scope device array that
// every GPU loading the library holds until the process exits.
//
// Limits and rules:
//   * popcount(descriptors) * L must not exceed kNoallocHistEntries (65536
//     int64 entries, 512 KiB): e.g. all four descriptors with up to 16384
//     levels.  Larger requests are rejected with EC_ERR_ARG.
//   * All calls share the one array per device; each call clears it first.
//     Calls whose work overlaps on the GPU (two streams, or two host threads)
//     race on it and give wrong curves: serialise them.
//   * The first call on a device looks up the array's device address (with
//     that device current).  With CUDA's lazy module loading that lookup is
//     what loads the library's device code on that device and reserves the
//     array, so the first call may allocate and synchronise implicitly: make
//     one warm-up call per device outside the latency-critical loop and
//     before any stream capture.  Later calls allocate nothing.
//   * Failures on the device (a bounded device wait that gave up) are not
//     turned into a status code: the call does not synchronise, and the
//     affected curve rows read INT64_MIN in every entry.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ec_internal.h"

using namespace ec;

namespace {

constexpr size_t kNoallocFlagBytes = 256;
constexpr size_t kNoallocHistEntries = 65536;
constexpr size_t kNoallocBytes = kNoallocFlagBytes + kNoallocHistEntries * sizeof(long long);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices];
int g_num_sms[kMaxDevices];

// Device address of the scratch array and the SM count for `dev` (the
// current device), looked up once per device.
int setup_device(int dev, void **addr, int *sms)
{
    if (dev < 0 || dev >= kMaxDevices) { set_error("device %d out of range", dev); return EC_ERR_ARG; }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        g_num_sms[dev] = n;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    *sms = g_num_sms[dev];
    return EC_OK;
}

}  // namespace

extern "C" int ec_curve_3d_noalloc(const void *field_dev, const int64_t dims[3], int dtype,
                                   const void *thresholds_dev, int32_t L, int connectivity, uint32_t descriptors,
                                   int64_t *out_dev, void *stream)
{
    clear_error();
    int rc = validate_request(3, field_dev, dims, dtype, thresholds_dev, L, connectivity, descriptors, out_dev);
    if (rc) return rc;
    if (L == 0) return EC_OK;
    const RowMap rows = row_map(descriptors);
    const size_t entries = (size_t)rows.nd * (size_t)L;
    if (entries > kNoallocHistEntries) {
        set_error("request needs %zu histogram entries; the fixed scratch holds %zu "
                  "(popcount(descriptors) * L must be <= %zu)",
                  entries, kNoallocHistEntries, kNoallocHistEntries);
        return EC_ERR_ARG;
    }
    int dev = 0;
    EC_CUDA(cudaGetDevice(&dev));
    void *scratch = nullptr;
    int sms = 0;
    rc = setup_device(dev, &scratch, &sms);
    if (rc) return rc;
    // the launch sequence of ec_curve_3d (reset, histogram kernels, scan) on
    // the fixed array, which has the layout curve_scratch_bytes describes
    static_assert(kNoallocBytes >= kNoallocFlagBytes + kNoallocHistEntries * sizeof(long long), "scratch layout");
    if (curve_scratch_bytes(descriptors, L) > kNoallocBytes) {
        set_error("scratch layout mismatch");
        return EC_ERR_ARG;
    }
    CurvePlan plan;
    plan.algo = ALGO_AUTO;
    plan.num_sms = sms;
    return enqueue_curve(plan, 3, field_dev, dims, dtype, thresholds_dev, L, connectivity, descriptors, out_dev,
                         scratch, (cudaStream_t)stream);
}

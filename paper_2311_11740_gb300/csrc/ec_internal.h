// ec_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/ec.h"

namespace ec {

// Thread-local error reporting behind ec_last_error().
void set_error(const char *fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char *what);
#define EC_CUDA(call)                                               \
    do {                                                            \
        cudaError_t _e = (call);                                    \
        if (_e != cudaSuccess) return ::ec::cuda_fail(_e, #call);   \
    } while (0)

// Descriptor rows of the output, in the order EC, PERIMETER, AREA, VOLUME.
constexpr int kMaxDesc = 4;
struct RowMap {
    int nd;             // number of output rows
    int row[kMaxDesc];  // row index for EC, PER, AREA, VOL, or -1
};
inline RowMap row_map(uint32_t desc)
{
    RowMap r{0, {-1, -1, -1, -1}};
    for (int i = 0; i < kMaxDesc; i++)
        if (desc & (1u << i)) r.row[i] = r.nd++;
    return r;
}

// Everything a histogram kernel needs to turn a raw value into its level.
// Largest level count of the fast paths (paired 16-bit-lane comparisons):
// every key, including the never-active level L, fits a lane below 0x8000.
constexpr int kMaxFastL3 = 32767;

struct BinArgs {
    int32_t L;          // number of levels; bin L = never active
    int dtype;          // EC_U8 / EC_U16 / EC_F32
    const void *thr;    // device thresholds (L values of dtype) or nullptr = identity
    int uni_ready = 0;  // float32: the uniform-spacing check already ran into err_flag[2..4]
};

// Scratch histogram: int64 [nd][L], zeroed before the kernels run.
struct HistArgs {
    RowMap rows;
    long long *hist;    // global int64 [nd][L]
    int smem_hist;      // 1: block-private shared-memory int32 histogram, flushed at the end
    int schedule = 0;   // shared-memory update schedule: 0 auto, 1 one atomic per voxel, 2 warp-aggregated
    int planar = 0;     // 3D per-voxel kernels: count with the planar form (ec_slice.h) where it applies
    int test_give_up = 0;   // testing: every block gives up its first bounded wait (EC_OPT_TEST_GIVE_UP)
};

// Launch helpers implemented in ec_kernels.cu.  All are stream-ordered and
// return EC_OK or an error status.
// conn6 = 1: the EC row under 6-connectivity (voxel_delta_3d6 / Table3D6).
int launch_curve_3d(const void *field, const int64_t dims[3], const BinArgs &ba, const HistArgs &ha,
                    int algo, int tile_z, int grid, int num_sms, cudaStream_t s, const int zrange[4] = nullptr,
                    int conn6 = 0);
int launch_curve_2d(const void *field, const int64_t dims[2], const BinArgs &ba, const HistArgs &ha,
                    int connectivity, int algo, int grid, int num_sms, cudaStream_t s);
// The fast per-voxel 3D kernel (TMA staging, paired comparisons).  Returns
// EC_ERR_UNSUPPORTED without launching when a request does not fit it.
// zrange (optional): {first, end} planes to count and {first, end} planes
// that exist in the field; planes of the buffer outside the latter are read
// as never active (slab halos at the field's ends).
int launch_fast_3d(const void *field, const int64_t dims[3], const BinArgs &ba, const HistArgs &ha, int tile_z,
                   int grid_override, int num_sms, int *err_flag, cudaStream_t s, const int zrange[4] = nullptr);
// Does the planar kernel take this 3D request (dtype, levels, descriptor
// set, row alignment for the tensor map)?
bool planar_3d_supported(const void *field, const int64_t dims[3], int dtype, const void *thr, int32_t L,
                         uint32_t desc);
// The planar-form kernel for fields staged by TMA (float32 with at most 1024
// levels and descriptor sets EC, EC|AREA|VOLUME or all four; uint16 with
// identity levels, EC or EC|VOLUME); EC_ERR_UNSUPPORTED without launching
// for anything else.
int launch_planar_3d(const void *field, const int64_t dims[3], const BinArgs &ba, const HistArgs &ha, int tile_z,
                     int grid_override, int num_sms, int *err_flag, cudaStream_t s, const int zrange[4] = nullptr);
// cuTensorMapEncodeTiled from the driver (nullptr if unavailable).
void *tma_encode_fn();
// The fast per-pixel 2D kernel; EC_ERR_UNSUPPORTED without launching when a
// request does not fit it (more than 32767 levels).
int launch_fast_2d(const void *field, const int64_t dims[2], const BinArgs &ba, const HistArgs &ha, int connectivity,
                   int grid_override, int num_sms, int *err_flag, cudaStream_t s);
// Spacing check of float thresholds for the fast binning (writes uni[0..1]).
int launch_uniform_check(const float *thr, int32_t L, int *uni, cudaStream_t s);
// Running sum over levels and exact division by each row's scale.
int launch_scan(const long long *hist, int nd, int32_t L, const int32_t scale[kMaxDesc],
                int64_t *out, int *err_flag, cudaStream_t s);
int launch_check_sorted(const void *thr, int dtype, int32_t L, int *flag, cudaStream_t s);

// Scale of each descriptor row for an algorithm (1 for the per-top-cell path,
// the table scales for the per-vertex path).
void row_scales(int ndim, int algo, uint32_t desc, int32_t out[kMaxDesc]);

// Shared-memory budget for the block-private histogram.
constexpr size_t kSmemHistBudget = 96 * 1024;
inline bool use_smem_hist(int nd, int32_t L) { return (size_t)nd * ((size_t)L + 1) * 4 <= kSmemHistBudget; }

enum { ALGO_AUTO = 0, ALGO_VOXEL = 1, ALGO_VERTEX = 2, ALGO_PLANAR = 3 };

// Argument checks shared by every curve entry point.
int validate_request(int ndim, const void *field, const int64_t *dims, int dtype, const void *thr, int32_t L,
                     int connectivity, uint32_t descriptors, const int64_t *out);

// Sets the device for a scope and restores the caller's afterwards.
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) switched = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (switched && prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace ec

struct ec_ctx {
    int device = 0;
    int num_sms = 0;
    int algo = ec::ALGO_AUTO;
    int validate = 0;
    int tile_z = 0;
    int grid = 0;
    int profile = 0;
    int hist_schedule = 0;
    void *ws = nullptr;        // device scratch: [flags 256 B][int64 histogram]
    size_t ws_bytes = 0;
    int *host_flag = nullptr;  // pinned, for validation read-back
    std::vector<cudaEvent_t> prof_events;   // start/stop pairs of the main kernel
    size_t prof_used = 0;
    void *batch_state = nullptr;            // ec_batch tables, graph and pinned staging
    void *tune_cache = nullptr;             // autotuned plans per shape class
    void *stream_state = nullptr;           // streaming buffers, streams and events
    int autotune = 0;
    int test_give_up = 0;
    std::mutex mu;
};

namespace ec {
// How to launch one curve request.
struct CurvePlan {
    int algo = ALGO_AUTO;
    int hist_schedule = 0;
    int tile_z = 0;
    int grid = 0;
    int num_sms = 1;
    ec_ctx *prof = nullptr;   // bracket the histogram kernel with this context's events
    int test_give_up = 0;     // EC_OPT_TEST_GIVE_UP
};
// Scratch bytes of one curve request (flags + int64 histogram).
size_t curve_scratch_bytes(uint32_t descriptors, int32_t L);
// Enqueue a validated request on `s` using `scratch` (curve_scratch_bytes).
int enqueue_curve(const CurvePlan &plan, int ndim, const void *field, const int64_t *dims, int dtype,
                  const void *thr, int32_t L, int connectivity, uint32_t descriptors, int64_t *out, void *scratch,
                  cudaStream_t s);
// Grow the context's scratch to at least `bytes` (device-synchronising when it grows).
int ensure_scratch(ec_ctx *ctx, size_t bytes);
// Blocks of `kern` (threads per block, dynamic shared bytes) resident per SM
// on the current device, with the kernel's dynamic shared-memory limit raised
// as needed.  Cached per device, kernel and size (the queries cost host time
// on every small request otherwise).
int kernel_occupancy(const void *kern, int threads, size_t smem, int *occ);
// Autotuner (EC_OPT_AUTOTUNE): fill `plan` from the cache, timing the
// candidate plans on this request first when its shape class is new.
int tuned_plan(ec_ctx *ctx, int ndim, const void *field, const int64_t *dims, int dtype, const void *thr,
               int32_t L, int connectivity, uint32_t desc, int64_t *out, cudaStream_t s, CurvePlan &plan);
void tune_release(ec_ctx *ctx);
// `to` uses (and adds to) the tuned plans of `from` from now on; called with
// from->mu held, before `to` is used.
void tune_share(ec_ctx *from, ec_ctx *to);
// Plans kept by the tuner under other keys (ec_batch's mix classes): three
// integers and the time they took.  Called with ctx->mu held.
bool tune_lookup(ec_ctx *ctx, const std::string &key, int out[3]);
void tune_store(ec_ctx *ctx, const std::string &key, const int v[3], double us);
// Free what ec_batch keeps in a context.
void batch_release(ec_ctx *ctx);
void stream_release(ec_ctx *ctx);
// Kernel timing (EC_OPT_PROFILE): bracket the main histogram kernel of a request.
int prof_begin(ec_ctx *ctx, cudaStream_t s);
int prof_end(ec_ctx *ctx, cudaStream_t s);
}  // namespace ec

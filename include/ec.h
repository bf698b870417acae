/*
 * ec.h -- C ABI of libec: Euler-characteristic, perimeter, area and volume
 * curves of 2D / 3D fields on one NVIDIA GB300 (sm_103a), by vertex
 * contributions (Laky & Zavala, arXiv 2311.11740).
 *
 * Problem statement (Sec. 2): a field of w x h pixels (2D) or w x h x d voxels
 * (3D) is the top-cell layer of a closed cubical complex.  At filtration level
 * t_k the complex holds every top cell with value <= t_k (Eq. sublevel_set)
 * together with all of its faces, edges and vertices.  The EC curve is
 * chi_k = V - E + F - C of that complex (Eq. EC_formula) for every level k.
 * Perimeter, area and volume are the per-vertex descriptors of Tables 1 and 2.
 * The library computes them from per-vertex contributions accumulated into a
 * histogram over levels and prefix-summed (Sec. 2, Algorithms 1-3), exactly,
 * in integers.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every function returns an int status (EC_OK = 0 or an EC_ERR_* code) and
 *    never throws.  ec_last_error() returns a message for the calling thread's
 *    most recent failure.
 *  - Fields are C-contiguous, last dimension fastest: dims = {h, w} (2D) or
 *    {d, h, w} (3D); element [y][x] / [z][y][x].  dims[i] >= 1.
 *  - dtype: EC_U8, EC_U16 or EC_F32.  Thresholds are L values of the field's
 *    type, non-decreasing.  NULL thresholds mean identity levels t_k = k
 *    (integer dtypes only).  A top cell is active at level k iff
 *    value <= t_k compared in the field's type (float32 for EC_F32; a NaN is
 *    never active; -0.0 == +0.0).  1 <= L <= 65535; L == 0 is a no-op.
 *  - descriptors: OR of EC_DESC_*; the output holds popcount(descriptors)
 *    rows of L int64 values, rows ordered EC, PERIMETER, AREA, VOLUME.
 *    Units: EC is the integer Euler characteristic; 2D perimeter counts unit
 *    edges on the boundary of the active set; 2D area counts active pixels;
 *    3D area counts unit faces on the boundary; 3D perimeter is the crease
 *    length (Table 2's "Perimeter" column summed over vertices); volume counts
 *    active voxels.  Cells outside the field are never active.
 *  - connectivity: 2D 8 (the paper's choice, Sec. 2) or 4 (Table 1's 4-C
 *    columns); 3D 26 (the paper's choice) or 6.  Only the EC curve depends
 *    on it.  Under 6-connectivity a cell of the grid is in the complex when
 *    ALL its incident voxels are active, so the EC is #voxels - #face-adjacent
 *    pairs + #2x2 squares - #2x2x2 cubes of the active set (the paper gives a
 *    second connectivity only in 2D; in 2D the same reading is Table 1's 4-C
 *    column).  6-connected requests run on the generic kernels.
 *  - Device pointers (suffix _dev) must be device-accessible on the context's
 *    device.  The caller owns every buffer; the library never frees caller
 *    memory.  Work is ordered on `stream` (a cudaStream_t; NULL = legacy
 *    default stream) and results are valid once the stream has reached the
 *    call's end.  One context's scratch memory serves one call in flight at a
 *    time: give concurrent streams their own contexts.
 */
#ifndef EC_H
#define EC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum ec_status {
    EC_OK = 0,
    EC_ERR_ARG = 1,          /* bad dims, L, pointer, descriptor/connectivity combination, unsorted thresholds */
    EC_ERR_DTYPE = 2,        /* unknown dtype, or NULL thresholds with EC_F32 */
    EC_ERR_UNSUPPORTED = 3,  /* valid request the library does not implement (internal: a kernel that does not fit) */
    EC_ERR_OOM = 4,          /* scratch allocation failed, or a memory cap / budget is too small */
    EC_ERR_CUDA = 5,         /* a CUDA runtime call failed; ec_last_error() has its message */
    EC_ERR_TIMEOUT = 6,      /* a bounded device or host wait gave up */
    EC_ERR_OVERFLOW = 7,     /* an internal counter bound was exceeded (debug check) */
    EC_ERR_BUSY = 8          /* server: no slot or memory free and the queue is full */
};

typedef enum { EC_U8 = 0, EC_U16 = 1, EC_F32 = 2 } ec_dtype;

enum {
    EC_DESC_EC = 1,
    EC_DESC_PERIMETER = 2,
    EC_DESC_AREA = 4,
    EC_DESC_VOLUME = 8       /* 3D only */
};

typedef struct ec_ctx ec_ctx;

/* Message of the calling thread's last failed call ("" if none).  The pointer
 * stays valid until the thread's next ec_* call. */
const char *ec_last_error(void);

/* Create a context on CUDA device `device`: per-device tables, the plan
 * cache and (grown on demand) scratch memory.  *ctx receives the handle. */
int ec_ctx_create(ec_ctx **ctx, int device);
/* Release everything the context owns.  Waits for its device to be idle. */
int ec_ctx_destroy(ec_ctx *ctx);

/* Tuning / checking options (ec_ctx_set_option).
 *  EC_OPT_ALGO: 0 = auto (the fast per-voxel path), 1 = per-voxel regrouped
 *    contributions (one histogram update per top cell), 2 = per-vertex
 *    sorted contributions (Algorithms 1 and 3: sort the 4 or 8 values, add the
 *    type change at each sorted value).  All give identical curves.
 *  EC_OPT_VALIDATE: 1 = check device thresholds are non-decreasing (one
 *    stream synchronisation per call; EC_ERR_ARG if not), 0 = trust them.
 *  EC_OPT_TILE_Z: z planes per work item of the 3D kernels (0 = planner).
 *  EC_OPT_GRID: blocks per launch (0 = planner).
 *  EC_OPT_PROFILE: 1 = bracket the main histogram kernel of every request
 *    with CUDA events on the request's stream (see ec_ctx_profile_read).
 *  EC_OPT_HIST_SCHEDULE: how the fast 3D kernel updates its shared-memory
 *    histogram: 0 = auto, 1 = one atomic per voxel and descriptor,
 *    2 = warp-aggregated (lanes of a warp with the same level are summed
 *    first and one lane per level issues the atomics), 3 = two descriptors
 *    per 32-bit word in two lane-parity copies (half the atomics, fewer
 *    same-address collisions).  All give identical curves.
 *  EC_OPT_AUTOTUNE: 1 = the first request of every shape class (ndim, dtype,
 *    level-count and size buckets, descriptors) times the candidate plans
 *    (tile depth, grid, schedule) on itself, synchronously, and later
 *    requests of the class use the fastest.  ec_batch does the same per mix
 *    class (field count, total cells, share of 3D cells, largest level count,
 *    bucketed): the first batch of a class times its own launch plans (z
 *    planes per 3D work item 16 / 32 / 64, rows per 2D item 32 / 64 / 128,
 *    one or all resident blocks per SM) by coordinate descent.  With the
 *    environment variable EC_AUTOTUNE_CACHE naming a file, tuned plans
 *    persist there as JSON.
 *  EC_OPT_TEST_GIVE_UP (testing the failure path only): 1 = in the next 3D
 *    curve requests on the float32 tensor-map path (the row-copy staging has
 *    no bounded device wait), every block gives up its first
 *    bounded device wait at once, as if the staged plane had not arrived in
 *    time.  The copies already requested still land (the block waits for
 *    them, bounded) before it returns; the curves read INT64_MIN and, with
 *    EC_OPT_VALIDATE, the call returns EC_ERR_TIMEOUT.  0 = normal.        */
enum { EC_OPT_ALGO = 1, EC_OPT_VALIDATE = 2, EC_OPT_TILE_Z = 3, EC_OPT_GRID = 4, EC_OPT_PROFILE = 5,
       EC_OPT_HIST_SCHEDULE = 6, EC_OPT_AUTOTUNE = 7, EC_OPT_TEST_GIVE_UP = 8 };
int ec_ctx_set_option(ec_ctx *ctx, int option, int64_t value);

/* The tuned plan of a shape class, if the autotuner has one:
 * out = {tile_z, grid, schedule}; EC_ERR_ARG when the class is not tuned yet. */
int ec_tuned_plan(ec_ctx *ctx, int32_t ndim, int dtype, int32_t L, uint32_t descriptors, const int64_t *dims,
                  int32_t out[3]);

/* Summed device time (ms) and count of the main histogram kernel launches
 * bracketed since the last read (EC_OPT_PROFILE); waits for the last one to
 * finish, then resets the count. */
int ec_ctx_profile_read(ec_ctx *ctx, double *kernel_ms, int64_t *launches);

/* EC / perimeter / area curves of a 2D field resident on the device.
 * field_dev: h*w values of `dtype`; thresholds_dev: L values of `dtype` or
 * NULL (identity, integer dtypes); out_dev: int64 [popcount(descriptors)][L].
 * Algorithms 1-2 of the paper, Table 1 weights. */
int ec_curve_2d(ec_ctx *ctx, const void *field_dev, const int64_t dims[2], int dtype,
                const void *thresholds_dev, int32_t L, int connectivity,
                uint32_t descriptors, int64_t *out_dev, void *stream);

/* EC / perimeter / area / volume curves of a 3D field resident on the device.
 * Same conventions; dims = {d, h, w}.  Algorithm 3 of the paper (Appendix),
 * Table 2 weights; 26-connectivity (or 6, see the conventions above).
 * Performance note (results do not depend on it): float32 fields with at
 * most 1024 levels whose start is 16-byte aligned run on the fastest kernel,
 * their rows staged by the tensor memory accelerator when the row length is
 * a multiple of 4 and by per-row asynchronous 16-byte copies otherwise
 * (about 1.3x the time per voxel); other fields that start 16-byte aligned
 * are staged by asynchronous 16-byte copies; fields that start unaligned by
 * plain loads (slowest).  The same holds for ec_curve_2d's rows. */
int ec_curve_3d(ec_ctx *ctx, const void *field_dev, const int64_t dims[3], int dtype,
                const void *thresholds_dev, int32_t L, int connectivity,
                uint32_t descriptors, int64_t *out_dev, void *stream);

/* ec_curve_3d for callers that cannot allocate device memory.  The paper has
 * no counterpart to this entry point.  Who needs it: code whose device memory
 * is planned by someone else (a framework's caching allocator, a real-time
 * sensor loop with a fixed budget) and code that must not let an allocation
 * synchronise the device in the middle of a latency-critical loop.  It takes
 * no ec_ctx and calls no allocator: its scratch (flags and the int64 level
 * histogram) is a fixed 512 KiB + 256 B device array inside the library,
 * held by every GPU that loads the library until the process exits.
 * Arguments, layout and results are those of ec_curve_3d.  Limits and rules:
 *  - popcount(descriptors) * L <= 65536 (e.g. all four descriptors with up
 *    to 16384 levels); larger requests return EC_ERR_ARG.
 *  - Every call shares that array and clears it first; calls whose work
 *    overlaps on the GPU (other streams or host threads) race on it and give
 *    wrong curves, so serialise them.
 *  - The first call on a device looks up the array's address with that
 *    device current.  Under CUDA's lazy module loading this lookup loads the
 *    library's device code on that device and reserves the array, so the
 *    first call may allocate and synchronise implicitly: make one warm-up
 *    call per device outside the latency-critical loop and before any stream
 *    capture.  Later calls allocate nothing.
 *  - The call does not synchronise, so failures on the device are not
 *    turned into a status: when a bounded device wait gives up, every entry
 *    of the affected curve rows reads INT64_MIN (a value no curve can take);
 *    check for it if you need to tell such a failure from a real curve.    */
int ec_curve_3d_noalloc(const void *field_dev, const int64_t dims[3], int dtype, const void *thresholds_dev,
                        int32_t L, int connectivity, uint32_t descriptors, int64_t *out_dev, void *stream);

/* Low-memory 3D processing (Sec. 2.3 "Low-Memory Processing"): the field is
 * never resident as a whole.  It is processed in z-slabs of `slab_planes`
 * planes plus one halo plane on each side, with at most `device_mem_cap`
 * bytes of device memory in use by this call (slab buffers, scratch and
 * tables; 0 = no cap).  Slabs come either from `host_field` (a host pointer
 * to the whole d*h*w field; page-locked memory overlaps copies with compute)
 * or, when host_field is NULL, from `producer`, which must enqueue on
 * `stream` the writing of planes [z0, z1) (z0 may be -1 and z1 may be d+1 to
 * ask for halo planes outside the field: fill them with anything, they are
 * ignored) into dst_dev (C-contiguous (z1-z0) x h x w of dtype) and return 0.
 * thresholds_host: L values on the host (or NULL = identity).  out_host:
 * int64 [popcount(descriptors)][L] on the host, written before return (the
 * call is synchronous).  Results are bit-identical to ec_curve_3d.  The slab
 * buffers, their two streams and events stay in the context for the next
 * call (reallocated when a call needs more memory, or when they exceed that
 * call's cap) and are freed by ec_ctx_destroy. */
typedef int (*ec_slab_fn)(void *user, int64_t z0, int64_t z1, void *dst_dev, void *stream);
int ec_curve_3d_stream(ec_ctx *ctx, const void *host_field, ec_slab_fn producer, void *user,
                       const int64_t dims[3], int dtype, const void *thresholds_host,
                       int32_t L, int connectivity, uint32_t descriptors,
                       int64_t slab_planes, size_t device_mem_cap, int64_t *out_host);

/* One field of a batch or a served request. */
typedef struct {
    const void *field;        /* device pointer (ec_batch) or host/device pointer (server) */
    int32_t ndim;             /* 2 or 3 */
    int64_t dims[3];          /* {h, w, 0} or {d, h, w} */
    int32_t dtype;            /* ec_dtype */
    const void *thresholds;   /* device (ec_batch) / host (server) pointer, or NULL = identity */
    int32_t L;
    int32_t connectivity;
    uint32_t descriptors;
    int64_t *out;             /* device (ec_batch) / host (server): [popcount][L] int64 */
} ec_field_desc;

/* Curves of n independent fields of uneven sizes, dtypes and level counts in
 * one persistent-kernel launch (Sec. 4 notes that small images parallelise
 * poorly one at a time), captured in a CUDA graph; 3D fields of at least
 * 2^21 voxels that the fastest 3D kernel takes run as their own launches on
 * parallel branches of the same graph.  All pointers in `fields` are device
 * pointers.  Results are identical to n separate ec_curve_2d / ec_curve_3d
 * calls.
 * With EC_OPT_AUTOTUNE the first batch of a mix class runs several times
 * (synchronously) while its plan is chosen. */
int ec_batch(ec_ctx *ctx, const ec_field_desc *fields, int32_t n, void *stream);

/* The plan the autotuner keeps for the mix class of `fields` (host array of
 * n >= 1 descriptors; only ndim and dims are read): out = {z planes per 3D
 * item, blocks per launch (0 = all resident), rows per 2D item};
 * EC_ERR_ARG when the class is not tuned yet. */
int ec_batch_tuned_plan(ec_ctx *ctx, const ec_field_desc *fields, int32_t n, int32_t out[3]);

/* ----------------------------------------------------- workload generator
 * The hash-box field of the low-memory workload (input generation only):
 * with m the 32-bit finaliser of MurmurHash3, a = m(lo32(seed) ^
 * m(hi32(seed))) and u = m(m(m(a ^ z) ^ y) ^ floor(x/2)) (taken mod 2^32),
 * h(x,y,z) = the low 16 bits of u for even x, its high 16 bits for odd x;
 * v = floor(sum of h over the 5x5x5 box around (x,y,z) / 2000), in
 * [0, 4095], defined for every integer coordinate.  ec_gen_hashbox_u16 writes the nz x ny x nx box with origin
 * (x0, y0, z0) to dst_dev (uint16, C-contiguous) on `stream`.
 * ec_hashbox_producer is an ec_slab_fn: with user -> ec_hashbox_spec it
 * writes planes [z0, z1) of the box (relative to spec->z0) for
 * ec_curve_3d_stream. */
typedef struct { uint64_t seed; int64_t x0, y0, z0, nx, ny; } ec_hashbox_spec;
int ec_gen_hashbox_u16(uint64_t seed, int64_t x0, int64_t y0, int64_t z0, int64_t nx, int64_t ny, int64_t nz,
                       void *dst_dev, void *stream);
int ec_hashbox_producer(void *user, int64_t z0, int64_t z1, void *dst_dev, void *stream);

/* Bytes of scratch memory ec_curve_2d / ec_curve_3d need for a request. */
size_t ec_workspace_bytes(int dtype, int32_t ndim, const int64_t *dims, int32_t L,
                          uint32_t descriptors);

/* ------------------------------------------------------------------ serving
 * A request loop that admits fields while earlier ones are on the GPU
 * (continuous batching): when one of `max_slots` slots is free, the run of
 * queued requests at the head of the queue whose device bytes fit in
 * `device_mem_budget` (at most 256 requests and 64 MiB of fields, or one
 * larger request) is admitted as a group; a group's inputs are copied in,
 * its curves computed by one batched launch (ec_batch) on the slot's own
 * stream and context, and its outputs copied back, so groups overlap on the
 * device.  Under light load a group is a single request.  A request field
 * is a host pointer (copied in) or a device pointer (read in place, not
 * counted in the budget); thresholds and outputs are host pointers.  All
 * must stay valid until the request is done.  When `ctx` has
 * EC_OPT_AUTOTUNE set at creation, the slots tune their groups' mix classes
 * (as ec_batch does) into ctx's plans.                                     */
typedef struct ec_server ec_server;
int ec_server_create(ec_ctx *ctx, size_t device_mem_budget, int32_t max_slots, ec_server **server);
/* Queue a request; *ticket identifies it.  EC_ERR_BUSY if the pending queue
 * is full; EC_ERR_OOM if the request alone exceeds the budget. */
int ec_server_submit(ec_server *server, const ec_field_desc *request, uint64_t *ticket);
/* Queue n requests in order under one lock (a burst from a front end):
 * tickets[i] identifies request i.  All are validated first; if one is
 * malformed (EC_ERR_ARG), exceeds the budget alone (EC_ERR_OOM) or the queue
 * has no room for all (EC_ERR_BUSY), none is queued. */
int ec_server_submit_many(ec_server *server, const ec_field_desc *requests, int32_t n, uint64_t *tickets);
/* *done = 1 once the request finished; *status is its ec_status. */
int ec_server_poll(ec_server *server, uint64_t ticket, int *done, int32_t *status);
/* Block until the request is done or timeout_ms passes (EC_ERR_TIMEOUT). */
int ec_server_wait(ec_server *server, uint64_t ticket, int64_t timeout_ms, int32_t *status);
/* Latency (submit to completion) and timing statistics of finished requests:
 * out[0] = count, out[1] = p50 us, out[2] = p99 us, out[3] = mean us,
 * out[4] = first-submit-to-last-completion us. */
int ec_server_stats(ec_server *server, double out[5]);
/* Block until every request submitted so far is done, or timeout_ms passes
 * (EC_ERR_TIMEOUT). */
int ec_server_wait_all(ec_server *server, int64_t timeout_ms);
/* Forget the statistics of requests finished so far (e.g. after a warm-up). */
int ec_server_reset_stats(ec_server *server);
int ec_server_destroy(ec_server *server);

/* Low-memory 3D processing straight from a raw file (Algorithm 1 reads a raw
 * data file; Sec. 2.3 reads from it only what is needed): the field is the
 * d*h*w values of `dtype` (native byte order, x fastest) stored contiguously
 * from byte `offset` of the file at `path`.  Runs ec_curve_3d_stream with a
 * producer that reads each slab's planes (with its halo planes) by pread into
 * one of two page-locked staging buffers of (min(slab_planes, d) + 2) planes,
 * allocated for the call, and copies them to the device on the streaming
 * side stream; the host reads the next slab while the GPU counts this one.
 * Slabs of 4 MiB or more are read by up to 8 threads.  Other arguments and
 * the result (written to out_host before return) are those of
 * ec_curve_3d_stream.  Errors: EC_ERR_ARG if the file cannot be opened, is
 * shorter than offset + d*h*w*sizeof(dtype), or a read fails (the message
 * names the plane); EC_ERR_OOM if the staging cannot be allocated. */
int ec_curve_3d_file(ec_ctx *ctx, const char *path, int64_t offset, const int64_t dims[3], int dtype,
                     const void *thresholds_host, int32_t L, int connectivity, uint32_t descriptors,
                     int64_t slab_planes, size_t device_mem_cap, int64_t *out_host);

/* ------------------------------------------------------------ BMP input
 * The paper's experiments read their images as BMP files (Sec. 2.3, Table 5).
 * Accepted: uncompressed Windows bitmaps (BITMAPINFOHEADER or later), 8 bits
 * per pixel with a grayscale palette (R = G = B in every entry; a pixel's
 * value is its entry's gray level) or 24 / 32 bits per pixel whose pixels all
 * have R = G = B; rows bottom-up (positive height) or top-down (negative),
 * padded to 4 bytes.  The field is uint8 with row 0 = the image's top row.
 * Errors: EC_ERR_ARG (cannot open, truncated, not a BMP, slices of different
 * sizes), EC_ERR_DTYPE (compressed, other bit depths, colour pixels). */

/* Read a BMP: dims_out = {h, w}; with pixels_host non-NULL also its h*w
 * pixels (caller's buffer).  Host only; no device or context needed. */
int ec_bmp_read(const char *path, int64_t dims_out[2], uint8_t *pixels_host);

/* 2D curves of one BMP image (as ec_curve_2d with dtype EC_U8; thresholds
 * uint8 on the host or NULL for identity levels; out_host int64
 * [popcount(descriptors)][L] on the host, written before return).  Allocates
 * and frees the device copy of the image itself; synchronous. */
int ec_curve_2d_bmp(ec_ctx *ctx, const char *path, const void *thresholds_host, int32_t L, int connectivity,
                    uint32_t descriptors, int64_t *out_host);

/* 3D curves of a stack of BMP slices, paths[z] = the plane z (all of one
 * size), streamed through ec_curve_3d_stream: slabs of slab_planes planes are
 * read into page-locked staging while the GPU counts the previous slab, with
 * at most device_mem_cap bytes of device memory in use (0 = no cap).  The
 * volume is never resident as a whole.  Synchronous; out_host as above. */
int ec_curve_3d_bmp(ec_ctx *ctx, const char *const *paths, int64_t nslices, const void *thresholds_host,
                    int32_t L, int connectivity, uint32_t descriptors, int64_t slab_planes, size_t device_mem_cap,
                    int64_t *out_host);

/* ----------------------------------------------- contribution-type map
 * The paper's full output (Sec. 2, Algorithm 1 and Table 1; Sec. 2.2,
 * Algorithm 3 and Table 2; Sec. 4): how many grid vertices have each
 * contribution type at each level.  A field of h x w pixels has (h+1)(w+1)
 * vertices, one of d x h x w voxels (d+1)(h+1)(w+1); a vertex's type is the
 * class (under the symmetries of the square / cube) of the set of active
 * cells among the 2^n cells around it, cells outside the field never active.
 * Types are numbered by the tables' rows from 0:
 *   2D (EC_NTYPES_2D = 6): Q0 (empty), Q1, Q2 (two pixels sharing an edge),
 *      QD (two diagonal pixels), Q3, Q4;
 *   3D (EC_NTYPES_3D = 22): the rows of Table 2 in printed order, 0 = empty,
 *      21 = all eight voxels (ec_type_table gives the type of every mask).
 * The types do not depend on connectivity; only the weights do. */
#define EC_NTYPES_2D 6
#define EC_NTYPES_3D 22

/* counts_dev: int64 [T][L] on the device, T = EC_NTYPES_2D or _3D;
 * counts[t][k] = number of vertices of type t at level k (active iff the
 * cell's bin is <= k, bins as for ec_curve_2d / ec_curve_3d).  Every column
 * sums to the number of vertices.  ndim = 2 (dims {h, w}) or 3 (dims
 * {d, h, w}); field, dtype, thresholds and L as in ec_curve_2d/3d.  Stream
 * ordered; uses the context's scratch ((T-1) * L * 8 bytes + 256).  With
 * EC_OPT_PROFILE the histogram kernel is timed like a curve request's. */
int ec_type_map(ec_ctx *ctx, int32_t ndim, const void *field_dev, const int64_t *dims, int dtype,
                const void *thresholds_dev, int32_t L, int64_t *counts_dev, void *stream);

/* Weighted curves from a type map (Sec. 4: any descriptor that is a weighted
 * sum of vertex contributions):
 *   out[d][k] = sum_t weights[d][t] * counts[t][k] / scales[d]
 * counts_dev: int64 [ntypes][L] (device); weights_host: int32 [nd][ntypes]
 * (host, row-major); scales_host: int32 [nd] >= 1, or NULL for all 1;
 * out_dev: int64 [nd][L] (device).  1 <= ntypes <= 22, 1 <= nd <= 16.
 * Sums are exact (128-bit); an entry whose sum is not a multiple of its
 * scale, or does not fit int64, is written as INT64_MIN, and with
 * EC_OPT_VALIDATE the call then returns EC_ERR_ARG (it synchronises the
 * stream to find out).  Example: Table 2's columns times 8, 2, 4, 8 with
 * scales {8, 2, 4, 8} give ec_curve_3d's EC, perimeter, area and volume. */
int ec_apply_weights(ec_ctx *ctx, int32_t ntypes, const int64_t *counts_dev, int32_t L, int32_t nd,
                     const int32_t *weights_host, const int32_t *scales_host, int64_t *out_dev, void *stream);

/* Type of every neighbourhood mask (host): ndim 2 -> out[16], ndim 3 ->
 * out[256]; mask bit x + 2y (+ 4z) for the cell at offset (x, y[, z]) in
 * {0,1}^n from the vertex's lower corner, x the fastest field axis. */
int ec_type_table(int32_t ndim, int32_t *out);

/* ---------------------------------------------------- host-side inspection
 * The per-vertex contribution tables the kernels use, derived at build time
 * from the closed-complex rule (Tables 1 and 2 of the paper are what they
 * must reproduce).  2D: out[16][4] = {4*EC(8-C), 4*EC(4-C), 2*perimeter,
 * 4*area} per 4-bit neighbourhood mask (bit x + 2y).  3D: out[256][4] =
 * {8*EC, 2*perimeter, 4*area, 8*volume} per 8-bit mask (bit x + 2y + 4z). */
int ec_vertex_table_2d(int32_t *out);
int ec_vertex_table_3d(int32_t *out);
/* 8 * EC per vertex under 3D 6-connectivity, out[256] per 8-bit mask: the
 * active voxels of the mask, minus 2 per quarter face whose two voxels are
 * active, plus 4 per half edge whose four voxels are active, minus 8 when all
 * eight are.  Constant on every vertex type (ec_type_table), so it is also
 * the 6-connected EC weight row for ec_apply_weights (scale 8). */
int ec_vertex_table_3d_ec6(int32_t *out);
/* Exhaustive host check that the per-top-cell closed forms the fast kernels
 * evaluate equal the per-vertex tables regrouped by entering cell, over all
 * 2^8 (2D) and 2^26 (3D) neighbour precedence patterns.  Returns the number
 * of mismatching patterns (0 = consistent). */
int64_t ec_selfcheck_rules(void);

#ifdef __cplusplus
}
#endif
#endif /* EC_H */

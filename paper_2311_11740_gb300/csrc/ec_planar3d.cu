// ec_planar3d.cu -- the planar-form 3D histogram kernel for fields staged by
// the Tensor Memory Accelerator (the per-voxel changes of ec_slice.h, two
// stacked quads per thread): float32 fields with thresholds, and uint16
// fields with identity levels.
//
// One block of 256 threads owns a 64 x 32 column of voxels and walks it
// along z in work items of `tz` planes.  Per plane:
//   * the TMA copies a box of the plane (float32: 72 x 34 from x0-4; uint16:
//     80 x 34 from x0-8, so every row starts 16-byte aligned; y from y0-1)
//     into a 6-deep shared-memory ring tracked by mbarriers, four planes
//     ahead of use.  Out-of-bounds float elements arrive as NaN, which bins to
//     the never-active level, as cells outside the field; out-of-bounds
//     integers arrive as 0, so items whose box reaches outside the field test
//     coordinates;
//   * every thread bins fixed pairs of values of two staged planes per
//     barrier into a 4-deep ring of 16-bit key planes (float32: spacing guess
//     and one threshold read; uint16: one lane-wise minimum with L);
//   * every thread then handles 8 voxels (x .. x+3 of rows y and y+1): it
//     keeps rows y-1 .. y+2 of two planes in registers, evaluates the layer
//     image of plane s and the minimum image of planes s, s+1 (ec_slice.h,
//     the y pairs between its two rows compared once) and adds each voxel's
//     changes at its level to the block's shared-memory histograms.
// Histogram traffic: the shared-memory pipe is the scarce resource (each
// warp-wide atomic over noisy levels costs about three wavefronts), so with
// the area descriptor the area and volume changes share one 32-bit word per
// level: the low 17 bits add up 6 - nF (the faces a voxel brings, 0..6) and
// the high 15 bits count voxels.  Each word is exchanged to zero and decoded
// into the int32 area and volume rows at every third barrier, so at most 8
// planes of 2048 voxels (16384 voxels) reach it between two exchanges:
// 6 * 16384 < 2^17 and 16384 < 2^15, so neither field overflows.
// Waits on mbarriers are bounded: a wait that gives up sets an error flag,
// waits (bounded) for the block's copies still in flight and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "ec_internal.h"
#include "ec_rules.h"
#include "ec_slice.h"
#include "ec_swar.h"

#include "ec_fast3d.cuh"

namespace ec {

namespace planar3d {

using fast3d::FBin;

constexpr int kThreads = 256;
constexpr int TX = 64, TY = 32;              // voxels per plane of a tile
constexpr int BY = TY + 2;                   // staged rows: y0-1 .. y0+32
constexpr int KP = 36;                       // key row pitch in words (34 pairs + 2)
constexpr int KWORDS = BY * KP;              // words per key plane
constexpr int NS = 6;                        // staged plane ring depth
constexpr int NK = 4;                        // key plane ring depth
constexpr int kPairs = BY * 34;              // key pairs of one plane: 34 rows x 34 (x0-2 .. x0+65)
constexpr int kLeft = kPairs - 32 * 32;      // pairs outside the fixed 4-per-thread shares (132)
static_assert(kLeft == 132 && 2 * kLeft <= 2 * kThreads, "leftover binning shares");

// Staged box per element type: x from x0 - XOFF (a 16-byte aligned start),
// BX elements per row (a multiple of 16 bytes); key pair p of a row is at
// elements XOFF - 2 + 2p.
template <typename T>
constexpr int XOFF() { return 16 / (int)sizeof(T); }
template <typename T>
constexpr int BXT() { return TX + 2 * XOFF<T>(); }
// Row-copy staging (float32 rows that are not a multiple of 16 bytes, which
// a tensor map cannot describe): each staged row is one 16-byte aligned
// bulk copy of RPITCH floats starting at or up to 3 floats before x0 - 4.
constexpr int RPITCH = BXT<float>() + 4;
template <typename T, bool RW = false>
constexpr int SLOT_BYTES()
{
    return RW ? (RPITCH * BY * 4 + 127) / 128 * 128 : (BXT<T>() * BY * (int)sizeof(T) + 127) / 128 * 128;
}
// Levels the shared histograms hold.
template <typename T>
constexpr int LCAP() { return sizeof(T) == 4 ? 1024 : 4096; }
template <typename T>
constexpr int HW() { return LCAP<T>() + 1; }   // words per histogram row (level L = never active)

// shared-memory layout (bytes)
template <typename T, bool RW = false>
constexpr size_t OFF_KEYS() { return (size_t)NS * SLOT_BYTES<T, RW>(); }
template <typename T, bool RW = false>
constexpr size_t OFF_BARS() { return OFF_KEYS<T, RW>() + (size_t)NK * KWORDS * 4; }
template <typename T, bool RW = false>
constexpr size_t OFF_HIST() { return OFF_BARS<T, RW>() + NS * 8 + 16; }
// Histogram rows per descriptor set:
//   EC (1):                  EC
//   EC | VOLUME (9):         EC, volume (one +1 atomic per voxel)
//   EC | AREA | VOLUME (13): EC, packed (free faces, voxels), area, volume
//   all four (15):           the same and perimeter
template <int DM>
constexpr int hist_rows() { return DM == 1 ? 1 : (DM == 9 ? 2 : (DM == 13 ? 4 : 5)); }
template <int DM>
constexpr int R_VOL() { return DM == 9 ? 1 : 3; }
enum { R_EC = 0, R_PACK = 1, R_AREA = 2, R_PER = 4 };
template <typename T, int DM, bool RW = false>
constexpr size_t off_thr() { return OFF_HIST<T, RW>() + (((size_t)hist_rows<DM>() * HW<T>() * 4 + 15) & ~(size_t)15); }
template <typename T, int DM, bool RW = false>
constexpr size_t smem_bytes() { return off_thr<T, DM, RW>() + (sizeof(T) == 4 ? (size_t)LCAP<T>() * 4 : 0); }

struct Params {
    int64_t D, H, W;
    int nbx, nby, nbz, tz;
    int zc0, zc1;          // planes whose voxels are counted
    int zv0, zv1;          // planes that belong to the field (others read as never active)
    int32_t L;
    const float *thr;      // float32 fields: thresholds (uint16 fields: identity levels)
    long long *hist;       // int64 [nd][L]
    int rows[kMaxDesc];
    int *err;              // bit 2: a bounded wait gave up
    const int *uni;        // [0] = 1 if the uniform-spacing guess is exact, [1], [2] = its scale and offset
    int test_give_up;      // testing: give up the first bounded wait of every block
    const float *field;    // row-copy staging: the field (16-byte aligned start) and its element count
    int64_t nelem;
};

struct Ctx {
    unsigned char *ring;       // staged planes
    uint32_t *kring;
    uint64_t *bars;
    volatile int *abort_flag;
    int *err;
    FBin fb;
    int tr, tc;
    uint32_t left0, left1;     // leftover binning pairs: row | pair << 16 | plane << 31, or ~0
    int x0, y0, z0, z1, zv0, zv1;
    int64_t H, W;
    bool edge;                 // the item's staged box reaches outside the field (uint16 and row-copy
                               // staging test coordinates; float32 tensor-map staging reads NaN there)
    const float *field;        // row-copy staging
    int64_t nelem;
    int64_t HW;                // H * W
    int hw4, w4;               // H * W and W mod 4 (a staged row's start phase)
    int Hi, Wi;                // H, W as 32-bit values
    uint32_t emask;            // out_mask bits of this thread's four fixed key pairs on edge items
    uint32_t base;             // ring sequence number of plane z0 - 1
    uint32_t parity;
    uint32_t inflight;         // thread 0: ring slots with a TMA copy issued and not yet waited for
    int give_up;               // thread 0, testing: treat the next wait as timed out
};

__device__ __forceinline__ uint32_t slot_of(const Ctx &c, int plane) { return (c.base + (uint32_t)(plane - (c.z0 - 1))) % NS; }

__device__ __forceinline__ void drain(Ctx &c)
{
    for (int s = 0; s < NS; s++)
        if ((c.inflight >> s) & 1u) {
            fast3d::mbar_wait(&c.bars[s], (c.parity >> s) & 1u, 1000000000ll);
            c.inflight &= ~(1u << s);
        }
}

// Leftover binning share j of a barrier step (two planes of kLeft pairs each).
__device__ __forceinline__ uint32_t left_share(int j)
{
    if (j >= 2 * kLeft) return ~0u;
    const uint32_t plane = j >= kLeft ? 1u : 0u;
    if (j >= kLeft) j -= kLeft;
    int row, pair;
    if (j < 64) { row = j >> 1; pair = 32 + (j & 1); }
    else { row = 32 + (j - 64) / 34; pair = (j - 64) % 34; }
    return (uint32_t)row | ((uint32_t)pair << 16) | (plane << 31);
}

// Cells of key pair (row, pair) outside the field: bit 0 for the pair's
// first cell, bit 1 for its second (coordinates fit in 32 bits).
__device__ __forceinline__ uint32_t out_mask(const Ctx &c, int row, int pair)
{
    const int gy = c.y0 - 1 + row, gx = c.x0 - 2 + 2 * pair;
    const bool yin = gy >= 0 && gy < c.Hi;
    return ((yin && gx >= 0 && gx < c.Wi) ? 0u : 1u) | ((yin && gx + 1 >= 0 && gx + 1 < c.Wi) ? 0u : 2u);
}

// Key pair (row, pair p) of a staged plane.  float32: the spacing guess with
// one threshold read (UNI) or the general search (cells outside the field
// were staged as NaN and bin to L).  uint16 with identity levels: min(v, L)
// per lane; cells outside the field (om, see out_mask) read L (the tensor
// map stages them as 0).
template <typename T, bool UNI>
__device__ __forceinline__ void bin_pair2(const Ctx &c, uint32_t *kp, const T *fp, uint32_t om)
{
    if constexpr (sizeof(T) == 4) {
        const float2 v = *(const float2 *)fp;
        const uint32_t b0 = UNI ? fast3d::fbin_uniform(v.x, c.fb) : fast3d::fbin(v.x, c.fb);
        const uint32_t b1 = UNI ? fast3d::fbin_uniform(v.y, c.fb) : fast3d::fbin(v.y, c.fb);
        *kp = b0 | (b1 << 16);
    } else {
        const uint32_t L = (uint32_t)c.fb.L;
        uint32_t k = vmin2(*(const uint32_t *)fp, L | (L << 16));
        if (om & 1u) k = (k & 0xFFFF0000u) | L;
        if (om & 2u) k = (k & 0x0000FFFFu) | (L << 16);
        *kp = k;
    }
}

// Row-copy staging: key pair p of a staged row whose element x0 - 4 sits r
// floats into the row (the copy starts at the 16-byte boundary at or below
// it); cells outside the field (om) read L.
template <bool UNI>
__device__ __forceinline__ void bin_pair_rw(const Ctx &c, uint32_t *kp, const float *srow, int pair, uint32_t om)
{
    const float *fp = srow + 2 + 2 * pair;
    const float v0 = fp[0], v1 = fp[1];
    const uint32_t L = (uint32_t)c.fb.L;
    uint32_t b0 = UNI ? fast3d::fbin_uniform(v0, c.fb) : fast3d::fbin(v0, c.fb);
    uint32_t b1 = UNI ? fast3d::fbin_uniform(v1, c.fb) : fast3d::fbin(v1, c.fb);
    if (om & 1u) b0 = L;
    if (om & 2u) b1 = L;
    *kp = b0 | (b1 << 16);
}

// Staged row `row` of a row-copy slot, from its element x0 - 4 on: rb is
// the start phase of row 0 ((plane * H + y0 - 1) * W + x0 mod 4).
__device__ __forceinline__ const float *rw_row(const Ctx &c, const float *slot, uint32_t rb, int row)
{
    return slot + row * RPITCH + (int)((rb + (uint32_t)(row * c.w4)) & 3u);
}

template <bool UNI>
__device__ __forceinline__ void bin_plane_rw(const Ctx &c, uint32_t *kp, const float *slot, int plane, uint32_t q)
{
    const int ko = c.tr * KP + c.tc;
    const uint32_t rb = (uint32_t)plane * (uint32_t)c.hw4 + (uint32_t)((c.y0 - 1) * c.w4 + c.x0);
    const float *r0 = rw_row(c, slot, rb, c.tr), *r1 = rw_row(c, slot, rb, c.tr + 16);
    bin_pair_rw<UNI>(c, kp + ko, r0, c.tc, c.emask & 3u);
    bin_pair_rw<UNI>(c, kp + ko + 16, r0, c.tc + 16, (c.emask >> 2) & 3u);
    bin_pair_rw<UNI>(c, kp + ko + 16 * KP, r1, c.tc, (c.emask >> 4) & 3u);
    bin_pair_rw<UNI>(c, kp + ko + 16 * KP + 16, r1, c.tc + 16, (c.emask >> 6) & 3u);
#pragma unroll
    for (int e = 0; e < 2; e++) {
        const uint32_t lv = e ? c.left1 : c.left0;
        if (lv != ~0u && (lv >> 31) == q) {
            const int row = (int)(lv & 0xFFFFu), pair = (int)((lv >> 16) & 0x7FFFu);
            bin_pair_rw<UNI>(c, kp + row * KP + pair, rw_row(c, slot, rb, row), pair,
                             c.edge ? out_mask(c, row, pair) : 0u);
        }
    }
}

// Row-copy staging of plane `plane` (every thread): the 34 staged rows are
// 19 16-byte chunks each, from the 16-byte boundary at or below element
// x0 - 4 of the row (646 chunks, thread t takes chunks t, t + 256, t + 512).
// A chunk is one cp.async; the part of a chunk outside the field's memory is
// zero-filled (those positions lie outside the field and are binned to L).
// Rows and planes outside the field are not read.  The caller closes the
// copies of two planes as one cp.async group.
__device__ __forceinline__ void issue_plane_rw(Ctx &c, int plane)
{
    constexpr int CPR = RPITCH / 4;   // chunks per row
    const uint32_t s = slot_of(c, plane);
    unsigned char *slot = c.ring + (size_t)s * SLOT_BYTES<float, true>();
    if (plane >= c.zv0 && plane < c.zv1) {
        const int64_t pb = (int64_t)plane * c.HW + (c.x0 - 4);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int q = threadIdx.x + k * kThreads;
            if (q < BY * CPR) {
                const int row = q / CPR, ch = q - row * CPR;
                const int gy = c.y0 - 1 + row;
                if (gy >= 0 && gy < c.H) {
                    const int64_t src = ((pb + (int64_t)gy * (int)c.W) & ~(int64_t)3) + 4 * ch;
                    const int64_t left = c.nelem - src;
                    const uint32_t bytes = src < 0 ? 0u : (left >= 4 ? 16u : (uint32_t)(left > 0 ? left * 4 : 0));
                    const float *g = bytes ? c.field + src : c.field;
                    fast3d::cp_async16(fast3d::smem_u32(slot + (size_t)row * RPITCH * 4 + ch * 16), g, bytes);
                }
            }
        }
    }
}

// Bin one staged plane (q = 0: the first of the barrier step, 1: the second):
// rows tr, tr+16 x pairs tc, tc+16, plus this thread's leftover pairs.
template <typename T, bool UNI>
__device__ __forceinline__ void bin_plane(const Ctx &c, uint32_t *kp, const T *fp, uint32_t q)
{
    constexpr int BX = BXT<T>(), F0 = XOFF<T>() - 2;
    const int fo = c.tr * BX + F0 + 2 * c.tc, ko = c.tr * KP + c.tc;
    bin_pair2<T, UNI>(c, kp + ko, fp + fo, c.emask & 3u);
    bin_pair2<T, UNI>(c, kp + ko + 16, fp + fo + 32, (c.emask >> 2) & 3u);
    bin_pair2<T, UNI>(c, kp + ko + 16 * KP, fp + fo + 16 * BX, (c.emask >> 4) & 3u);
    bin_pair2<T, UNI>(c, kp + ko + 16 * KP + 16, fp + fo + 16 * BX + 32, (c.emask >> 6) & 3u);
#pragma unroll
    for (int e = 0; e < 2; e++) {
        const uint32_t lv = e ? c.left1 : c.left0;
        if (lv != ~0u && (lv >> 31) == q) {
            const int row = (int)(lv & 0xFFFFu), pair = (int)((lv >> 16) & 0x7FFFu);
            bin_pair2<T, UNI>(c, kp + row * KP + pair, fp + row * BX + F0 + 2 * pair,
                              c.edge ? out_mask(c, row, pair) : 0u);
        }
    }
}

__device__ __forceinline__ void fill_never(uint32_t *kp, int L)
{
    const uint32_t never = (uint32_t)L | ((uint32_t)L << 16);
    for (int i = threadIdx.x; i < kPairs; i += kThreads) {
        const int row = i / 34, jp = i - row * 34;
        kp[row * KP + jp] = never;
    }
}

template <typename T>
__device__ __forceinline__ void issue_plane(Ctx &c, const CUtensorMap *tmap, int plane)
{
    const uint32_t s = slot_of(c, plane);
    fast3d::mbar_expect_tx(&c.bars[s], BXT<T>() * BY * (uint32_t)sizeof(T));
    fast3d::tma_load_plane(c.ring + (size_t)s * SLOT_BYTES<T>(), tmap, c.x0 - XOFF<T>(), c.y0 - 1, plane, &c.bars[s]);
    c.inflight |= 1u << s;
}

// Barrier step at h = z0 - 4 + t (t even): thread 0 waits for the staged
// planes h+3, h+4; the block synchronises; thread 0 requests planes h+NS+1,
// h+NS+2 into the slots of planes h+1, h+2 (binned at the previous barrier
// step); the block bins planes h+3, h+4.  Returns false if the block must stop.
template <typename T, bool RW>
__device__ __forceinline__ bool barrier_step(Ctx &c, const CUtensorMap *tmap, int h, int L)
{
    if constexpr (RW) {
        // planes h+3, h+4 are the older of this thread's two open groups
        fast3d::cp_async_wait<1>();
    } else if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 3; q <= 4; q++) {
            const int pb = h + q;
            if (pb > c.z1) break;
            const uint32_t s = slot_of(c, pb);
            // (testing) a wait given up at once leaves the copy in flight and
            // its phase unconsumed: the drain below waits for it
            const bool arrived = c.give_up ? false : fast3d::mbar_wait(&c.bars[s], (c.parity >> s) & 1u);
            c.give_up = 0;
            if (!arrived) {
                *c.abort_flag = 1;
                atomicOr(c.err, 4);
                break;
            }
            c.parity ^= 1u << s;
            c.inflight &= ~(1u << s);
        }
    }
    __syncthreads();
    if (!RW && *c.abort_flag) {
        if (threadIdx.x == 0) drain(c);
        return false;
    }
    if (RW || threadIdx.x == 0) {
#pragma unroll
        for (int q = NS + 1; q <= NS + 2; q++) {
            const int pi = h + q;
            if (pi > c.z1) break;
            if constexpr (RW) issue_plane_rw(c, pi);
            else issue_plane<T>(c, tmap, pi);
        }
        if constexpr (RW) fast3d::cp_async_commit();   // one group per barrier step, possibly empty
    }
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int pb = h + 3 + q;
        if (pb > c.z1) break;
        uint32_t *kp = c.kring + (uint32_t)(pb & (NK - 1)) * KWORDS;
        if (pb < c.zv0 || pb >= c.zv1) {
            fill_never(kp, L);
        } else if constexpr (RW) {
            const float *fp = (const float *)(c.ring + (size_t)slot_of(c, pb) * SLOT_BYTES<float, true>());
            if (c.fb.uniform) bin_plane_rw<true>(c, kp, fp, pb, (uint32_t)q);
            else bin_plane_rw<false>(c, kp, fp, pb, (uint32_t)q);
        } else {
            const T *fp = (const T *)(c.ring + (size_t)slot_of(c, pb) * SLOT_BYTES<T>());
            if (sizeof(T) != 4 || c.fb.uniform) bin_plane<T, true>(c, kp, fp, (uint32_t)q);
            else bin_plane<T, false>(c, kp, fp, (uint32_t)q);
        }
    }
    return true;
}

// Rows y-1 .. y+2 of key plane `plane` around this thread's quads.
__device__ __forceinline__ void load_rows(const Ctx &c, int plane, Row5 (&W)[4])
{
    const uint32_t *kp = c.kring + (uint32_t)(plane & (NK - 1)) * KWORDS + (2 * c.tr) * KP + 2 * c.tc;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const uint2 a = *(const uint2 *)(kp + r * KP), b = *(const uint2 *)(kp + r * KP + 2);
        W[r].a = __byte_perm(a.x, a.y, 0x5432);   // keys x-1, x
        W[r].b = a.y;                             // x, x+1
        W[r].c = __byte_perm(a.y, b.x, 0x5432);   // x+1, x+2
        W[r].d = b.x;                             // x+2, x+3
        W[r].e = __byte_perm(b.x, b.y, 0x5432);   // x+3, x+4
    }
}

// Add one quad's changes at its levels (key pairs kb = voxels 0, 1 and
// kd = voxels 2, 3).  SKIP (items whose counted box reaches past the field):
// voxels at the never-active level L are left out.  Their changes belong to
// the discarded level L, and outside the field they would all hit the same
// word and serialise the warp's atomics.
template <typename T, int DM, bool SKIP>
__device__ __forceinline__ void add_quad(int *h, uint32_t kb, uint32_t kd, const SliceOut &o, uint32_t L)
{
    constexpr int hw = HW<T>();
    const uint32_t key[4] = {kb & 0xFFFFu, kb >> 16, kd & 0xFFFFu, kd >> 16};
    const int ecv[4] = {sbyte<0>(o.ec), sbyte<1>(o.ec), sbyte<2>(o.ec), sbyte<3>(o.ec)};
#pragma unroll
    for (int v = 0; v < 4; v++) {
        if (SKIP && key[v] >= L) continue;
        int *const e = h + key[v];
        atomicAdd(e + R_EC * hw, ecv[v]);
        if (DM & 4) {
            // free faces (byte v of o.area, 0..6) plus one voxel at bit 17
            const uint32_t w = __byte_perm(o.area, 0x00020000u, 0x7650u + (uint32_t)v);
            atomicAdd((unsigned int *)(e + R_PACK * hw), w);
        } else if (DM & 8) {
            atomicAdd(e + R_VOL<DM>() * hw, 1);
        }
        if (DM & 2) {
            const int pv[4] = {sbyte<0>(o.per), sbyte<1>(o.per), sbyte<2>(o.per), sbyte<3>(o.per)};
            atomicAdd(e + R_PER * hw, pv[v]);
        }
    }
}

// Exchange the packed (free faces, voxels) words of this thread's levels to
// zero and add them into the area and volume rows.
template <typename T>
__device__ __forceinline__ void flush_packed(int *h, int L)
{
    constexpr int hw = HW<T>();
    for (int k = threadIdx.x; k <= L; k += kThreads) {
        const uint32_t w = atomicExch((unsigned int *)(h + R_PACK * hw + k), 0u);
        if (w) {
            const int n = (int)(w >> 17), f = (int)(w & 0x1FFFFu);
            h[R_AREA * hw + k] += 2 * f - 6 * n;
            h[3 * hw + k] += n;
        }
    }
}

template <typename T, int DM, bool SKIP>
__device__ __forceinline__ void half_step(Ctx &c, int *hist, Row5 (&P)[4], Row5 (&Q)[4], SliceState &sa,
                                          SliceState &sb, int h, uint32_t L)
{
    constexpr bool PER = (DM & 2) != 0;
    if (h >= c.z0 - 2) load_rows(c, h + 1, Q);
    if (h == c.z0 - 1) {
        slice_pair_begin<PER>(P, Q, sa, sb);
    } else if (h >= c.z0) {
        SliceOut oa, ob;
        slice_pair<(DM & 4) ? AREA_FREE_FACES : AREA_NONE, PER>(P, Q, sa, sb, oa, ob);
        add_quad<T, DM, SKIP>(hist, P[1].b, P[1].d, oa, L);
        add_quad<T, DM, SKIP>(hist, P[2].b, P[2].d, ob, L);
    }
}

// The plane walk of one item (z0-4 .. z1-1 in barrier steps of two planes).
// False when a bounded wait gave up (the block then returns).
template <typename T, int DM, bool SKIP, bool RW>
__device__ __forceinline__ bool walk_item(Ctx &c, const CUtensorMap *tmap, int *hist, Row5 (&W0)[4],
                                          Row5 (&W1)[4], SliceState &sa, SliceState &sb, uint32_t &nbar, int L)
{
    const int nsteps = c.z1 - c.z0 + 4;
    for (int t = 0; t < nsteps; t += 2) {
        const int h = c.z0 - 4 + t;
        if (!barrier_step<T, RW>(c, tmap, h, L)) return false;
        if (DM & 4) {
            if (++nbar == 3) {
                nbar = 0;
                flush_packed<T>(hist, L);
            }
        }
        half_step<T, DM, SKIP>(c, hist, W0, W1, sa, sb, h, (uint32_t)L);
        if (t + 1 < nsteps) half_step<T, DM, SKIP>(c, hist, W1, W0, sa, sb, h + 1, (uint32_t)L);
    }
    return true;
}

template <typename T, int DM, bool RW>
__global__ void __launch_bounds__(kThreads, 2) k_planar3d(const __grid_constant__ CUtensorMap tmap, Params p)
{
    constexpr int hw = HW<T>();
    extern __shared__ __align__(128) unsigned char smem[];
    Ctx c;
    c.ring = smem;
    c.kring = (uint32_t *)(smem + OFF_KEYS<T, RW>());
    c.bars = (uint64_t *)(smem + OFF_BARS<T, RW>());
    c.abort_flag = (volatile int *)(smem + OFF_BARS<T, RW>() + NS * 8);
    c.err = p.err;
    c.field = p.field;
    c.nelem = p.nelem;
    c.HW = p.H * p.W;
    c.hw4 = (int)(c.HW & 3);
    c.w4 = (int)(p.W & 3);
    c.Hi = (int)p.H;
    c.Wi = (int)p.W;
    int *const hist = (int *)(smem + OFF_HIST<T, RW>());
    const int L = p.L;
    for (int i = threadIdx.x; i < hist_rows<DM>() * hw; i += kThreads) hist[i] = 0;
    c.fb = FBin{};
    c.fb.L = L;
    if constexpr (sizeof(T) == 4) {
        float *const thr = (float *)(smem + off_thr<T, DM, RW>());
        for (int k = threadIdx.x; k < L; k += kThreads) thr[k] = p.thr[k];
        c.fb.t = thr;
        c.fb.t0 = p.thr[0];
        c.fb.tl = p.thr[L - 1];
        c.fb.inv = (L > 1 && c.fb.tl > c.fb.t0) ? (float)(L - 1) / (c.fb.tl - c.fb.t0) : 0.f;
        c.fb.lm1 = (float)(L - 1);
        c.fb.off = 0.f;
        c.fb.uniform = 0;
        if (p.uni[0]) {
            c.fb.uniform = 1;
            c.fb.inv = __int_as_float(p.uni[1]);
            c.fb.off = __int_as_float(p.uni[2]);
        }
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; i++) fast3d::mbar_init(&c.bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *c.abort_flag = 0;
    }
    __syncthreads();

    c.tr = threadIdx.x >> 4;
    c.tc = threadIdx.x & 15;
    c.left0 = left_share(threadIdx.x);
    c.left1 = left_share(threadIdx.x + kThreads);
    c.parity = 0;
    c.inflight = 0;
    c.give_up = p.test_give_up;
    c.zv0 = p.zv0;
    c.zv1 = p.zv1;
    c.H = p.H;
    c.W = p.W;
    uint32_t seq = 0;
    uint32_t nbar = 0;   // barrier steps since the packed words were last exchanged
    const int nitems = p.nbx * p.nby * p.nbz;
    Row5 W0[4], W1[4];
    SliceState sa{}, sb{};

    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % p.nbx, by = (item / p.nbx) % p.nby, bz = item / (p.nbx * p.nby);
        c.x0 = bx * TX;
        c.y0 = by * TY;
        c.z0 = p.zc0 + bz * p.tz;
        c.z1 = min(c.z0 + p.tz, p.zc1);
        // binned cells x0-2 .. x0+65, y0-1 .. y0+32
        c.edge = c.x0 < 2 || c.x0 + 66 > p.W || c.y0 < 1 || c.y0 + 33 > p.H;
        c.emask = 0;
        if (c.edge && (sizeof(T) == 2 || RW))
            c.emask = out_mask(c, c.tr, c.tc) | out_mask(c, c.tr, c.tc + 16) << 2 |
                      out_mask(c, c.tr + 16, c.tc) << 4 | out_mask(c, c.tr + 16, c.tc + 16) << 6;
        __syncthreads();   // the previous item is done with both rings
        c.base = seq;
        if constexpr (RW) {
            // planes z0-1, z0 and z0+1, z0+2 as two groups
            for (int q = 0; q < NS - 2; q++) {
                const int pz = c.z0 - 1 + q;
                if (pz <= c.z1) issue_plane_rw(c, pz);
                if (q & 1) fast3d::cp_async_commit();
            }
        } else if (threadIdx.x == 0) {
            for (int q = 0; q < NS - 2; q++) {
                const int pz = c.z0 - 1 + q;
                if (pz > c.z1) break;
                issue_plane<T>(c, &tmap, pz);
            }
        }
        // counted voxels x0 .. x0+63, y0 .. y0+31: past the field's edge the
        // walk leaves out voxels at level L
        const bool skip = c.x0 + TX > p.W || c.y0 + TY > p.H;
        const bool ok = skip ? walk_item<T, DM, true, RW>(c, &tmap, hist, W0, W1, sa, sb, nbar, L)
                             : walk_item<T, DM, false, RW>(c, &tmap, hist, W0, W1, sa, sb, nbar, L);
        if (!ok) return;
        seq += (uint32_t)(c.z1 - c.z0 + 2);
    }
    __syncthreads();
    if (DM & 4) {
        flush_packed<T>(hist, L);
        __syncthreads();
    }
    // global rows are [nd][L] in the order EC, PER, AREA, VOL; level L is dropped
    for (int k = threadIdx.x; k < L; k += kThreads) {
        long long *g = p.hist;
        int v = hist[R_EC * hw + k];
        if (v) atomicAdd((unsigned long long *)&g[(size_t)p.rows[0] * L + k], (unsigned long long)(long long)v);
        if (DM & 2) {
            v = hist[R_PER * hw + k];
            if (v) atomicAdd((unsigned long long *)&g[(size_t)p.rows[1] * L + k], (unsigned long long)(long long)v);
        }
        if (DM & 4) {
            v = hist[R_AREA * hw + k];
            if (v) atomicAdd((unsigned long long *)&g[(size_t)p.rows[2] * L + k], (unsigned long long)(long long)v);
        }
        if (DM & 8) {
            v = hist[R_VOL<DM>() * hw + k];
            if (v) atomicAdd((unsigned long long *)&g[(size_t)p.rows[3] * L + k], (unsigned long long)(long long)v);
        }
    }
}

// Item depth when the caller leaves it to the planner: the depth in 16..128
// that minimises the planes the busiest block walks, (items per block,
// rounded up) x (depth + the 4-step ramp of each item), for a grid of
// `grid` blocks over columns x planes.
static int plan_tile_z(int64_t columns, int planes, int grid)
{
    int best = 64;
    int64_t best_cost = INT64_MAX;
    for (int tz = 16; tz <= 128; tz++) {
        const int64_t nbz = (planes + tz - 1) / tz;
        const int depth = (int)((planes + nbz - 1) / nbz);
        const int64_t per_block = (columns * nbz + grid - 1) / grid;
        const int64_t cost = per_block * (depth + 4);
        if (cost < best_cost) { best_cost = cost; best = tz; }
    }
    return best;
}

template <typename T, int DM, bool RW = false>
static int launch_dm(const CUtensorMap &map, Params p, int tile_z, int num_sms, int grid_override, cudaStream_t s)
{
    auto kern = k_planar3d<T, DM, RW>;
    const size_t smem = smem_bytes<T, DM, RW>();
    int occ = 0;
    if (const int orc = kernel_occupancy((const void *)kern, kThreads, smem, &occ)) return orc;
    if (occ < 1) { set_error("planar 3D kernel does not fit (%zu B shared)", smem); return EC_ERR_UNSUPPORTED; }
    int grid = grid_override > 0 ? grid_override : num_sms * occ;
    const int planes = p.zc1 - p.zc0;
    const int64_t columns = (int64_t)p.nbx * p.nby;
    p.tz = tile_z > 0 ? tile_z : plan_tile_z(columns, planes, grid);
    p.nbz = (planes + p.tz - 1) / p.tz;
    const int64_t items64 = columns * p.nbz;
    if (items64 > INT32_MAX) return EC_ERR_UNSUPPORTED;
    grid = grid > items64 ? (int)items64 : grid;
    kern<<<grid, kThreads, smem, s>>>(map, p);
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

}  // namespace planar3d

// The planar kernel for fields the TMA can stage (start 16-byte aligned, rows
// a multiple of 16 bytes): float32 with thresholds, at most 1024 levels and
// the descriptor sets EC, EC|AREA|VOLUME or all four; uint16 with identity
// levels, at most 4096 levels and EC or EC|VOLUME.  Returns
// EC_ERR_UNSUPPORTED (without launching) for anything else.
bool planar_3d_supported(const void *field, const int64_t dims[3], int dtype, const void *thr, int32_t L,
                         uint32_t desc)
{
    using namespace planar3d;
    const bool f32 = dtype == EC_F32 && thr && L >= 1 && L <= LCAP<float>() &&
                     (desc == 1u || desc == 13u || desc == 15u);
    const bool u16 = dtype == EC_U16 && !thr && L >= 1 && L <= LCAP<uint16_t>() && (desc == 1u || desc == 9u);
    if (!f32 && !u16) return false;
    if (((uintptr_t)field % 16) != 0 || dims[0] > INT32_MAX / 2 || dims[1] > INT32_MAX / 2 ||
        dims[2] > INT32_MAX / 2)
        return false;
    // float32 rows of any width (tensor map, or row copies when a row is not
    // a multiple of 16 bytes); uint16 rows through the tensor map only
    return f32 || (dims[2] * 2) % 16 == 0;
}

int launch_planar_3d(const void *field, const int64_t dims[3], const BinArgs &ba, const HistArgs &ha, int tile_z,
                     int grid_override, int num_sms, int *err_flag, cudaStream_t s, const int zrange[4])
{
    using namespace planar3d;
    uint32_t desc = 0;
    for (int i = 0; i < kMaxDesc; i++)
        if (ha.rows.row[i] >= 0) desc |= 1u << i;
    if (!planar_3d_supported(field, dims, ba.dtype, ba.thr, ba.L, desc)) return EC_ERR_UNSUPPORTED;
    const bool f32 = ba.dtype == EC_F32;
    const int esz = f32 ? 4 : 2;
    const bool rw = f32 && (dims[2] * 4) % 16 != 0;   // row copies instead of the tensor map
    PFN_cuTensorMapEncodeTiled_v12000 enc = (PFN_cuTensorMapEncodeTiled_v12000)tma_encode_fn();
    if (!enc && !rw) return EC_ERR_UNSUPPORTED;
    Params p{};
    p.D = dims[0]; p.H = dims[1]; p.W = dims[2];
    p.zc0 = zrange ? zrange[0] : 0;
    p.zc1 = zrange ? zrange[1] : (int)p.D;
    p.zv0 = zrange ? zrange[2] : 0;
    p.zv1 = zrange ? zrange[3] : (int)p.D;
    p.nbx = (int)((p.W + TX - 1) / TX);
    p.nby = (int)((p.H + TY - 1) / TY);
    if (p.zc1 <= p.zc0) return EC_OK;
    p.L = ba.L;
    p.thr = f32 ? (const float *)ba.thr : nullptr;
    p.hist = ha.hist;
    for (int i = 0; i < kMaxDesc; i++) p.rows[i] = ha.rows.row[i];
    p.err = err_flag;
    p.uni = err_flag + 2;
    p.test_give_up = ha.test_give_up;
    p.field = (const float *)field;
    p.nelem = dims[0] * dims[1] * dims[2];
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    if (rw) {
        if (!ba.uni_ready) {
            const int rc = launch_uniform_check((const float *)ba.thr, ba.L, err_flag + 2, s);
            if (rc) return rc;
        }
        if (desc == 1u) return launch_dm<float, 1, true>(map, p, tile_z, num_sms, grid_override, s);
        if (desc == 13u) return launch_dm<float, 13, true>(map, p, tile_z, num_sms, grid_override, s);
        return launch_dm<float, 15, true>(map, p, tile_z, num_sms, grid_override, s);
    }
    cuuint64_t gdim[3] = {(cuuint64_t)p.W, (cuuint64_t)p.H, (cuuint64_t)p.D};
    cuuint64_t gstride[2] = {(cuuint64_t)(p.W * esz), (cuuint64_t)(p.W * p.H * esz)};
    cuuint32_t box[3] = {(cuuint32_t)(f32 ? BXT<float>() : BXT<uint16_t>()), (cuuint32_t)BY, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    // float32: out-of-bounds elements read NaN (never active); uint16: zero,
    // replaced by L through the edge items' coordinate test
    CUresult r = enc(&map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
                     const_cast<void *>(field), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     f32 ? CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA : CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return EC_ERR_UNSUPPORTED;
    if (f32) {
        if (!ba.uni_ready) {
            const int rc = launch_uniform_check((const float *)ba.thr, ba.L, err_flag + 2, s);
            if (rc) return rc;
        }
        if (desc == 1u) return launch_dm<float, 1>(map, p, tile_z, num_sms, grid_override, s);
        if (desc == 13u) return launch_dm<float, 13>(map, p, tile_z, num_sms, grid_override, s);
        return launch_dm<float, 15>(map, p, tile_z, num_sms, grid_override, s);
    }
    if (desc == 1u) return launch_dm<uint16_t, 1>(map, p, tile_z, num_sms, grid_override, s);
    return launch_dm<uint16_t, 9>(map, p, tile_z, num_sms, grid_override, s);
}

}  // namespace ec

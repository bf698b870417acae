// ec_fast3d.cuh -- device building blocks of the fast per-voxel 3D path,
// shared by the single-field kernel (ec_fast3d.cu) and the batched
// persistent kernel (ec_batch.cu).  See ec_fast3d.cu for the data flow.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ec_internal.h"
#include "ec_rules.h"
#include "ec_slice.h"
#include "ec_swar.h"

namespace ec {

namespace fast3d {

constexpr int kThreads = 256;
constexpr int TXF = 64, TYF = 16;           // voxels per plane of a tile
constexpr int BX = TXF + 8, BY = TYF + 2;   // staged box: x0-4 .. x0+67, y0-1 .. y0+16
constexpr int KP = 36;                      // key row pitch in 32-bit words (even: 8-byte row loads)
constexpr int KWORDS = BY * KP;             // words per key plane
constexpr int NS = 8;                       // float plane ring depth (TMA path)
constexpr int NK = 4;                       // key plane ring depth
constexpr int kThrSmem = 4096;
constexpr int kPairsPerPlane = BY * (BX - 4) / 2;   // key pairs j = 2..69 of 18 rows
constexpr int KAP = 3;                      // planes copied ahead by the one-plane cp.async walk (ec_batch)
constexpr int NRAWP = KAP + 2;              // its raw plane ring: plane being binned, waited, KAP in flight
constexpr int NRAWP2 = 6;                   // raw plane ring of the two-plane cp.async walk: 2 binned, 4 in flight

// Raw plane of the asynchronous path: rows y0-1 .. y0+16, each with the
// tile's 64 voxels and A elements (16 bytes) of halo on each side, so every
// 16-byte chunk starts aligned.
template <typename T>
constexpr int rpad() { return 16 / (int)sizeof(T); }
template <typename T>
constexpr int rrow_bytes() { return (TXF + 2 * rpad<T>()) * (int)sizeof(T); }
template <typename T>
constexpr int rplane_bytes() { return BY * rrow_bytes<T>(); }
// Staging kinds of the cp.async path: STG_ALIGNED, rows start 16-byte
// aligned and a row slot holds x0-A .. x0+63+A; STG_COVER, rows of any
// width (field start 16-byte aligned) and a row slot holds the 16-byte
// aligned cover of the row's in-field part of x0-2 .. x0+65 (at most
// 68 * sizeof(T) + 15 bytes: the same slot size).
enum { STG_ALIGNED = 0, STG_COVER = 1 };

struct Params {
    const void *field;
    int64_t D, H, W;
    int nbx, nby, nbz, tz;
    int zc0, zc1;          // planes whose voxels are counted
    int zv0, zv1;          // planes that belong to the field (others read as never active)
    int32_t L;
    const void *thr;
    long long *hist;       // int64 [nd][L]
    int rows[kMaxDesc];
    int nd;
    int smem_hist;
    int *err;              // bit 2: a bounded wait gave up
    const int *uni;        // [0] = 1 if the uniform-spacing guess is exact, [1], [2] = its scale and offset (float bits)
    int agg;               // 1: warp-aggregated shared-memory updates (lanes grouped by level)
    int pairs;             // 1: two descriptors per 32-bit word, two lane-parity copies (see PairHist)
    int planar;            // 1: count with the planar form (ec_slice.h); needs the shared histogram
};

// ------------------------------------------------------------- mbarriers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity: gives up after `limit`
// clock cycles (default: about two seconds).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = 4000000000ll)
{
    const uint32_t addr = smem_u32(bar);
    const long long t0 = clock64();
    for (uint32_t it = 0; it < (1u << 26); it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) break;
    }
    return false;
}

__device__ __forceinline__ void tma_load_plane(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------- binning

struct FBin {
    const float *t;
    float t0, tl, inv;
    float off, lm1;   // uniform guess: offset -t0 * inv and L - 1
    int L;
    int uniform;      // the guess below is always the bin or the bin minus one
};

// Parameters of the uniform-spacing guess, from the first and last threshold.
__device__ __forceinline__ void guess_params(float t0, float tl, int L, float &inv, float &off)
{
    inv = (L > 1 && tl > t0) ? (float)(L - 1) / (tl - t0) : 0.f;
    off = -__fmul_rn(t0, inv);
}

// Guess of the bin of x from the spacing of the thresholds: the nearest
// integer to x * inv - t0 * inv, clamped to [0, L-1] (NaN lands on L-1).
// For x in (t_{k-1}, t_k] of near-uniform thresholds this is k-1 or k.  The
// pre-check and the binning call this same function, with explicit
// round-to-nearest operations, so the two agree bit for bit.  fminf sends
// NaN to L-1; the saturating round-to-nearest conversion clamps negative
// values to 0.
__device__ __forceinline__ int bin_guess(float x, float inv, float off, float lm1)
{
    const float y = fminf(__fmaf_rn(x, inv, off), lm1);
    uint32_t g;
    asm("cvt.rni.sat.u32.f32 %0, %1;" : "=r"(g) : "f"(y));
    return (int)g;
}

// Is the guess the bin or the bin minus one for every x whose bin is k?  The
// guess is monotone in x, so both ends of the level's interval (t_{k-1}, t_k]
// decide (k = 0: (-inf, t_0]; k = L: the values above t_{L-1}).
__device__ __forceinline__ bool guess_ok_for_level(const float *t, int L, int k, float inv, float off)
{
    const float lm1 = (float)(L - 1);
    if (k == 0) return t[0] == t[0] && bin_guess(t[0], inv, off, lm1) <= 0;
    const float lo = t[k - 1];
    if (lo != lo) return false;
    if (k == L) return !(lo < INFINITY) || bin_guess(nextafterf(lo, INFINITY), inv, off, lm1) >= L - 1;
    const float hi = t[k];
    if (hi != hi) return false;
    if (!(lo < hi)) return true;   // empty interval
    return bin_guess(nextafterf(lo, INFINITY), inv, off, lm1) >= k - 1 && bin_guess(hi, inv, off, lm1) <= k;
}

// Exact bin when the guess is known to be the bin or the bin minus one:
// one threshold read and one comparison (NaN: guess L-1, comparison false -> L).
__device__ __forceinline__ uint32_t fbin_uniform(float x, const FBin &b)
{
    const int g = bin_guess(x, b.inv, b.off, b.lm1);
    return (uint32_t)(g + (x <= b.t[g] ? 0 : 1));
}

__device__ __forceinline__ uint32_t bsearch_f(float x, const float *t, int lo, int hi)
{
    // first k in [lo, hi) with x <= t[k]; hi if none
    int n = hi - lo;
    while (n > 0) {
        const int half = n >> 1;
        if (!(x <= t[lo + half])) { lo += half + 1; n -= half + 1; }
        else n = half;
    }
    return (uint32_t)lo;
}

__device__ __forceinline__ uint32_t fbin(float x, const FBin &b)
{
    if (!(x <= b.tl)) return (uint32_t)b.L;      // NaN or above every threshold
    if (x <= b.t0) return 0u;
    int k = (int)((x - b.t0) * b.inv);
    k = min(max(k, 0), b.L - 1);
    if (x <= b.t[k]) {
        if (k == 0 || !(x <= b.t[k - 1])) return (uint32_t)k;
        return bsearch_f(x, b.t, 0, k - 1);
    }
    if (x <= b.t[k + 1]) return (uint32_t)(k + 1);   // k + 1 <= L - 1 because x <= t[L-1]
    return bsearch_f(x, b.t, k + 2, b.L - 1);
}

template <typename T>
struct IBin {
    const T *t;        // thresholds or nullptr (identity)
    const uint16_t *table;
    int L;
    __device__ __forceinline__ uint32_t operator()(T v) const
    {
        if constexpr (sizeof(T) == 1) {
            return table[v];
        } else {
            if (!t) return v < (uint32_t)L ? (uint32_t)v : (uint32_t)L;
            int lo = 0, n = L;
            while (n > 0) {
                const int half = n >> 1;
                if (t[lo + half] < v) { lo += half + 1; n -= half + 1; }
                else n = half;
            }
            return (uint32_t)lo;
        }
    }
};

// ----------------------------------------------------------------- kernel

constexpr int FSTRIDE = ((BX * BY * 4 + 127) / 128) * 128 / 4;   // float slot stride (128-byte aligned)

template <typename T>
struct Ctx {
    Params p;
    float *fring;
    unsigned char *raw;        // raw plane ring (asynchronous plain-load path)
    uint32_t *kring;
    uint64_t *bars;
    volatile int *abort_flag;
    int *sh_hist;              // [nd][L] (run-time rows) or [L+1][nd] (compile-time rows, see zstep)
    uint32_t *pw1, *pw2;       // paired first-level words: [EC | count] and [area | perimeter], 2 copies each
    int pstride;               // words between the two copies (odd multiple of banks apart)
    FBin fb;
    IBin<T> ib;
    int tr, tc;
    uint32_t bin3;             // third binning share of this thread: float offset | key offset << 16, or ~0
    // current item
    int x0, y0, z0, z1;
    uint32_t base;
    uint32_t parity;
    uint32_t inflight;         // thread 0: ring slots with a TMA copy issued and not yet waited for
    bool interior;
    // the item's counted box reaches past the field: voxels at the
    // never-active level L are left out of the interleaved histogram (their
    // changes belong to the discarded level; past the edge they would all hit
    // one word and serialise the warp's atomics)
    bool skip;
};

template <typename T>
__device__ __forceinline__ uint32_t bin_value(const Ctx<T> &c, T v)
{
    if constexpr (sizeof(T) == 4) return c.fb.uniform ? fbin_uniform(v, c.fb) : fbin(v, c.fb);
    else return c.ib(v);
}

// Paired 16-bit fields in one 32-bit word: value = lo + 65536 * hi with lo a
// signed 16-bit field (its borrow runs into hi), so any sequence of adds
// decodes exactly while |lo| and |hi| stay below 2^15.  A thread that sees a
// field pass 16000 after its add moves the word into the int32 histogram
// (atomicExch), which keeps both fields far from their limits.
__device__ __forceinline__ void pair_decode(uint32_t w, int &lo, int &hi)
{
    lo = (int)(int16_t)(w & 0xFFFFu);
    hi = (int)(w - (uint32_t)lo) >> 16;
}

__device__ __forceinline__ void pair_add(uint32_t *word, uint32_t add, int *row_lo, int *row_hi, uint32_t k)
{
    const uint32_t old = atomicAdd(word, add);
    int lo, hi;
    pair_decode(old + add, lo, hi);
    if (lo > 16000 || lo < -16000 || hi > 16000 || hi < -16000) {
        const uint32_t w = atomicExch(word, 0u);
        pair_decode(w, lo, hi);
        if (row_lo) atomicAdd(&row_lo[k], lo);
        if (row_hi) atomicAdd(&row_hi[k], hi);
    }
}

template <int DM, int D>
constexpr int dm_row() { return ((DM & 1) && D > 0) + ((DM & 2) && D > 1) + ((DM & 4) && D > 2); }

template <int DM>
constexpr int dm_nd() { return (DM & 1) + ((DM >> 1) & 1) + ((DM >> 2) & 1) + ((DM >> 3) & 1); }

// Histogram layout of a kernel instantiation: rows interleaved per level
// ([L+1][nd]) for compile-time rows with one atomic per descriptor.
template <int DM, int SCHED>
constexpr bool interleaved_hist() { return DM != 0 && SCHED != 3; }

// Bin the 18 x 34 value pairs of one staged float plane into a key plane.
// Thread (tr, tc) takes pairs tc and tc + 16 of row tr (fixed offsets, so
// the addresses are immediates); the 100 pairs left (rows 16-17, pairs 32-33
// of rows 0-15) go to threads 0-99 through their precomputed offsets.
template <bool UNI>
__device__ __forceinline__ void bin_pair(uint32_t *kp, const float *fp, const FBin &fb)
{
    const float2 v = *(const float2 *)fp;
    const uint32_t b0 = UNI ? fbin_uniform(v.x, fb) : fbin(v.x, fb);
    const uint32_t b1 = UNI ? fbin_uniform(v.y, fb) : fbin(v.y, fb);
    *kp = b0 | (b1 << 16);
}

template <bool UNI, typename T>
__device__ __forceinline__ void bin_plane_f32(uint32_t *kp, const float *fp, const Ctx<T> &c, bool extra)
{
    const int fo = c.tr * BX + 2 + 2 * c.tc, ko = c.tr * KP + c.tc;
    bin_pair<UNI>(kp + ko, fp + fo, c.fb);
    bin_pair<UNI>(kp + ko + 16, fp + fo + 32, c.fb);
    if (extra && c.bin3 != ~0u) bin_pair<UNI>(kp + (c.bin3 >> 16), fp + (c.bin3 & 0xFFFFu), c.fb);
}

// Fill a key plane with the never-active level (planes outside the field).
__device__ __forceinline__ void fill_never(uint32_t *kp, int L)
{
    const uint32_t never = (uint32_t)L | ((uint32_t)L << 16);
    for (int i = threadIdx.x; i < kPairsPerPlane; i += kThreads) {
        const int row = i / ((BX - 4) / 2), jp = i - row * ((BX - 4) / 2);
        kp[row * KP + jp] = never;
    }
}

// Offsets of a thread's third binning share (see bin_plane_f32): the 100
// pairs left over go to threads 0-99 in one plane of a barrier step and to
// threads 128-227 in the other.
__device__ __forceinline__ uint32_t bin3_offsets(int tid)
{
    if (tid >= 128) tid -= 128;
    int row, jp;
    if (tid < 2 * 34) { row = 16 + tid / 34; jp = tid % 34; }
    else if (tid < 2 * 34 + 32) { row = (tid - 68) >> 1; jp = 32 + ((tid - 68) & 1); }
    else return ~0u;
    return (uint32_t)(row * BX + 2 + 2 * jp) | ((uint32_t)(row * KP + jp) << 16);
}
static_assert(BY == 18 && (BX - 4) / 2 == 34 && kThreads == 256, "binning shares assume 18 x 34 pairs, 256 threads");

// ---- asynchronous plain-load path: the 18 rows of a plane are copied into
// shared memory KAP planes ahead with cp.async (16-byte chunks, zero-filled
// outside the field); used when every row starts 16-byte aligned.

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Start this thread's copies of plane pz (nothing if not wanted) and close
// them as one group.  STG_ALIGNED: row widths and starts are multiples of 16
// bytes, so a chunk lies wholly inside or wholly outside the field.
// STG_COVER: each row copies the 16-byte aligned cover of its in-field part
// (bytes of neighbouring rows in the cover are never read), the field's last
// chunk clipped to its end.
template <typename T, int STG, int NRING = NRAWP2, bool COMMIT = true>
__device__ __forceinline__ void copy_plane(const Ctx<T> &c, int pz, bool wanted)
{
    constexpr int A = rpad<T>(), CPR = rrow_bytes<T>() / 16, sz = (int)sizeof(T);
    if (wanted) {
        const bool zin = pz >= 0 && pz < c.p.D;
        unsigned char *slot = c.raw + (uint32_t)((pz + 16) % NRING) * rplane_bytes<T>();
        if constexpr (STG == STG_ALIGNED) {
            const T *base = (const T *)c.p.field;
            for (int q = threadIdx.x; q < BY * CPR; q += kThreads) {
                const int row = q / CPR, ch = q - row * CPR;
                const int64_t gy = (int64_t)c.y0 - 1 + row, gx = (int64_t)c.x0 - A + (int64_t)ch * A;
                const bool in = zin && gy >= 0 && gy < c.p.H && gx >= 0 && gx < c.p.W;
                cp_async16(smem_u32(slot + row * rrow_bytes<T>() + ch * 16),
                           in ? base + ((int64_t)pz * c.p.H + gy) * c.p.W + gx : base, in ? 16u : 0u);
            }
        } else if (zin) {
            const unsigned char *fb = (const unsigned char *)c.p.field;
            const int64_t total = c.p.D * c.p.H * c.p.W * sz;
            const int64_t xlo = max((int64_t)c.x0 - 2, (int64_t)0), xhi = min((int64_t)c.x0 + 66, c.p.W);
            for (int q = threadIdx.x; q < BY * CPR; q += kThreads) {
                const int row = q / CPR, ch = q - row * CPR;
                const int64_t gy = (int64_t)c.y0 - 1 + row;
                if (gy < 0 || gy >= c.p.H) continue;
                const int64_t rs = (((int64_t)pz * c.p.H + gy) * c.p.W + xlo) * sz;
                const int64_t cs = (rs & ~(int64_t)15) + 16 * ch;
                if (cs >= rs + (xhi - xlo) * sz) continue;
                const int64_t left = total - cs;
                cp_async16(smem_u32(slot + row * rrow_bytes<T>() + ch * 16), fb + cs, left < 16 ? (uint32_t)left : 16u);
            }
        }
    }
    if (COMMIT) cp_async_commit();
}

// One value pair (row, jp) of a raw plane slot into the key plane.
template <typename T, int STG>
__device__ __forceinline__ void bin_pair_raw(Ctx<T> &c, uint32_t *kp, const unsigned char *raw, int pb, int row, int jp)
{
    constexpr int A = rpad<T>(), sz = (int)sizeof(T);
    const uint32_t L = (uint32_t)c.p.L;
    const int64_t gy = (int64_t)c.y0 - 1 + row, gx = (int64_t)c.x0 - 2 + 2 * jp;
    const bool yin = gy >= 0 && gy < c.p.H;
    const unsigned char *r;
    if constexpr (STG == STG_ALIGNED) {
        r = raw + row * rrow_bytes<T>() + (A - 2 + 2 * jp) * sz;
    } else {
        const int64_t xlo = max((int64_t)c.x0 - 2, (int64_t)0);
        const int off = (int)(((((int64_t)pb * c.p.H + gy) * c.p.W + xlo) * sz) & 15);
        r = raw + row * rrow_bytes<T>() + off + (gx - xlo) * sz;
    }
    const uint32_t b0 = (yin && (c.interior || (gx >= 0 && gx < c.p.W))) ? bin_value(c, *(const T *)r) : L;
    const uint32_t b1 = (yin && (c.interior || (gx + 1 >= 0 && gx + 1 < c.p.W))) ? bin_value(c, *(const T *)(r + sz)) : L;
    kp[row * KP + jp] = b0 | (b1 << 16);
}

// Bin a raw plane with the fixed per-thread shares of bin_plane_f32 (pairs
// tc and tc+16 of row tr, plus the leftover pair of bin3 when `extra`).
template <typename T, int STG>
__device__ __forceinline__ void bin_plane_raw2(Ctx<T> &c, int pb, uint32_t *kp, bool extra)
{
    const unsigned char *raw = c.raw + (uint32_t)((pb + 16) % NRAWP2) * rplane_bytes<T>();
    bin_pair_raw<T, STG>(c, kp, raw, pb, c.tr, c.tc);
    bin_pair_raw<T, STG>(c, kp, raw, pb, c.tr, c.tc + 16);
    if (extra && c.bin3 != ~0u) {
        const int ko = (int)(c.bin3 >> 16), row = ko / KP;
        bin_pair_raw<T, STG>(c, kp, raw, pb, row, ko - row * KP);
    }
}

// Bin plane pb from its raw slot into the key ring; values outside the
// field bin to L.
template <typename T, int STG>
__device__ __forceinline__ void bin_plane_raw(Ctx<T> &c, int pb, uint32_t *kp)
{
    constexpr int A = rpad<T>(), sz = (int)sizeof(T);
    const uint32_t L = (uint32_t)c.p.L;
    const unsigned char *raw = c.raw + (uint32_t)((pb + 16) % NRAWP) * rplane_bytes<T>();
    const int64_t xlo = max((int64_t)c.x0 - 2, (int64_t)0);
    for (int i = threadIdx.x; i < kPairsPerPlane; i += kThreads) {
        const int row = i / ((BX - 4) / 2), jp = i - row * ((BX - 4) / 2);
        const int64_t gy = (int64_t)c.y0 - 1 + row, gx = (int64_t)c.x0 - 2 + 2 * jp;
        const bool yin = gy >= 0 && gy < c.p.H;
        const unsigned char *r;
        if constexpr (STG == STG_ALIGNED) {
            r = raw + row * rrow_bytes<T>() + (A - 2 + 2 * jp) * sz;
        } else {
            // the slot starts at the 16-byte boundary below element xlo of the row
            const int off = (int)(((((int64_t)pb * c.p.H + gy) * c.p.W + xlo) * sz) & 15);
            r = raw + row * rrow_bytes<T>() + off + (gx - xlo) * sz;
        }
        const uint32_t b0 = (yin && (c.interior || (gx >= 0 && gx < c.p.W))) ? bin_value(c, *(const T *)r) : L;
        const uint32_t b1 =
            (yin && (c.interior || (gx + 1 >= 0 && gx + 1 < c.p.W))) ? bin_value(c, *(const T *)(r + sz)) : L;
        kp[row * KP + jp] = b0 | (b1 << 16);
    }
}

// Load key plane s+1 into window slot (R+1)%3 and add the contributions of
// plane s (R = position of plane s in the 3-plane register window).
template <typename T, bool PER, int R, int DM, int SCHED>
__device__ __forceinline__ void count_plane(Ctx<T> &c, uint32_t (&win)[3][3][5], int s)
{
    const int L = c.p.L;
    // ---- load key plane s+1 into window slot (R+1)%3
    if (s >= c.z0 - 2) {
        const uint32_t *kp = c.kring + (uint32_t)((s + 1 + 8) % NK) * KWORDS;
        constexpr int W = (R + 1) % 3;
#pragma unroll
        for (int dy = 0; dy < 3; dy++) {
            const uint32_t *r = kp + (c.tr + dy) * KP + 2 * c.tc;
            const uint2 a = *(const uint2 *)r, b = *(const uint2 *)(r + 2);
            const uint32_t w0 = a.x, w1 = a.y, w2 = b.x, w3 = b.y;
            win[W][dy][0] = w1;
            win[W][dy][1] = w2;
            win[W][dy][2] = __byte_perm(w0, w1, 0x5432);   // keys x-1, x
            win[W][dy][3] = __byte_perm(w1, w2, 0x5432);   // keys x+1, x+2
            win[W][dy][4] = __byte_perm(w2, w3, 0x5432);   // keys x+3, x+4
        }
    }
    // ---- contributions of plane s
    if (s >= c.z0) {
        constexpr int SL[3] = {(R + 2) % 3, R, (R + 1) % 3};   // window slots of planes s-1, s, s+1
        uint32_t n0[27], n1[27];
#pragma unroll
        for (int dz = 0; dz < 3; dz++)
#pragma unroll
            for (int dy = 0; dy < 3; dy++) {
                const int i = 1 + 3 * dy + 9 * dz;
                const uint32_t *w = win[SL[dz]][dy];
                n0[i - 1] = w[2]; n0[i] = w[0]; n0[i + 1] = w[3];
                n1[i - 1] = w[3]; n1[i] = w[1]; n1[i + 1] = w[4];
            }
        const uint32_t c0 = win[R][1][0], c1 = win[R][1][1];
        const QuadDelta q = quad_delta<PER>(n0, c0, n1, c1);
        const uint32_t key[4] = {c0 & 0xFFFFu, c0 >> 16, c1 & 0xFFFFu, c1 >> 16};
        const int ecv[4] = {sbyte<0>(q.ec), sbyte<1>(q.ec), sbyte<2>(q.ec), sbyte<3>(q.ec)};
        const int arv[4] = {sbyte<0>(q.area), sbyte<1>(q.area), sbyte<2>(q.area), sbyte<3>(q.area)};
        const int pev[4] = {sbyte<0>(q.per), sbyte<1>(q.per), sbyte<2>(q.per), sbyte<3>(q.per)};
        if constexpr (DM != 0) {
            // descriptor rows fixed at compile time; shared histogram guaranteed
            int *const h = c.sh_hist;
            if constexpr (SCHED == 3) {
                const uint32_t cp = (threadIdx.x & 1u) * (uint32_t)c.pstride;
                int *const r_ec = (DM & 1) ? h + dm_row<DM, 0>() * L : nullptr;
                int *const r_pe = (DM & 2) ? h + dm_row<DM, 1>() * L : nullptr;
                int *const r_ar = (DM & 4) ? h + dm_row<DM, 2>() * L : nullptr;
                int *const r_vo = (DM & 8) ? h + dm_row<DM, 3>() * L : nullptr;
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    const uint32_t k = key[v];
                    if (k < (uint32_t)L) {
                        if (DM & 9) {
                            const uint32_t add = ((DM & 1) ? (uint32_t)ecv[v] : 0u) + ((DM & 8) ? 65536u : 0u);
                            pair_add(c.pw1 + cp + k, add, r_ec, r_vo, k);
                        }
                        if (DM & 6) {
                            const uint32_t add = ((DM & 4) ? (uint32_t)arv[v] : 0u) +
                                                 ((DM & 2) ? (uint32_t)pev[v] * 65536u : 0u);
                            pair_add(c.pw2 + cp + k, add, r_ar, r_pe, k);
                        }
                    }
                }
            } else {
                // interleaved rows [L+1][ND]: one address per voxel, the rows at
                // immediate offsets; the never-active level L has its own
                // (discarded) slot, so no test is needed
                constexpr int ND = dm_nd<DM>();
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    if (c.skip && key[v] >= (uint32_t)L) continue;
                    int *const e = h + key[v] * ND;
                    if (DM & 1) atomicAdd(e + dm_row<DM, 0>(), ecv[v]);
                    if (DM & 2) atomicAdd(e + dm_row<DM, 1>(), pev[v]);
                    if (DM & 4) atomicAdd(e + dm_row<DM, 2>(), arv[v]);
                    if (DM & 8) atomicAdd(e + dm_row<DM, 3>(), 1);
                }
            }
        } else if constexpr (SCHED == 2) {
            // warp-aggregated update with descriptor rows known at run time
            const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const uint32_t k = key[v] < (uint32_t)L ? key[v] : 0xFFFFFFFFu;
                const uint32_t grp = __match_any_sync(0xFFFFFFFFu, k);
                const uint32_t pk = (uint32_t)(ecv[v] + 13) | ((uint32_t)(arv[v] + 6) << 10) |
                                    ((uint32_t)(pev[v] + 12) << 20);
                const uint32_t sum = __reduce_add_sync(grp, pk);
                if (k != 0xFFFFFFFFu && lane == (uint32_t)(__ffs(grp) - 1)) {
                    const int n = __popc(grp);
                    const int vals[4] = {(int)(sum & 1023u) - 13 * n, (int)((sum >> 20) & 1023u) - 12 * n,
                                         (int)((sum >> 10) & 1023u) - 6 * n, n};
#pragma unroll
                    for (int dsc = 0; dsc < kMaxDesc; dsc++) {
                        const int r = c.p.rows[dsc];
                        if (r < 0) continue;
                        if (c.sh_hist) atomicAdd(&c.sh_hist[r * L + k], vals[dsc]);
                        else atomicAdd((unsigned long long *)&c.p.hist[(size_t)r * L + k],
                                       (unsigned long long)(long long)vals[dsc]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const uint32_t k = key[v];
                if (k >= (uint32_t)L) continue;
                const int vals[4] = {ecv[v], pev[v], arv[v], 1};
#pragma unroll
                for (int dsc = 0; dsc < kMaxDesc; dsc++) {
                    const int r = c.p.rows[dsc];
                    if (r < 0 || vals[dsc] == 0) continue;
                    if (c.sh_hist) atomicAdd(&c.sh_hist[r * L + k], vals[dsc]);
                    else atomicAdd((unsigned long long *)&c.p.hist[(size_t)r * L + k],
                                   (unsigned long long)(long long)vals[dsc]);
                }
            }
        }
    }
}

// One step of the z walk with plain loads: bin plane s+2 into the key ring
// (one barrier per plane), then count plane s.  R = t mod 3, s = z0 - 3 + t.
// Returns false if the block must stop.
// Barrier step of the plain-load z walk at s = z0 - 3 + t: synchronise and
// bin plane s+2 into the key ring (one barrier per plane).  Returns false if
// the block must stop.
template <typename T>
__device__ __forceinline__ bool plain_barrier(Ctx<T> &c, int s)
{
    const int pb = s + 2;
    const int L = c.p.L;
    __syncthreads();
    if (*c.abort_flag) return false;
    if (pb <= c.z1) {
        uint32_t *kp = c.kring + (uint32_t)((pb + 8) % NK) * KWORDS;
        if (pb < c.p.zv0 || pb >= c.p.zv1) {
            fill_never(kp, L);
        } else {
            const T *f = (const T *)c.p.field;
            for (int i = threadIdx.x; i < kPairsPerPlane; i += kThreads) {
                const int row = i / ((BX - 4) / 2), jp = i - row * ((BX - 4) / 2);
                const int j = 2 + 2 * jp;
                const int64_t gy = (int64_t)c.y0 - 1 + row, gx = (int64_t)c.x0 - 4 + j;
                uint32_t b0 = (uint32_t)L, b1 = (uint32_t)L;
                if (gy >= 0 && gy < c.p.H) {
                    const T *rowp = f + ((int64_t)pb * c.p.H + gy) * c.p.W;
                    if (c.interior || (gx >= 0 && gx < c.p.W)) b0 = bin_value(c, rowp[gx]);
                    if (c.interior || (gx + 1 >= 0 && gx + 1 < c.p.W)) b1 = bin_value(c, rowp[gx + 1]);
                }
                kp[row * KP + jp] = b0 | (b1 << 16);
            }
        }
    }
    return true;
}

// One step of the z walk with plain loads: bin plane s+2 into the key ring
// (plain_barrier), then count plane s.  R = t mod 3, s = z0 - 3 + t.
// Returns false if the block must stop.
template <typename T, bool PER, int R, int DM, int SCHED = 0>
__device__ __forceinline__ bool zstep(Ctx<T> &c, uint32_t (&win)[3][3][5], int t)
{
    const int s = c.z0 - 3 + t;
    if (!plain_barrier(c, s)) return false;
    count_plane<T, PER, R, DM, SCHED>(c, win, s);
    return true;
}

// After a wait gave up: wait (bounded, about half a second each) for the
// block's other TMA copies still in flight, so none lands after the block
// has left.
template <typename T>
__device__ __forceinline__ void drain_tma(Ctx<T> &c)
{
    for (int slot = 0; slot < NS; slot++)
        if ((c.inflight >> slot) & 1u) {
            mbar_wait(&c.bars[slot], (c.parity >> slot) & 1u, 1000000000ll);
            c.inflight &= ~(1u << slot);
        }
}

// One half-step of the TMA z walk (float32 fields), counting plane
// h = z0 - 4 + t.  Every other half-step (t even) is a barrier step: thread 0
// waits for the staged float planes h+3 and h+4, the block synchronises,
// thread 0 requests planes h+NS+1 and h+NS+2 into the ring slots of planes
// h+1 and h+2 (binned before this barrier), and the block bins planes h+3
// and h+4.  Every half-step then loads key plane h+1 (binned at least one
// barrier earlier) and counts plane h.  Key ring: between two barriers the
// block reads planes h+1, h+2 and writes h+3, h+4: four distinct slots.
// Returns false if the block must stop.
// Barrier step of the TMA z walk (float32 fields) at h = z0 - 4 + t, t even:
// thread 0 waits for the staged float planes h+3 and h+4, the block
// synchronises, thread 0 requests planes h+NS+1 and h+NS+2 into the ring
// slots of planes h+1 and h+2 (binned before this barrier), and the block bins
// planes h+3 and h+4.  Returns false if the block must stop.
template <typename T>
__device__ __forceinline__ bool tma_barrier(Ctx<T> &c, const CUtensorMap *tmap, int h)
{
    const int L = c.p.L;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 3; q <= 4; q++) {
            const int pb = h + q;
            if (pb > c.z1) break;
            const uint32_t slot = (c.base + (uint32_t)(pb - (c.z0 - 1))) % NS;
            if (!mbar_wait(&c.bars[slot], (c.parity >> slot) & 1u)) {
                *c.abort_flag = 1;
                atomicOr(c.p.err, 4);
                break;
            }
            c.parity ^= 1u << slot;
            c.inflight &= ~(1u << slot);
        }
    }
    __syncthreads();
    if (*c.abort_flag) {
        if (threadIdx.x == 0) drain_tma(c);
        return false;
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = NS + 1; q <= NS + 2; q++) {
            const int pi = h + q;
            if (pi > c.z1) break;
            const uint32_t slot = (c.base + (uint32_t)(pi - (c.z0 - 1))) % NS;
            mbar_expect_tx(&c.bars[slot], BX * BY * 4);
            tma_load_plane(c.fring + slot * FSTRIDE, tmap, c.x0 - 4, c.y0 - 1, pi, &c.bars[slot]);
            c.inflight |= 1u << slot;
        }
    }
    // ---- bin planes h+3 (extra pairs on threads 0-99) and h+4 (threads 128-227)
#pragma unroll
    for (int q = 3; q <= 4; q++) {
        const int pb = h + q;
        if (pb > c.z1) break;
        uint32_t *kp = c.kring + (uint32_t)((pb + 8) % NK) * KWORDS;
        if (pb < c.p.zv0 || pb >= c.p.zv1) {
            fill_never(kp, L);
        } else {
            const float *fp = c.fring + ((c.base + (uint32_t)(pb - (c.z0 - 1))) % NS) * FSTRIDE;
            const bool extra = (q == 3) == (threadIdx.x < 128);
            if (c.fb.uniform) bin_plane_f32<true>(kp, fp, c, extra);
            else bin_plane_f32<false>(kp, fp, c, extra);
        }
    }
    return true;
}

// One half-step of the TMA z walk, counting plane h = z0 - 4 + t.  Every
// other half-step (t even) is a barrier step (tma_barrier).  Every half-step
// then loads key plane h+1 (binned at least one barrier earlier) and counts
// plane h.  Key ring: between two barriers the block reads planes h+1, h+2
// and writes h+3, h+4: four distinct slots.  Returns false if the block must
// stop.
template <typename T, bool PER, int R, int DM, int SCHED = 0>
__device__ __forceinline__ bool zstep_tma(Ctx<T> &c, const CUtensorMap *tmap, uint32_t (&win)[3][3][5], int t)
{
    const int h = c.z0 - 4 + t;
    if ((t & 1) == 0 && !tma_barrier(c, tmap, h)) return false;
    count_plane<T, PER, R, DM, SCHED>(c, win, h);
    return true;
}

// One step of the one-plane cp.async walk (s = z0 - 3 + t, pb = s + 2),
// used by the batched kernel, whose register budget the two-plane walk
// exceeds:
// wait for this thread's copies of plane pb, synchronise, bin it, start the
// copies of plane pb + KAP (into the slot of plane pb - 2, binned two steps
// ago), then count plane s.  Returns false if the block must stop.
template <typename T, bool PER, int R, int DM, int SCHED = 0, int STG = STG_ALIGNED>
__device__ __forceinline__ bool zstep_async(Ctx<T> &c, uint32_t (&win)[3][3][5], int t)
{
    const int s = c.z0 - 3 + t;
    const int pb = s + 2;
    cp_async_wait<KAP - 1>();
    __syncthreads();
    if (*c.abort_flag) return false;
    if (pb <= c.z1) {
        uint32_t *kp = c.kring + (uint32_t)((pb + 8) % NK) * KWORDS;
        if (pb < c.p.zv0 || pb >= c.p.zv1) fill_never(kp, c.p.L);
        else bin_plane_raw<T, STG>(c, pb, kp);
    }
    copy_plane<T, STG, NRAWP>(c, pb + KAP, pb + KAP <= c.z1);
    count_plane<T, PER, R, DM, SCHED>(c, win, s);
    return true;
}

// One half-step of the two-plane cp.async walk (same plane schedule as
// zstep_tma), counting plane h = z0 - 4 + t.  Barrier steps (t even): wait
// for this thread's copies of planes h+3 and h+4 (issued two barrier steps
// ago), synchronise, bin them, and start the copies of planes h+7 and h+8
// (one group) into the slots of planes h+1 and h+2, binned one barrier step
// ago.  Returns false if the block must stop.
// Barrier step of the two-plane cp.async walk at h = z0 - 4 + t, t even:
// wait for this thread's copies of planes h+3 and h+4 (issued two barrier
// steps ago), synchronise, bin them, and start the copies of planes h+7 and
// h+8 (one group) into the slots of planes h+1 and h+2, binned one barrier
// step ago.  Returns false if the block must stop.
template <typename T, int STG>
__device__ __forceinline__ bool async2_barrier(Ctx<T> &c, int h)
{
    cp_async_wait<1>();
    __syncthreads();
    if (*c.abort_flag) return false;
#pragma unroll
    for (int q = 3; q <= 4; q++) {
        const int pb = h + q;
        if (pb > c.z1) break;
        uint32_t *kp = c.kring + (uint32_t)((pb + 8) % NK) * KWORDS;
        if (pb < c.p.zv0 || pb >= c.p.zv1) fill_never(kp, c.p.L);
        else bin_plane_raw2<T, STG>(c, pb, kp, (q == 3) == (threadIdx.x < 128));
    }
    copy_plane<T, STG, NRAWP2, false>(c, h + 7, h + 7 <= c.z1);
    copy_plane<T, STG, NRAWP2, false>(c, h + 8, h + 8 <= c.z1);
    cp_async_commit();
    return true;
}

// Start the copies of planes z0-1 .. z0+2 (two groups) for the two-plane walk.
template <typename T, int STG>
__device__ __forceinline__ void async2_prologue(Ctx<T> &c)
{
    copy_plane<T, STG, NRAWP2, false>(c, c.z0 - 1, true);
    copy_plane<T, STG, NRAWP2, false>(c, c.z0, c.z0 <= c.z1);
    cp_async_commit();
    copy_plane<T, STG, NRAWP2, false>(c, c.z0 + 1, c.z0 + 1 <= c.z1);
    copy_plane<T, STG, NRAWP2, false>(c, c.z0 + 2, c.z0 + 2 <= c.z1);
    cp_async_commit();
}

// One half-step of the two-plane cp.async walk (same plane schedule as
// zstep_tma), counting plane h = z0 - 4 + t; barrier steps (t even) run
// async2_barrier first.  Returns false if the block must stop.
template <typename T, bool PER, int R, int DM, int SCHED, int STG>
__device__ __forceinline__ bool zstep_async2(Ctx<T> &c, uint32_t (&win)[3][3][5], int t)
{
    const int h = c.z0 - 4 + t;
    if ((t & 1) == 0 && !async2_barrier<T, STG>(c, h)) return false;
    count_plane<T, PER, R, DM, SCHED>(c, win, h);
    return true;
}

// Walk one item with zstep_async2: planes z0-1 .. z1 binned, z0 .. z1-1 counted.
template <typename T, bool PER, int DM, int SCHED, int STG>
__device__ __forceinline__ bool walk_item_async2(Ctx<T> &c, uint32_t (&win)[3][3][5])
{
    async2_prologue<T, STG>(c);
    const int nsteps = c.z1 - c.z0 + 4;
    bool ok = true;
    for (int t = 0; ok && t < nsteps; t += 3) {
        ok = zstep_async2<T, PER, 0, DM, SCHED, STG>(c, win, t);
        if (ok && t + 1 < nsteps) ok = zstep_async2<T, PER, 1, DM, SCHED, STG>(c, win, t + 1);
        if (ok && t + 2 < nsteps) ok = zstep_async2<T, PER, 2, DM, SCHED, STG>(c, win, t + 2);
    }
    cp_async_wait<0>();
    return ok;
}

// ------------------------------------------- planar (slice) counting, ec_slice.h

// Load the rows y-1, y, y+1 of key plane `plane` around this thread's quad.
template <typename T>
__device__ __forceinline__ void load_rows5(const Ctx<T> &c, int plane, Row5 (&W)[3])
{
    const uint32_t *kp = c.kring + (uint32_t)((plane + 8) % NK) * KWORDS;
#pragma unroll
    for (int dy = 0; dy < 3; dy++) {
        const uint32_t *r = kp + (c.tr + dy) * KP + 2 * c.tc;
        const uint2 a = *(const uint2 *)r, b = *(const uint2 *)(r + 2);
        W[dy].a = __byte_perm(a.x, a.y, 0x5432);   // keys x-1, x
        W[dy].b = a.y;                             // x, x+1
        W[dy].c = __byte_perm(a.y, b.x, 0x5432);   // x+1, x+2
        W[dy].d = b.x;                             // x+2, x+3
        W[dy].e = __byte_perm(b.x, b.y, 0x5432);   // x+3, x+4
    }
}

// Add the changes of the quad's four voxels at their levels (key pairs kb =
// voxels 0, 1 and kd = voxels 2, 3).  Histogram rows interleaved per level,
// [L+1][nd], with the never-active level L in its own (discarded) slot.
// DM != 0: descriptor rows fixed at compile time; DM == 0: rows[] at run time.
// skip: voxels at level L are left out (items reaching past the field).
template <int DM>
__device__ __forceinline__ void slice_hist(int *h, int nd, const int (&rows)[kMaxDesc], uint32_t kb, uint32_t kd,
                                           const SliceOut &o, bool skip, uint32_t L)
{
    const uint32_t key[4] = {kb & 0xFFFFu, kb >> 16, kd & 0xFFFFu, kd >> 16};
    const int ecv[4] = {sbyte<0>(o.ec), sbyte<1>(o.ec), sbyte<2>(o.ec), sbyte<3>(o.ec)};
    if constexpr (DM != 0) {
        constexpr int ND = dm_nd<DM>();
#pragma unroll
        for (int v = 0; v < 4; v++) {
            if (skip && key[v] >= L) continue;
            int *const e = h + key[v] * ND;
            if (DM & 1) atomicAdd(e + dm_row<DM, 0>(), ecv[v]);
            if (DM & 2) {
                const int pv[4] = {sbyte<0>(o.per), sbyte<1>(o.per), sbyte<2>(o.per), sbyte<3>(o.per)};
                atomicAdd(e + dm_row<DM, 1>(), pv[v]);
            }
            if (DM & 4) {
                const int av[4] = {sbyte<0>(o.area), sbyte<1>(o.area), sbyte<2>(o.area), sbyte<3>(o.area)};
                atomicAdd(e + dm_row<DM, 2>(), av[v]);
            }
            if (DM & 8) atomicAdd(e + dm_row<DM, 3>(), 1);
        }
    } else {
        const int pv[4] = {sbyte<0>(o.per), sbyte<1>(o.per), sbyte<2>(o.per), sbyte<3>(o.per)};
        const int av[4] = {sbyte<0>(o.area), sbyte<1>(o.area), sbyte<2>(o.area), sbyte<3>(o.area)};
#pragma unroll
        for (int v = 0; v < 4; v++) {
            if (skip && key[v] >= L) continue;
            int *const e = h + key[v] * nd;
            if (rows[0] >= 0) atomicAdd(e + rows[0], ecv[v]);
            if (rows[1] >= 0) atomicAdd(e + rows[1], pv[v]);
            if (rows[2] >= 0) atomicAdd(e + rows[2], av[v]);
            if (rows[3] >= 0) atomicAdd(e + rows[3], 1);
        }
    }
}

// One step of a planar walk at plane h (same plane schedule as the
// 26-neighbour walks): load key plane h+1 into Q; at h = z0 - 1 start the
// state from planes z0 - 1 (P) and z0 (Q); from h = z0 on, count plane h.
template <typename T, bool PER, int DM>
__device__ __forceinline__ void slice_step(Ctx<T> &c, Row5 (&P)[3], Row5 (&Q)[3], SliceState &st, int h)
{
    if (h >= c.z0 - 2) load_rows5(c, h + 1, Q);
    if (h == c.z0 - 1) {
        slice_begin<PER>(P, Q, st);
    } else if (h >= c.z0) {
        constexpr bool AREA = DM == 0 || (DM & 4) != 0;
        const SliceOut o = slice_quad<AREA, PER>(P, Q, st);
        slice_hist<DM>(c.sh_hist, c.p.nd, c.p.rows, P[1].b, P[1].d, o, c.skip, (uint32_t)c.p.L);
    }
}

// Planar walks of one item (planes z0-1 .. z1 binned, z0 .. z1-1 counted).
// The two window registers alternate between plane h and h+1, so the loop
// runs two half-steps per turn; barrier steps are the even ones.
template <typename T, bool PER, int DM>
__device__ __forceinline__ bool walk_slice_tma(Ctx<T> &c, const CUtensorMap *tmap)
{
    Row5 W0[3], W1[3];
    SliceState st{};
    const int nsteps = c.z1 - c.z0 + 4;
    for (int t = 0; t < nsteps; t += 2) {
        const int h = c.z0 - 4 + t;
        if (!tma_barrier(c, tmap, h)) return false;
        slice_step<T, PER, DM>(c, W0, W1, st, h);
        if (t + 1 < nsteps) slice_step<T, PER, DM>(c, W1, W0, st, h + 1);
    }
    return true;
}

template <typename T, bool PER, int DM, int STG>
__device__ __forceinline__ bool walk_slice_async2(Ctx<T> &c)
{
    Row5 W0[3], W1[3];
    SliceState st{};
    async2_prologue<T, STG>(c);
    const int nsteps = c.z1 - c.z0 + 4;
    bool ok = true;
    for (int t = 0; ok && t < nsteps; t += 2) {
        const int h = c.z0 - 4 + t;
        ok = async2_barrier<T, STG>(c, h);
        if (!ok) break;
        slice_step<T, PER, DM>(c, W0, W1, st, h);
        if (t + 1 < nsteps) slice_step<T, PER, DM>(c, W1, W0, st, h + 1);
    }
    cp_async_wait<0>();
    return ok;
}

template <typename T, bool PER, int DM>
__device__ __forceinline__ bool walk_slice_plain(Ctx<T> &c)
{
    Row5 W0[3], W1[3];
    SliceState st{};
    const int nsteps = c.z1 - c.z0 + 3;
    for (int t = 0; t < nsteps; t += 2) {
        const int s = c.z0 - 3 + t;
        if (!plain_barrier(c, s)) return false;
        slice_step<T, PER, DM>(c, W0, W1, st, s);
        if (t + 1 < nsteps) {
            if (!plain_barrier(c, s + 1)) return false;
            slice_step<T, PER, DM>(c, W1, W0, st, s + 1);
        }
    }
    return true;
}

}  // namespace fast3d

}  // namespace ec

// ec_fast3d.cuh -- device building blocks of the fast per-voxel 3D path,
// shared by the single-field kernel (ec_fast3d.cu) and the batched
// persistent kernel (ec_batch.cu).  See ec_fast3d.cu for the data flow.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ec_internal.h"
#include "ec_rules.h"
#include "ec_swar.h"

namespace ec {

namespace fast3d {

constexpr int kThreads = 256;
constexpr int TXF = 64, TYF = 16;           // voxels per plane of a tile
constexpr int BX = TXF + 8, BY = TYF + 2;   // staged box: x0-4 .. x0+67, y0-1 .. y0+16
constexpr int KP = 37;                      // key row pitch in 32-bit words (odd: conflict-free rows)
constexpr int KWORDS = BY * KP;             // words per key plane
constexpr int NS = 4;                       // float plane ring depth
constexpr int NK = 4;                       // key plane ring depth
constexpr int kThrSmem = 4096;
constexpr int kPairsPerPlane = BY * (BX - 4) / 2;   // key pairs j = 2..69 of 18 rows

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
    const int *uni;        // [0] = 1 if the uniform-spacing guess is exact, [1] = its scale (float bits)
    int packed;            // 1: one 64-bit shared atomic per voxel, flushed per work item
    int agg;               // 1: warp-aggregated shared-memory updates (lanes grouped by level)
    int pairs;             // 1: two descriptors per 32-bit word, two lane-parity copies (see PairHist)
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

// Bounded wait for the phase with the given parity: gives up after about a
// second of device time.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
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
        if (clock64() - t0 > 4000000000ll) break;
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
    int L;
    int uniform;   // the guess below is always the bin or the bin minus one
};

// Guess of the bin of x from the spacing of the thresholds: the nearest
// integer to (x - t0) / spacing.  For x in (t_{k-1}, t_k] of near-uniform
// thresholds this is k-1 or k.  The pre-check kernel and the binning call
// this same function; explicit round-to-nearest intrinsics keep the two
// bit-identical.
__device__ __forceinline__ int bin_guess(float x, float t0, float inv, int L)
{
    const int g = (int)__fmaf_rn(__fsub_rn(x, t0), inv, 0.5f);
    return min(max(g, 0), L - 1);
}

// Exact bin when the guess is known to be the bin or the bin minus one:
// one threshold read and one comparison.  NaN -> L.
__device__ __forceinline__ uint32_t fbin_uniform(float x, const FBin &b)
{
    const int g = bin_guess(x, b.t0, b.inv, b.L);
    const int k = g + (x > b.t[g] ? 1 : 0);
    return x != x ? (uint32_t)b.L : (uint32_t)k;
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
    uint32_t *kring;
    uint64_t *bars;
    volatile int *abort_flag;
    int *sh_hist;
    unsigned long long *h64;   // packed first-level histogram (EC+13 | area+6 << 21 | count << 42)
    unsigned int *h32;         // packed perimeter (perimeter + 12)
    uint32_t *pw1, *pw2;       // paired first-level words: [EC | count] and [area | perimeter], 2 copies each
    int pstride;               // words between the two copies (odd multiple of banks apart)
    FBin fb;
    IBin<T> ib;
    int tr, tc;
    // current item
    int x0, y0, z0, z1;
    uint32_t base;
    uint32_t parity;
    bool interior;
};

template <typename T>
__device__ __forceinline__ uint32_t bin_value(const Ctx<T> &c, T v)
{
    if constexpr (sizeof(T) == 4) return c.fb.uniform ? fbin_uniform(v, c.fb) : fbin(v, c.fb);
    else return c.ib(v);
}

constexpr uint64_t kMask21 = (1ull << 21) - 1;

// Move the packed first-level counts into the block's int32 histogram.
template <typename T, bool PER>
__device__ __forceinline__ void flush_packed(Ctx<T> &c)
{
    const int L = c.p.L;
    for (int b = threadIdx.x; b < L; b += kThreads) {
        const unsigned long long v = c.h64[b];
        if (!v) continue;
        c.h64[b] = 0ull;
        const int cnt = (int)(v >> 42);
        const int ec = (int)(v & kMask21) - 13 * cnt;
        const int ar = (int)((v >> 21) & kMask21) - 6 * cnt;
        if (c.p.rows[0] >= 0) c.sh_hist[c.p.rows[0] * L + b] += ec;
        if (c.p.rows[2] >= 0) c.sh_hist[c.p.rows[2] * L + b] += ar;
        if (c.p.rows[3] >= 0) c.sh_hist[c.p.rows[3] * L + b] += cnt;
        if (PER) {
            const int pe = (int)c.h32[b] - 12 * cnt;
            c.h32[b] = 0u;
            if (c.p.rows[1] >= 0) c.sh_hist[c.p.rows[1] * L + b] += pe;
        }
    }
}

// One step of the z walk: bin plane t+z0-1 (if needed), load key plane
// s+1 into window slot (R+1)%3, and add the contributions of plane s.
// R = t mod 3 where s = z0 - 3 + t.  Returns false if the block must stop.
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

// Bin the pairs of one staged float plane into a key plane (3 fixed
// iterations, the last one partial, so the code is straight-line).
template <bool UNI>
__device__ __forceinline__ void bin_plane_f32(uint32_t *kp, const float *fp, const FBin &fb)
{
#pragma unroll
    for (int it = 0; it < (kPairsPerPlane + kThreads - 1) / kThreads; it++) {
        const int i = threadIdx.x + it * kThreads;
        if (i < kPairsPerPlane) {
            const int row = i / ((BX - 4) / 2), jp = i - row * ((BX - 4) / 2);
            const int j = 2 + 2 * jp;
            const float2 v = *(const float2 *)(fp + row * BX + j);
            const uint32_t b0 = UNI ? fbin_uniform(v.x, fb) : fbin(v.x, fb);
            const uint32_t b1 = UNI ? fbin_uniform(v.y, fb) : fbin(v.y, fb);
            kp[row * KP + (j >> 1)] = b0 | (b1 << 16);
        }
    }
}

template <typename T, bool TMA, bool PER, int R, int DM, int SCHED = 0>
__device__ __forceinline__ bool zstep(Ctx<T> &c, const CUtensorMap *tmap, uint32_t (&win)[3][3][5], int t)
{
    const int s = c.z0 - 3 + t;
    const int pb = s + 2;
    const int L = c.p.L;
    if (TMA && threadIdx.x == 0 && pb <= c.z1) {
        const uint32_t q = (uint32_t)(pb - (c.z0 - 1));
        const uint32_t slot = (c.base + q) % NS;
        if (!mbar_wait(&c.bars[slot], (c.parity >> slot) & 1u)) {
            *c.abort_flag = 1;
            atomicOr(c.p.err, 4);
        }
        c.parity ^= 1u << slot;
    }
    __syncthreads();
    if (*c.abort_flag) return false;
    if (TMA && threadIdx.x == 0) {
        const int pi = s + NS + 1;
        if (pi <= c.z1) {
            const uint32_t q = (uint32_t)(pi - (c.z0 - 1));
            const uint32_t slot = (c.base + q) % NS;
            mbar_expect_tx(&c.bars[slot], BX * BY * 4);
            tma_load_plane(c.fring + slot * FSTRIDE, tmap, c.x0 - 4, c.y0 - 1, pi, &c.bars[slot]);
        }
    }
    // ---- bin plane pb
    if (pb <= c.z1) {
        uint32_t *kp = c.kring + (uint32_t)((pb + 8) % NK) * KWORDS;
        if (pb < c.p.zv0 || pb >= c.p.zv1) {
            const uint32_t never = (uint32_t)L | ((uint32_t)L << 16);
            for (int i = threadIdx.x; i < kPairsPerPlane; i += kThreads) {
                const int row = i / ((BX - 4) / 2), jp = i - row * ((BX - 4) / 2);
                kp[row * KP + 1 + jp] = never;
            }
        } else if constexpr (TMA) {
            const float *fp = c.fring + ((c.base + (uint32_t)(pb - (c.z0 - 1))) % NS) * FSTRIDE;
            if (c.fb.uniform) bin_plane_f32<true>(kp, fp, c.fb);
            else bin_plane_f32<false>(kp, fp, c.fb);
        } else {
            const T *f = (const T *)c.p.field;
            const bool zin = true;
            for (int i = threadIdx.x; i < kPairsPerPlane; i += kThreads) {
                const int row = i / ((BX - 4) / 2), jp = i - row * ((BX - 4) / 2);
                const int j = 2 + 2 * jp;
                const int64_t gy = (int64_t)c.y0 - 1 + row, gx = (int64_t)c.x0 - 4 + j;
                uint32_t b0 = (uint32_t)L, b1 = (uint32_t)L;
                if (zin && gy >= 0 && gy < c.p.H) {
                    const T *rowp = f + ((int64_t)pb * c.p.H + gy) * c.p.W;
                    if (c.interior || (gx >= 0 && gx < c.p.W)) b0 = bin_value(c, rowp[gx]);
                    if (c.interior || (gx + 1 >= 0 && gx + 1 < c.p.W)) b1 = bin_value(c, rowp[gx + 1]);
                }
                kp[row * KP + (j >> 1)] = b0 | (b1 << 16);
            }
        }
    }
    // ---- load key plane s+1 into window slot (R+1)%3
    if (s >= c.z0 - 2) {
        const uint32_t *kp = c.kring + (uint32_t)((s + 1 + 8) % NK) * KWORDS;
        constexpr int W = (R + 1) % 3;
#pragma unroll
        for (int dy = 0; dy < 3; dy++) {
            const uint32_t *r = kp + (c.tr + dy) * KP + 1 + 2 * c.tc;
            const uint32_t w0 = r[0], w1 = r[1], w2 = r[2], w3 = r[3];
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
        const PairDelta d0 = pair_delta<PER>(n0, c0);
        const PairDelta d1 = pair_delta<PER>(n1, c1);
        const uint32_t key[4] = {c0 & 0xFFFFu, c0 >> 16, c1 & 0xFFFFu, c1 >> 16};
        const int ecv[4] = {d0.ec[0], d0.ec[1], d1.ec[0], d1.ec[1]};
        const int arv[4] = {d0.area[0], d0.area[1], d1.area[0], d1.area[1]};
        const int pev[4] = {d0.per[0], d0.per[1], d1.per[0], d1.per[1]};
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
                return true;
            } else {
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const uint32_t k = key[v];
                if (k < (uint32_t)L) {
                    if (DM & 1) atomicAdd(&h[dm_row<DM, 0>() * L + k], ecv[v]);
                    if (DM & 2) atomicAdd(&h[dm_row<DM, 1>() * L + k], pev[v]);
                    if (DM & 4) atomicAdd(&h[dm_row<DM, 2>() * L + k], arv[v]);
                    if (DM & 8) atomicAdd(&h[dm_row<DM, 3>() * L + k], 1);
                }
            }
            return true;
            }
        }
        if constexpr (SCHED == 2) {
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
            return true;
        }
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
    return true;
}

}  // namespace fast3d

}  // namespace ec

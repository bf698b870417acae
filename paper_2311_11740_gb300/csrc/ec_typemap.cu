// ec_typemap.cu -- the vertex-contribution type map and weighted curves.
//
// The paper's output is not only the EC curve but the number of vertices of
// each contribution type at each level (Sec. 2, Algorithm 1 and Table 1;
// Sec. 2.2, Algorithm 3 and Table 2); any descriptor that is a weighted sum
// of vertex contributions, for any connectivity, follows from that map by
// changing the weights (Sec. 4).  ec_type_map computes the map on the
// device (histogram of type transitions per level, running sums, empty type
// from the number of vertices); ec_apply_weights turns a map into curves.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "ec_fast3d.cuh"   // fbin / IBin: level of a value (uniform-spacing guess, binary-search fallback)
#include "ec_internal.h"
#include "ec_rules.h"
#include "ec_types.h"

using namespace ec;

namespace {

// ------------------------------------------------------------ histogram kernel
//
// The born/dies arrays of Algorithms 1-3 (Sec. 2 and 2.2), per vertex: sort
// the 2^n (level, position) keys of the vertex's neighbourhood and walk them
// in order.  At each distinct level b < L the vertex's type changes from the
// type of its cells below b to the type of its cells at or below b: +1 for
// the new type and -1 for the old one, both at b.  Equal levels are merged,
// so the running sums are the plain counts of vertices of each type at each
// level.  The empty type 0 is never written; it is back-calculated from the
// number of vertices (Sec. 2.1).
//
// A block stages the levels of one plane (3D) or row (2D) of cells at a
// time into a ring of three slots, so one barrier per plane suffices, and
// adds into a private shared-memory int32 histogram [L][stride] (odd row
// strides spread a warp's levels over the banks) that is added into the
// global int64 histogram [T-1][L] at the end.

constexpr int kTmThreads = 512;
constexpr int TX3 = 32, TY3 = 16, SW3 = TX3 + 1, SPLANE3 = SW3 * (TY3 + 1);   // 3D: vertices / staged cells
constexpr int TX2 = 512, SW2 = TX2 + 1, TY2 = 64;                              // 2D: vertices per row, rows per tile
constexpr int kStride3 = 23, kStride2 = 7;
constexpr int kThrSmem = 4096;
constexpr size_t kTypeHistBudget = 100 * 1024;

__constant__ TypeTable2D c_types2 = make_type_table_2d();
__constant__ TypeTable3D c_types3 = make_type_table_3d();

template <typename T>
struct TBin {
    fast3d::FBin f;
    fast3d::IBin<T> i;
    __device__ __forceinline__ uint32_t operator()(T v) const
    {
        if constexpr (std::is_same<T, float>::value) return fast3d::fbin(v, f);
        else return i(v);
    }
};

template <typename T>
__host__ __device__ constexpr size_t tbin_smem_bytes(int L, bool has_thr)
{
    return sizeof(T) == 1 ? 512 : ((has_thr && L <= kThrSmem) ? (((size_t)L * sizeof(T) + 15) & ~(size_t)15) : 0);
}

template <typename T>
__device__ TBin<T> make_tbin(const T *gthr, int L, unsigned char *sm)
{
    TBin<T> b{};
    if constexpr (std::is_same<T, float>::value) {
        const float *t = gthr;
        if (L <= kThrSmem) {
            float *st = (float *)sm;
            for (int k = threadIdx.x; k < L; k += blockDim.x) st[k] = gthr[k];
            t = st;
        }
        b.f.t = t;
        b.f.L = L;
        b.f.t0 = gthr[0];
        b.f.tl = gthr[L - 1];
        b.f.inv = (L > 1 && b.f.tl > b.f.t0) ? (float)(L - 1) / (b.f.tl - b.f.t0) : 0.f;
        b.f.off = 0.f;
        b.f.lm1 = (float)(L - 1);
        b.f.uniform = 0;
    } else if constexpr (sizeof(T) == 1) {
        uint16_t *tab = (uint16_t *)sm;
        for (int v = threadIdx.x; v < 256; v += blockDim.x) {
            int k;
            if (!gthr) {
                k = v < L ? v : L;
            } else {
                int lo = 0, n = L;
                while (n > 0) {
                    const int half = n >> 1;
                    if ((int)gthr[lo + half] < v) { lo += half + 1; n -= half + 1; }
                    else n = half;
                }
                k = lo;
            }
            tab[v] = (uint16_t)k;
        }
        b.i.table = tab;
        b.i.t = nullptr;
        b.i.L = L;
    } else {
        const T *t = gthr;
        if (gthr && L <= kThrSmem) {
            T *st = (T *)sm;
            for (int k = threadIdx.x; k < L; k += blockDim.x) st[k] = gthr[k];
            t = st;
        }
        b.i.table = nullptr;
        b.i.t = t;
        b.i.L = L;
    }
    return b;
}

struct G3 {
    const void *f;
    int D, H, W;                 // cells per axis
    int nbx, nby, nbz, tz;       // vertex tiles, vertex planes per tile
};
struct G2 {
    const void *f;
    int H, W;
    int nbx, nby;
};

// Vertex-type transitions of one vertex from its sorted keys (level << SH | position).
template <int NK, int SH, int STRIDE, bool SMEM>
__device__ __forceinline__ void walk_types(const uint32_t (&s)[NK], uint32_t L, const uint8_t *tl, int *sh,
                                           long long *g)
{
    auto add = [&](uint32_t b, int t, int v) {
        if constexpr (SMEM) atomicAdd(&sh[b * STRIDE + t], v);
        else atomicAdd((unsigned long long *)&g[(size_t)(t - 1) * L + b], (unsigned long long)(long long)v);
    };
    uint32_t m = 0;
    int tp = 0;
#pragma unroll
    for (int j = 0; j < NK; j++) {
        const uint32_t b = s[j] >> SH;
        m |= 1u << (s[j] & ((1u << SH) - 1u));
        // sorted keys: the next key has another level iff the xor reaches the level bits
        const bool boundary = j + 1 == NK || (s[j + 1 < NK ? j + 1 : j] ^ s[j]) >= (1u << SH);
        if (boundary && b < L) {
            const int t = tl[m];
            add(b, t, 1);
            if (tp) add(b, tp, -1);
            tp = t;
        }
    }
}

template <int NT, int STRIDE>
__device__ void flush_types(const int *sh, long long *g, int L)
{
    __syncthreads();
    for (int i = threadIdx.x; i < L * STRIDE; i += blockDim.x) {
        const int t = i % STRIDE, b = i / STRIDE;
        const int v = sh[i];
        if (v && t > 0 && t < NT) atomicAdd((unsigned long long *)&g[(size_t)(t - 1) * L + b], (unsigned long long)(long long)v);
    }
}

// Staging of the (TX3+1) x (TY3+1) cells of a plane with lower corner
// (x0-1, y0-1): thread t stages cells t and t + 512 of the plane (row-major,
// TX3+1 wide).  Offsets within a plane are fixed per tile; each plane's raw
// values are loaded one plane ahead into registers so that the loads are in
// flight during the barrier and the walk.  Cells outside the field get L.
template <typename T>
struct Stage3 {
    int64_t off[2];
    bool ok[2];
    T raw[2];
    bool zin;
    static constexpr int kPer = (SPLANE3 + kTmThreads - 1) / kTmThreads;

    __device__ __forceinline__ void setup(const G3 &g, int x0, int y0)
    {
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            const int i = threadIdx.x + q * kTmThreads;
            const int ly = i / SW3, lx = i - ly * SW3;
            const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            ok[q] = i < SPLANE3 && (unsigned)gx < (unsigned)g.W && (unsigned)gy < (unsigned)g.H;
            off[q] = ok[q] ? (int64_t)gy * g.W + gx : 0;
        }
    }
    __device__ __forceinline__ void load(const G3 &g, int z)
    {
        zin = z >= 0 && z < g.D;
        const T *plane = (const T *)g.f + (zin ? (int64_t)z * g.H * g.W : 0);
#pragma unroll
        for (int q = 0; q < kPer; q++)
            if (ok[q] && zin) raw[q] = __ldg(plane + off[q]);
    }
    __device__ __forceinline__ void store(uint16_t *slot, const TBin<T> &bin, uint32_t L) const
    {
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            const int i = threadIdx.x + q * kTmThreads;
            if (i < SPLANE3) slot[i] = (uint16_t)((ok[q] && zin) ? bin(raw[q]) : L);
        }
    }
};

template <typename T, bool SMEM>
__global__ void __launch_bounds__(kTmThreads, 2) k_types3(G3 g, const T *thr, int L, long long *ghist)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t hb = SMEM ? (((size_t)L * kStride3 * 4 + 15) & ~(size_t)15) : 0;
    int *sh = (int *)smem;
    const size_t bb = tbin_smem_bytes<T>(L, thr != nullptr);
    uint8_t *tl = smem + hb + bb;
    uint16_t *ring = (uint16_t *)(smem + hb + bb + 256);
    if (SMEM)
        for (int i = threadIdx.x; i < L * kStride3; i += kTmThreads) sh[i] = 0;
    for (int i = threadIdx.x; i < 256; i += kTmThreads) tl[i] = c_types3.t[i];
    const TBin<T> bin = make_tbin<T>(thr, L, smem + hb);
    __syncthreads();
    const uint32_t UL = (uint32_t)L;
    const int tx = threadIdx.x % TX3, ty = threadIdx.x / TX3;
    const int nitems = g.nbx * g.nby * g.nbz;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % g.nbx, by = (item / g.nbx) % g.nby, bz = item / (g.nbx * g.nby);
        const int x0 = bx * TX3, y0 = by * TY3, z0 = bz * g.tz, z1 = min(z0 + g.tz, g.D + 1);
        Stage3<T> st;
        st.setup(g, x0, y0);
        st.load(g, z0 - 1);
        __syncthreads();   // the ring is free again
        int prev = 0, cur = 1;
        st.store(ring + prev * SPLANE3, bin, UL);
        st.load(g, z0);
        const int X = x0 + tx, Y = y0 + ty;
        for (int Z = z0; Z < z1; Z++) {
            st.store(ring + cur * SPLANE3, bin, UL);
            if (Z + 1 < z1) st.load(g, Z + 1);
            __syncthreads();
            if (X <= g.W && Y <= g.H) {
                const uint16_t *r0 = ring + prev * SPLANE3 + ty * SW3 + tx;
                const uint16_t *r1 = ring + cur * SPLANE3 + ty * SW3 + tx;
                uint32_t s[8];
                s[0] = ((uint32_t)r0[0] << 3) | 0u;
                s[1] = ((uint32_t)r0[1] << 3) | 1u;
                s[2] = ((uint32_t)r0[SW3] << 3) | 2u;
                s[3] = ((uint32_t)r0[SW3 + 1] << 3) | 3u;
                s[4] = ((uint32_t)r1[0] << 3) | 4u;
                s[5] = ((uint32_t)r1[1] << 3) | 5u;
                s[6] = ((uint32_t)r1[SW3] << 3) | 6u;
                s[7] = ((uint32_t)r1[SW3 + 1] << 3) | 7u;
                // Batcher odd-even merge network, 19 comparators
#define CS(a, b) { const uint32_t lo_ = min(s[a], s[b]), hi_ = max(s[a], s[b]); s[a] = lo_; s[b] = hi_; }
                CS(0, 1) CS(2, 3) CS(4, 5) CS(6, 7) CS(0, 2) CS(1, 3) CS(4, 6) CS(5, 7) CS(1, 2) CS(5, 6)
                CS(0, 4) CS(1, 5) CS(2, 6) CS(3, 7) CS(2, 4) CS(3, 5) CS(1, 2) CS(3, 4) CS(5, 6)
#undef CS
                walk_types<8, 3, kStride3, SMEM>(s, UL, tl, sh, ghist);
            }
            const int nxt = 3 - prev - cur;
            prev = cur;
            cur = nxt;
        }
    }
    if (SMEM) flush_types<kTypes3, kStride3>(sh, ghist, L);
}

// Staging of the TX2+1 cells x0-1 .. x0+TX2-1 of a row (thread t: cells t
// and, for thread 0, TX2), loaded one row ahead like Stage3.
template <typename T>
struct Stage2 {
    int off[2];
    bool ok[2];
    T raw[2];
    bool yin;

    __device__ __forceinline__ void setup(const G2 &g, int x0)
    {
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int i = threadIdx.x + q * kTmThreads;
            const int gx = x0 - 1 + i;
            ok[q] = i < SW2 && (unsigned)gx < (unsigned)g.W;
            off[q] = ok[q] ? gx : 0;
        }
    }
    __device__ __forceinline__ void load(const G2 &g, int y)
    {
        yin = y >= 0 && y < g.H;
        const T *row = (const T *)g.f + (yin ? (int64_t)y * g.W : 0);
#pragma unroll
        for (int q = 0; q < 2; q++)
            if (ok[q] && yin) raw[q] = __ldg(row + off[q]);
    }
    __device__ __forceinline__ void store(uint16_t *slot, const TBin<T> &bin, uint32_t L) const
    {
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int i = threadIdx.x + q * kTmThreads;
            if (i < SW2) slot[i] = (uint16_t)((ok[q] && yin) ? bin(raw[q]) : L);
        }
    }
};

template <typename T, bool SMEM>
__global__ void __launch_bounds__(kTmThreads, 2) k_types2(G2 g, const T *thr, int L, long long *ghist)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t hb = SMEM ? (((size_t)L * kStride2 * 4 + 15) & ~(size_t)15) : 0;
    int *sh = (int *)smem;
    const size_t bb = tbin_smem_bytes<T>(L, thr != nullptr);
    uint8_t *tl = smem + hb + bb;
    uint16_t *ring = (uint16_t *)(smem + hb + bb + 16);
    if (SMEM)
        for (int i = threadIdx.x; i < L * kStride2; i += kTmThreads) sh[i] = 0;
    for (int i = threadIdx.x; i < 16; i += kTmThreads) tl[i] = c_types2.t[i];
    const TBin<T> bin = make_tbin<T>(thr, L, smem + hb);
    __syncthreads();
    const uint32_t UL = (uint32_t)L;
    const int tx = threadIdx.x;
    const int nitems = g.nbx * g.nby;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % g.nbx, by = item / g.nbx;
        const int x0 = bx * TX2, y0 = by * TY2, y1 = min(y0 + TY2, g.H + 1);
        Stage2<T> st;
        st.setup(g, x0);
        st.load(g, y0 - 1);
        __syncthreads();   // the ring is free again
        int prev = 0, cur = 1;
        st.store(ring + prev * SW2, bin, UL);
        st.load(g, y0);
        const int X = x0 + tx;
        for (int Y = y0; Y < y1; Y++) {
            st.store(ring + cur * SW2, bin, UL);
            if (Y + 1 < y1) st.load(g, Y + 1);
            __syncthreads();
            if (X <= g.W) {
                const uint16_t *r0 = ring + prev * SW2 + tx, *r1 = ring + cur * SW2 + tx;
                uint32_t s[4] = {((uint32_t)r0[0] << 2) | 0u, ((uint32_t)r0[1] << 2) | 1u,
                                 ((uint32_t)r1[0] << 2) | 2u, ((uint32_t)r1[1] << 2) | 3u};
#define CS(a, b) { const uint32_t lo_ = min(s[a], s[b]), hi_ = max(s[a], s[b]); s[a] = lo_; s[b] = hi_; }
                CS(0, 1) CS(2, 3) CS(0, 2) CS(1, 3) CS(1, 2)
#undef CS
                walk_types<4, 2, kStride2, SMEM>(s, UL, tl, sh, ghist);
            }
            const int nxt = 3 - prev - cur;
            prev = cur;
            cur = nxt;
        }
    }
    if (SMEM) flush_types<kTypes2, kStride2>(sh, ghist, L);
}

template <typename KernelT>
int grid_for(KernelT kernel, size_t smem, int num_sms, int64_t items, int grid_override, int *grid)
{
    int occ = 0;
    if (const int orc = kernel_occupancy((const void *)kernel, kTmThreads, smem, &occ)) return orc;
    if (occ < 1) { set_error("type-map kernel does not fit on an SM (%zu B shared)", smem); return EC_ERR_UNSUPPORTED; }
    int64_t gr = grid_override > 0 ? grid_override : (int64_t)num_sms * occ;
    if (gr > items) gr = items;
    *grid = (int)(gr < 1 ? 1 : gr);
    return EC_OK;
}

template <typename T>
int launch_types(int ndim, const void *field, const int64_t *dims, const void *thr, int L, long long *hist,
                 int tile_z, int grid_override, int num_sms, cudaStream_t s)
{
    const size_t bb = tbin_smem_bytes<T>(L, thr != nullptr);
    int grid = 0, rc;
    if (ndim == 3) {
        G3 g;
        g.f = field;
        g.D = (int)dims[0]; g.H = (int)dims[1]; g.W = (int)dims[2];
        g.tz = tile_z > 0 ? tile_z : 32;
        g.nbx = (g.W + 1 + TX3 - 1) / TX3;
        g.nby = (g.H + 1 + TY3 - 1) / TY3;
        g.nbz = (g.D + 1 + g.tz - 1) / g.tz;
        const int64_t items = (int64_t)g.nbx * g.nby * g.nbz;
        if (items > INT32_MAX) { set_error("field too large for one launch"); return EC_ERR_UNSUPPORTED; }
        const size_t hb = ((size_t)L * kStride3 * 4 + 15) & ~(size_t)15;
        const size_t rest = bb + 256 + 3 * SPLANE3 * sizeof(uint16_t);
        const T *t = (const T *)thr;
        if (hb <= kTypeHistBudget) {
            if ((rc = grid_for(k_types3<T, true>, hb + rest, num_sms, items, grid_override, &grid))) return rc;
            k_types3<T, true><<<grid, kTmThreads, hb + rest, s>>>(g, t, L, hist);
        } else {
            if ((rc = grid_for(k_types3<T, false>, rest, num_sms, items, grid_override, &grid))) return rc;
            k_types3<T, false><<<grid, kTmThreads, rest, s>>>(g, t, L, hist);
        }
    } else {
        G2 g;
        g.f = field;
        g.H = (int)dims[0]; g.W = (int)dims[1];
        g.nbx = (g.W + 1 + TX2 - 1) / TX2;
        g.nby = (g.H + 1 + TY2 - 1) / TY2;
        const int64_t items = (int64_t)g.nbx * g.nby;
        if (items > INT32_MAX) { set_error("field too large for one launch"); return EC_ERR_UNSUPPORTED; }
        const size_t hb = ((size_t)L * kStride2 * 4 + 15) & ~(size_t)15;
        const size_t rest = bb + 16 + 3 * SW2 * sizeof(uint16_t);
        const T *t = (const T *)thr;
        if (hb <= kTypeHistBudget) {
            if ((rc = grid_for(k_types2<T, true>, hb + rest, num_sms, items, grid_override, &grid))) return rc;
            k_types2<T, true><<<grid, kTmThreads, hb + rest, s>>>(g, t, L, hist);
        } else {
            if ((rc = grid_for(k_types2<T, false>, rest, num_sms, items, grid_override, &grid))) return rc;
            k_types2<T, false><<<grid, kTmThreads, rest, s>>>(g, t, L, hist);
        }
    }
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

int launch_type_map(int ndim, const void *field, const int64_t *dims, int dtype, const void *thr, int L,
                    long long *hist, int tile_z, int grid, int num_sms, cudaStream_t s)
{
    switch (dtype) {
    case EC_U8: return launch_types<uint8_t>(ndim, field, dims, thr, L, hist, tile_z, grid, num_sms, s);
    case EC_U16: return launch_types<uint16_t>(ndim, field, dims, thr, L, hist, tile_z, grid, num_sms, s);
    case EC_F32: return launch_types<float>(ndim, field, dims, thr, L, hist, tile_z, grid, num_sms, s);
    }
    set_error("unknown dtype %d", dtype);
    return EC_ERR_DTYPE;
}


constexpr size_t kFlagBytes = 256;
constexpr int kMaxWeightRows = 16;

// Running sum over levels of one type's transition row (block = type 1..T-1).
__global__ void __launch_bounds__(1024) k_type_scan(const long long *__restrict__ hist, int L,
                                                    int64_t *__restrict__ counts)
{
    __shared__ long long warp_tot[32];
    const int row = blockIdx.x;   // type row + 1
    const long long *h = hist + (size_t)row * L;
    int64_t *o = counts + (size_t)(row + 1) * L;
    const int per = (L + blockDim.x - 1) / blockDim.x;
    const int beg = min((int)threadIdx.x * per, L), end = min(beg + per, L);
    long long s = 0;
    for (int k = beg; k < end; k++) s += h[k];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long incl = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        long long w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += t;
        }
        if (lane < nw) warp_tot[lane] = w;
    }
    __syncthreads();
    long long run = incl - s + (wid > 0 ? warp_tot[wid - 1] : 0);
    for (int k = beg; k < end; k++) {
        run += h[k];
        o[k] = run;
    }
}

// Empty type (row 0): the vertices of no other type.
__global__ void k_type_empty(int64_t *__restrict__ counts, int nt, int L, long long nvert)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L) return;
    long long s = 0;
    for (int t = 1; t < nt; t++) s += counts[(size_t)t * L + k];
    counts[k] = nvert - s;
}

struct Weights {
    int32_t w[kMaxWeightRows][kTypes3];
    int32_t scale[kMaxWeightRows];
};

// out[d][k] = sum_t w[d][t] counts[t][k] / scale[d], accumulated in 128 bits;
// a sum that leaves int64 or is not a multiple of its scale poisons its
// entry with INT64_MIN and sets flag bit 0.
__global__ void k_apply_weights(const int64_t *__restrict__ counts, int nt, int L, Weights W,
                                int64_t *__restrict__ out, int *flag)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
    if (k >= L) return;
    __int128 acc = 0;
    for (int t = 0; t < nt; t++) acc += (__int128)W.w[d][t] * (__int128)counts[(size_t)t * L + k];
    const __int128 lo = (__int128)INT64_MIN, hi = (__int128)INT64_MAX;
    int64_t r = INT64_MIN;
    bool ok = acc >= lo && acc <= hi;
    if (ok) {
        const long long a = (long long)acc, sc = W.scale[d];
        const long long q = a / sc;
        ok = q * sc == a;
        if (ok) r = q;
    }
    if (!ok) atomicOr(flag, 1);
    out[(size_t)d * L + k] = r;
}

}  // namespace

extern "C" {

int ec_type_table(int32_t ndim, int32_t *out)
{
    clear_error();
    if (!out) { set_error("out is NULL"); return EC_ERR_ARG; }
    if (ndim == 2) {
        constexpr TypeTable2D t = make_type_table_2d();
        for (int m = 0; m < 16; m++) out[m] = t.t[m];
        return EC_OK;
    }
    if (ndim == 3) {
        constexpr TypeTable3D t = make_type_table_3d();
        for (int m = 0; m < 256; m++) out[m] = t.t[m];
        return EC_OK;
    }
    set_error("ndim must be 2 or 3 (got %d)", ndim);
    return EC_ERR_ARG;
}

int ec_type_map(ec_ctx *ctx, int32_t ndim, const void *field_dev, const int64_t *dims, int dtype,
                const void *thresholds_dev, int32_t L, int64_t *counts_dev, void *stream)
{
    clear_error();
    if (!ctx) { set_error("ctx is NULL"); return EC_ERR_ARG; }
    if (ndim != 2 && ndim != 3) { set_error("ndim must be 2 or 3 (got %d)", ndim); return EC_ERR_ARG; }
    int rc = validate_request(ndim, field_dev, dims, dtype, thresholds_dev, L, ndim == 2 ? 8 : 26, EC_DESC_EC,
                              counts_dev);
    if (rc) return rc;
    if (L == 0) return EC_OK;
    const int nt = ndim == 2 ? kTypes2 : kTypes3;
    long long nvert = 1;
    for (int i = 0; i < ndim; i++) {
        // 32-bit cell coordinates in the kernels
        if (dims[i] > ((int64_t)1 << 30)) { set_error("dims[%d] above 2^30", i); return EC_ERR_ARG; }
        nvert *= dims[i] + 1;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    const size_t hist_bytes = (size_t)(nt - 1) * L * sizeof(long long);
    rc = ensure_scratch(ctx, kFlagBytes + hist_bytes);
    if (rc) return rc;
    int *flags = (int *)ctx->ws;
    long long *hist = (long long *)((char *)ctx->ws + kFlagBytes);
    EC_CUDA(cudaMemsetAsync(ctx->ws, 0, kFlagBytes + hist_bytes, s));
    if (ctx->validate && thresholds_dev) {
        rc = launch_check_sorted(thresholds_dev, dtype, L, flags + 1, s);
        if (rc) return rc;
        EC_CUDA(cudaMemcpyAsync(ctx->host_flag, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        EC_CUDA(cudaStreamSynchronize(s));
        if (*ctx->host_flag) { set_error("thresholds are not non-decreasing"); return EC_ERR_ARG; }
    }
    if (ctx->profile && (rc = prof_begin(ctx, s))) return rc;
    rc = launch_type_map(ndim, field_dev, dims, dtype, thresholds_dev, L, hist, ctx->tile_z, ctx->grid,
                         ctx->num_sms, s);
    if (rc) return rc;
    if (ctx->profile && (rc = prof_end(ctx, s))) return rc;
    k_type_scan<<<nt - 1, 1024, 0, s>>>(hist, L, counts_dev);
    EC_CUDA(cudaGetLastError());
    k_type_empty<<<(L + 255) / 256, 256, 0, s>>>(counts_dev, nt, L, nvert);
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

int ec_apply_weights(ec_ctx *ctx, int32_t ntypes, const int64_t *counts_dev, int32_t L, int32_t nd,
                     const int32_t *weights_host, const int32_t *scales_host, int64_t *out_dev, void *stream)
{
    clear_error();
    if (!ctx) { set_error("ctx is NULL"); return EC_ERR_ARG; }
    if (ntypes < 1 || ntypes > kTypes3) { set_error("ntypes must be in [1, %d] (got %d)", kTypes3, ntypes); return EC_ERR_ARG; }
    if (nd < 1 || nd > kMaxWeightRows) { set_error("nd must be in [1, %d] (got %d)", kMaxWeightRows, nd); return EC_ERR_ARG; }
    if (L < 0 || L > 65535) { set_error("L = %d outside [0, 65535]", L); return EC_ERR_ARG; }
    if (!weights_host) { set_error("weights is NULL"); return EC_ERR_ARG; }
    if (L == 0) return EC_OK;
    if (!counts_dev || !out_dev) { set_error("counts or out is NULL"); return EC_ERR_ARG; }
    Weights W;
    memset(&W, 0, sizeof W);
    for (int d = 0; d < nd; d++) {
        for (int t = 0; t < ntypes; t++) W.w[d][t] = weights_host[(size_t)d * ntypes + t];
        W.scale[d] = scales_host ? scales_host[d] : 1;
        if (W.scale[d] < 1) { set_error("scale[%d] = %d < 1", d, W.scale[d]); return EC_ERR_ARG; }
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    int rc = ensure_scratch(ctx, kFlagBytes);
    if (rc) return rc;
    int *flags = (int *)ctx->ws;
    EC_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), s));
    dim3 grid((unsigned)((L + 255) / 256), (unsigned)nd);
    k_apply_weights<<<grid, 256, 0, s>>>(counts_dev, ntypes, L, W, out_dev, flags);
    EC_CUDA(cudaGetLastError());
    if (ctx->validate) {
        EC_CUDA(cudaMemcpyAsync(ctx->host_flag, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        EC_CUDA(cudaStreamSynchronize(s));
        if (*ctx->host_flag) {
            set_error("a weighted sum is not a multiple of its scale or leaves int64");
            return EC_ERR_ARG;
        }
    }
    return EC_OK;
}

}  // extern "C"

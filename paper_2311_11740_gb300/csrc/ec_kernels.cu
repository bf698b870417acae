// ec_kernels.cu -- histogram and scan kernels for sm_103a.
//
// Data flow of one curve request (Sec. 2, Algorithms 1-3 and the parallel
// scheme of Algorithm 2):
//   1. every block walks tiles of the field; each tile is staged plane by
//      plane into a shared-memory ring of 16-bit levels ("keys"): a value's
//      key is its bin, min{k : value <= t_k}, or L (never active) for NaN,
//      values above every threshold and cells outside the domain;
//   2. every top cell (per-voxel path) or every vertex (per-vertex path)
//      computes its contribution changes and adds them to the block's
//      private shared-memory histogram (the per-thread arrays of Algorithm 2
//      become per-block arrays);
//   3. each block adds its histogram into one int64 global histogram;
//   4. a scan kernel forms the running sum over levels and divides by the
//      descriptor's integer scale.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ec_internal.h"
#include "ec_rules.h"

namespace ec {

__constant__ Table2D c_tab2 = make_table_2d();
__constant__ Table3D c_tab3 = make_table_3d();
__constant__ Table3D6 c_tab3e6 = make_table_3d_ec6();

constexpr int kThreads = 256;
constexpr int kSmemThrMax = 4096;   // thresholds live in shared memory up to this many levels

// 3D tile: TX x TY columns per block, walked along z.
constexpr int TX3 = 32, TY3 = 8;
constexpr int RW3 = TX3 + 2, RH3 = TY3 + 2, RS3 = RW3 * RH3;
// 2D tile: TX2 columns per block, walked along y.
constexpr int TX2 = 256;
constexpr int RW2 = TX2 + 2;
constexpr int kRing = 4;

// ----------------------------------------------------------------- binning

// Smallest k with x <= t[k]; L when none (NaN compares false everywhere).
template <typename T>
__device__ __forceinline__ int lower_bound_dev(T x, const T *__restrict__ t, int L)
{
    int lo = 0, n = L;
    while (n > 0) {
        const int half = n >> 1;
        if (!(x <= t[lo + half])) { lo += half + 1; n -= half + 1; }
        else n = half;
    }
    return lo;
}

// Per-block binning state in shared memory.
template <typename T>
struct Binner {
    int L;
    const T *thr;            // thresholds (shared or global), nullptr = identity
    const uint16_t *table;   // uint8 fields: bin of every byte value

    __device__ __forceinline__ uint32_t operator()(T v) const
    {
        if constexpr (sizeof(T) == 1) {
            return table[v];
        } else if constexpr (sizeof(T) == 2) {
            if (!thr) return v < (uint32_t)L ? (uint32_t)v : (uint32_t)L;
            return (uint32_t)lower_bound_dev<T>(v, thr, L);
        } else {
            return (uint32_t)lower_bound_dev<T>(v, thr, L);
        }
    }
};

// Shared bytes for binning tables of a request.
template <typename T>
__host__ __device__ inline size_t binner_smem_bytes(int L, bool has_thr)
{
    if (sizeof(T) == 1) return 256 * sizeof(uint16_t);
    if (has_thr && L <= kSmemThrMax) return ((size_t)L * sizeof(T) + 15) & ~(size_t)15;
    return 0;
}

template <typename T>
__device__ Binner<T> make_binner(const BinArgs &ba, unsigned char *sm)
{
    Binner<T> b;
    b.L = ba.L;
    b.thr = nullptr;
    b.table = nullptr;
    const T *gthr = (const T *)ba.thr;
    if constexpr (sizeof(T) == 1) {
        uint16_t *tab = (uint16_t *)sm;
        for (int v = threadIdx.x; v < 256; v += blockDim.x) {
            uint32_t bin;
            if (!gthr) bin = v < ba.L ? (uint32_t)v : (uint32_t)ba.L;
            else bin = (uint32_t)lower_bound_dev<T>((T)v, gthr, ba.L);
            tab[v] = (uint16_t)bin;
        }
        b.table = tab;
    } else {
        if (gthr && ba.L <= kSmemThrMax) {
            T *s = (T *)sm;
            for (int k = threadIdx.x; k < ba.L; k += blockDim.x) s[k] = gthr[k];
            b.thr = s;
        } else {
            b.thr = gthr;
        }
    }
    return b;
}

// ------------------------------------------------------------- histogram

struct BlockHist {
    int *sh;            // shared int32 [nd][L] or nullptr
    long long *g;       // global int64 [nd][L]
    int L;
    int row[kMaxDesc];

    __device__ __forceinline__ void add(int d, uint32_t bin, int v) const
    {
        const int r = row[d];
        if (r < 0 || v == 0) return;
        if (sh) atomicAdd(&sh[r * L + bin], v);
        else atomicAdd((unsigned long long *)&g[(size_t)r * L + bin], (unsigned long long)(long long)v);
    }
};

__device__ BlockHist make_hist(const HistArgs &ha, int L, unsigned char *sm)
{
    BlockHist h;
    h.L = L;
    h.g = ha.hist;
    for (int i = 0; i < kMaxDesc; i++) h.row[i] = ha.rows.row[i];
    h.sh = nullptr;
    if (ha.smem_hist) {
        h.sh = (int *)sm;
        for (int i = threadIdx.x; i < ha.rows.nd * L; i += blockDim.x) h.sh[i] = 0;
    }
    return h;
}

__device__ void flush_hist(const BlockHist &h, int nd)
{
    if (!h.sh) return;
    __syncthreads();
    for (int i = threadIdx.x; i < nd * h.L; i += blockDim.x) {
        const int v = h.sh[i];
        if (v) atomicAdd((unsigned long long *)&h.g[i], (unsigned long long)(long long)v);
    }
}

__host__ __device__ inline size_t hist_smem_bytes(const HistArgs &ha, int L)
{
    return ha.smem_hist ? (((size_t)ha.rows.nd * L * 4 + 15) & ~(size_t)15) : 0;
}

// ------------------------------------------------------- 3D field geometry

struct Geom3 {
    int64_t D, H, W;
    int nbx, nby, nbz, tz;   // tile counts and z planes per tile
    int vertex;              // 1: tiles cover the (D+1)(H+1)(W+1) vertex grid
    int64_t zc0, zc1;        // planes (voxel or vertex) this launch counts
    int64_t zv0, zv1;        // voxel planes that belong to the field
};

template <typename T>
__device__ __forceinline__ void stage_plane3(uint16_t *slot, const T *__restrict__ f, const Geom3 &g,
                                             const Binner<T> &bin, int64_t z, int64_t x0, int64_t y0)
{
    for (int i = threadIdx.x; i < RS3; i += blockDim.x) {
        const int ly = i / RW3, lx = i - ly * RW3;
        const int64_t gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        uint32_t key = (uint32_t)bin.L;
        if (z >= g.zv0 && z < g.zv1 && gx >= 0 && gx < g.W && gy >= 0 && gy < g.H)
            key = bin(f[(z * g.H + gy) * g.W + gx]);
        slot[i] = (uint16_t)key;
    }
}

// Per-voxel regrouped path: one histogram update per voxel at its own level.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_voxel3d(const T *__restrict__ f, Geom3 g, BinArgs ba, HistArgs ha,
                                                      int conn6)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t hb = hist_smem_bytes(ha, ba.L);
    BlockHist hist = make_hist(ha, ba.L, smem);
    Binner<T> bin = make_binner<T>(ba, smem + hb);
    uint16_t *ring = (uint16_t *)(smem + hb + binner_smem_bytes<T>(ba.L, ba.thr != nullptr));
    const uint32_t L = (uint32_t)ba.L;
    const int tx = threadIdx.x % TX3, ty = threadIdx.x / TX3;
    const int nitems = g.nbx * g.nby * g.nbz;

    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % g.nbx, by = (item / g.nbx) % g.nby, bz = item / (g.nbx * g.nby);
        const int64_t x0 = (int64_t)bx * TX3, y0 = (int64_t)by * TY3;
        const int64_t z0 = g.zc0 + (int64_t)bz * g.tz, z1 = min(z0 + g.tz, g.zc1);
        __syncthreads();   // ring reuse across items
        stage_plane3<T>(ring + ((z0 + 3) & 3) * RS3, f, g, bin, z0 - 1, x0, y0);
        stage_plane3<T>(ring + ((z0 + 4) & 3) * RS3, f, g, bin, z0, x0, y0);
        const int64_t x = x0 + tx, y = y0 + ty;
        const int c = (ty + 1) * RW3 + (tx + 1);
        for (int64_t z = z0; z < z1; z++) {
            stage_plane3<T>(ring + ((z + 5) & 3) * RS3, f, g, bin, z + 1, x0, y0);
            __syncthreads();
            const uint16_t *r0 = ring + ((z + 3) & 3) * RS3;
            const uint16_t *r1 = ring + ((z + 4) & 3) * RS3;
            const uint16_t *r2 = ring + ((z + 5) & 3) * RS3;
            const uint32_t kc = r1[c];
            if (x < g.W && y < g.H && kc < L) {
                uint32_t P = 0;
#pragma unroll
                for (int dz = -1; dz <= 1; dz++) {
                    const uint16_t *r = dz < 0 ? r0 : (dz == 0 ? r1 : r2);
#pragma unroll
                    for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                        for (int dx = -1; dx <= 1; dx++) {
                            if (dx == 0 && dy == 0 && dz == 0) continue;
                            const uint32_t kn = r[c + dy * RW3 + dx];
                            // neighbours earlier in linear order win ties
                            const bool lower = dz < 0 || (dz == 0 && (dy < 0 || (dy == 0 && dx < 0)));
                            const bool prec = lower ? (kn <= kc) : (kn < kc);
                            P |= (uint32_t)prec << ((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1));
                        }
                }
                const Delta3 d = voxel_delta_3d(P);
                hist.add(0, kc, conn6 ? voxel_delta_3d6(P) : d.ec);
                hist.add(1, kc, d.per);
                hist.add(2, kc, d.area);
                hist.add(3, kc, 1);
            }
        }
    }
    flush_hist(hist, ha.rows.nd);
}

// Sort 8 keys ascending (Batcher odd-even merge network, 19 comparators).
__device__ __forceinline__ void cswap(uint32_t &a, uint32_t &b)
{
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo; b = hi;
}
__device__ __forceinline__ void sort8(uint32_t s[8])
{
    cswap(s[0], s[1]); cswap(s[2], s[3]); cswap(s[4], s[5]); cswap(s[6], s[7]);
    cswap(s[0], s[2]); cswap(s[1], s[3]); cswap(s[4], s[6]); cswap(s[5], s[7]);
    cswap(s[1], s[2]); cswap(s[5], s[6]);
    cswap(s[0], s[4]); cswap(s[1], s[5]); cswap(s[2], s[6]); cswap(s[3], s[7]);
    cswap(s[2], s[4]); cswap(s[3], s[5]);
    cswap(s[1], s[2]); cswap(s[3], s[4]); cswap(s[5], s[6]);
}

// Per-vertex path (Algorithm 3 with Algorithm 4's neighbourhood fill): sort
// the vertex's 8 (level, position) keys, then walk the prefixes of the sorted
// order; the vertex type changes from T[m] to T[m | bit] at each value.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_vertex3d(const T *__restrict__ f, Geom3 g, BinArgs ba, HistArgs ha,
                                                       int conn6)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t hb = hist_smem_bytes(ha, ba.L);
    BlockHist hist = make_hist(ha, ba.L, smem);
    const size_t bb = binner_smem_bytes<T>(ba.L, ba.thr != nullptr);
    Binner<T> bin = make_binner<T>(ba, smem + hb);
    int4 *tab = (int4 *)(smem + hb + bb);
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        tab[i] = make_int4(conn6 ? c_tab3e6.v[i] : c_tab3.v[i][0], c_tab3.v[i][1], c_tab3.v[i][2], c_tab3.v[i][3]);
    uint16_t *ring = (uint16_t *)(smem + hb + bb + 256 * sizeof(int4));
    const uint32_t L = (uint32_t)ba.L;
    const int tx = threadIdx.x % TX3, ty = threadIdx.x / TX3;
    const int nitems = g.nbx * g.nby * g.nbz;

    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % g.nbx, by = (item / g.nbx) % g.nby, bz = item / (g.nbx * g.nby);
        const int64_t x0 = (int64_t)bx * TX3, y0 = (int64_t)by * TY3;
        const int64_t z0 = g.zc0 + (int64_t)bz * g.tz, z1 = min(z0 + g.tz, g.zc1);
        __syncthreads();
        stage_plane3<T>(ring + ((z0 + 3) & 3) * RS3, f, g, bin, z0 - 1, x0, y0);
        const int64_t X = x0 + tx, Y = y0 + ty;
        for (int64_t Z = z0; Z < z1; Z++) {
            stage_plane3<T>(ring + ((Z + 4) & 3) * RS3, f, g, bin, Z, x0, y0);
            __syncthreads();
            if (X > g.W || Y > g.H) continue;
            const uint16_t *rz[2] = {ring + ((Z + 3) & 3) * RS3, ring + ((Z + 4) & 3) * RS3};
            uint32_t s[8];
#pragma unroll
            for (int b = 0; b < 8; b++) {
                const int dx = b & 1, dy = (b >> 1) & 1, dz = b >> 2;
                s[b] = ((uint32_t)rz[dz][(ty + dy) * RW3 + tx + dx] << 3) | (uint32_t)b;
            }
            sort8(s);
            uint32_t cur = s[0] >> 3;
            if (cur >= L) continue;
            unsigned m = 0;
            int4 prev = make_int4(0, 0, 0, 0), acc = make_int4(0, 0, 0, 0);
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const uint32_t b = s[j] >> 3;
                if (b != cur) {
                    hist.add(0, cur, acc.x); hist.add(1, cur, acc.y);
                    hist.add(2, cur, acc.z); hist.add(3, cur, acc.w);
                    acc = make_int4(0, 0, 0, 0);
                    cur = b;
                    if (cur >= L) break;
                }
                m |= 1u << (s[j] & 7u);
                const int4 e = tab[m];
                acc.x += e.x - prev.x; acc.y += e.y - prev.y; acc.z += e.z - prev.z; acc.w += e.w - prev.w;
                prev = e;
            }
            if (cur < L) {
                hist.add(0, cur, acc.x); hist.add(1, cur, acc.y);
                hist.add(2, cur, acc.z); hist.add(3, cur, acc.w);
            }
        }
    }
    flush_hist(hist, ha.rows.nd);
}

// ------------------------------------------------------------------- 2D

struct Geom2 {
    int64_t H, W;
    int nbx, nby, ty;   // tile counts, rows per tile
};

template <typename T>
__device__ __forceinline__ void stage_row2(uint16_t *slot, const T *__restrict__ f, const Geom2 &g,
                                           const Binner<T> &bin, int64_t y, int64_t x0)
{
    for (int i = threadIdx.x; i < RW2; i += blockDim.x) {
        const int64_t gx = x0 - 1 + i;
        uint32_t key = (uint32_t)bin.L;
        if (y >= 0 && y < g.H && gx >= 0 && gx < g.W) key = bin(f[y * g.W + gx]);
        slot[i] = (uint16_t)key;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_pixel2d(const T *__restrict__ f, Geom2 g, BinArgs ba, HistArgs ha, int conn4)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t hb = hist_smem_bytes(ha, ba.L);
    BlockHist hist = make_hist(ha, ba.L, smem);
    Binner<T> bin = make_binner<T>(ba, smem + hb);
    uint16_t *ring = (uint16_t *)(smem + hb + binner_smem_bytes<T>(ba.L, ba.thr != nullptr));
    const uint32_t L = (uint32_t)ba.L;
    const int tx = threadIdx.x;
    const int nitems = g.nbx * g.nby;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % g.nbx, by = item / g.nbx;
        const int64_t x0 = (int64_t)bx * TX2;
        const int64_t y0 = (int64_t)by * g.ty, y1 = min(y0 + g.ty, g.H);
        __syncthreads();
        stage_row2<T>(ring + ((y0 + 3) & 3) * RW2, f, g, bin, y0 - 1, x0);
        stage_row2<T>(ring + ((y0 + 4) & 3) * RW2, f, g, bin, y0, x0);
        const int64_t x = x0 + tx;
        for (int64_t y = y0; y < y1; y++) {
            stage_row2<T>(ring + ((y + 5) & 3) * RW2, f, g, bin, y + 1, x0);
            __syncthreads();
            const uint16_t *rr[3] = {ring + ((y + 3) & 3) * RW2, ring + ((y + 4) & 3) * RW2,
                                     ring + ((y + 5) & 3) * RW2};
            const uint32_t kc = rr[1][tx + 1];
            if (x < g.W && kc < L) {
                uint32_t P = 0;
#pragma unroll
                for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                    for (int dx = -1; dx <= 1; dx++) {
                        if (dx == 0 && dy == 0) continue;
                        const uint32_t kn = rr[dy + 1][tx + 1 + dx];
                        const bool lower = dy < 0 || (dy == 0 && dx < 0);
                        const bool prec = lower ? (kn <= kc) : (kn < kc);
                        P |= (uint32_t)prec << ((dx + 1) + 3 * (dy + 1));
                    }
                const Delta2 d = pixel_delta_2d(P);
                hist.add(0, kc, conn4 ? d.ec4 : d.ec8);
                hist.add(1, kc, d.per);
                hist.add(2, kc, 1);
            }
        }
    }
    flush_hist(hist, ha.rows.nd);
}

// Per-vertex 2D path (Algorithms 1-2): sort the 4 values around the vertex and
// add the Table 1 type change at each of them.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_vertex2d(const T *__restrict__ f, Geom2 g, BinArgs ba, HistArgs ha, int conn4)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t hb = hist_smem_bytes(ha, ba.L);
    BlockHist hist = make_hist(ha, ba.L, smem);
    const size_t bb = binner_smem_bytes<T>(ba.L, ba.thr != nullptr);
    Binner<T> bin = make_binner<T>(ba, smem + hb);
    int4 *tab = (int4 *)(smem + hb + bb);
    for (int i = threadIdx.x; i < 16; i += blockDim.x)
        tab[i] = make_int4(conn4 ? c_tab2.v[i][1] : c_tab2.v[i][0], c_tab2.v[i][2], c_tab2.v[i][3], 0);
    uint16_t *ring = (uint16_t *)(smem + hb + bb + 16 * sizeof(int4));
    const uint32_t L = (uint32_t)ba.L;
    const int tx = threadIdx.x;
    const int nitems = g.nbx * g.nby;
    const int64_t NY = g.H + 1;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % g.nbx, by = item / g.nbx;
        const int64_t x0 = (int64_t)bx * TX2;
        const int64_t y0 = (int64_t)by * g.ty, y1 = min(y0 + g.ty, NY);
        __syncthreads();
        stage_row2<T>(ring + ((y0 + 3) & 3) * RW2, f, g, bin, y0 - 1, x0);
        const int64_t X = x0 + tx;
        for (int64_t Y = y0; Y < y1; Y++) {
            stage_row2<T>(ring + ((Y + 4) & 3) * RW2, f, g, bin, Y, x0);
            __syncthreads();
            if (X > g.W) continue;
            const uint16_t *ry[2] = {ring + ((Y + 3) & 3) * RW2, ring + ((Y + 4) & 3) * RW2};
            uint32_t s[4];
#pragma unroll
            for (int b = 0; b < 4; b++) s[b] = ((uint32_t)ry[b >> 1][tx + (b & 1)] << 2) | (uint32_t)b;
            cswap(s[0], s[1]); cswap(s[2], s[3]); cswap(s[0], s[2]); cswap(s[1], s[3]); cswap(s[1], s[2]);
            uint32_t cur = s[0] >> 2;
            if (cur >= L) continue;
            unsigned m = 0;
            int4 prev = make_int4(0, 0, 0, 0), acc = make_int4(0, 0, 0, 0);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t b = s[j] >> 2;
                if (b != cur) {
                    hist.add(0, cur, acc.x); hist.add(1, cur, acc.y); hist.add(2, cur, acc.z);
                    acc = make_int4(0, 0, 0, 0);
                    cur = b;
                    if (cur >= L) break;
                }
                m |= 1u << (s[j] & 3u);
                const int4 e = tab[m];
                acc.x += e.x - prev.x; acc.y += e.y - prev.y; acc.z += e.z - prev.z;
                prev = e;
            }
            if (cur < L) { hist.add(0, cur, acc.x); hist.add(1, cur, acc.y); hist.add(2, cur, acc.z); }
        }
    }
    flush_hist(hist, ha.rows.nd);
}

// -------------------------------------------------------------- scan kernel

struct Scales { int32_t s[kMaxDesc]; };

__global__ void __launch_bounds__(1024) k_scan(const long long *__restrict__ hist, int L, Scales sc,
                                               int64_t *__restrict__ out, int *err)
{
    __shared__ long long warp_tot[32];
    const int row = blockIdx.x;
    const long long *h = hist + (size_t)row * L;
    int64_t *o = out + (size_t)row * L;
    const long long scale = sc.s[row];
    if (*(volatile int *)err & 4) {   // a histogram block gave up a bounded wait: poison the curve
        for (int k = threadIdx.x; k < L; k += blockDim.x) o[k] = INT64_MIN;
        return;
    }
    const int per = (L + blockDim.x - 1) / blockDim.x;
    const int beg = min((int)threadIdx.x * per, L), end = min(beg + per, L);
    long long s = 0;
    for (int k = beg; k < end; k++) s += h[k];
    // block-wide exclusive scan of the per-thread sums
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
        const long long q = run / scale;
        if (q * scale != run) atomicOr(err, 1);
        o[k] = q;
    }
}

__global__ void k_check_sorted_f32(const float *t, int L, int *flag)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k + 1 < L; k += gridDim.x * blockDim.x)
        if (!(t[k] <= t[k + 1])) atomicOr(flag, 1);
    if (blockIdx.x == 0 && threadIdx.x == 0 && L >= 1 && t[0] != t[0]) atomicOr(flag, 1);
}
template <typename T>
__global__ void k_check_sorted_int(const T *t, int L, int *flag)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k + 1 < L; k += gridDim.x * blockDim.x)
        if (t[k] > t[k + 1]) atomicOr(flag, 1);
}

// ------------------------------------------------------------ host launch

template <typename KernelT>
static int prepare_kernel(KernelT kernel, size_t smem, int num_sms, int items, int grid_override, int *grid_out)
{
    int occ = 0;
    if (const int orc = kernel_occupancy((const void *)kernel, kThreads, smem, &occ)) return orc;
    if (occ < 1) {
        set_error("kernel does not fit on an SM (%zu bytes of shared memory)", smem);
        return EC_ERR_UNSUPPORTED;
    }
    int grid = grid_override > 0 ? grid_override : num_sms * occ;
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    *grid_out = grid;
    return EC_OK;
}

template <typename T>
static int launch3(const void *field, const int64_t dims[3], const BinArgs &ba, const HistArgs &ha,
                   int algo, int tile_z, int grid_override, int num_sms, cudaStream_t s, const int zrange[4],
                   int conn6)
{
    Geom3 g;
    g.D = dims[0]; g.H = dims[1]; g.W = dims[2];
    const bool vertex = algo == ALGO_VERTEX;
    g.vertex = vertex ? 1 : 0;
    g.zc0 = zrange ? zrange[0] : 0;
    g.zc1 = zrange ? zrange[1] : (vertex ? g.D + 1 : g.D);
    g.zv0 = zrange ? zrange[2] : 0;
    g.zv1 = zrange ? zrange[3] : g.D;
    const int64_t nx = vertex ? g.W + 1 : g.W, ny = vertex ? g.H + 1 : g.H, nz = g.zc1 - g.zc0;
    if (nz < 1) return EC_OK;
    g.tz = tile_z > 0 ? tile_z : 32;
    g.nbx = (int)((nx + TX3 - 1) / TX3);
    g.nby = (int)((ny + TY3 - 1) / TY3);
    g.nbz = (int)((nz + g.tz - 1) / g.tz);
    const int64_t items64 = (int64_t)g.nbx * g.nby * g.nbz;
    if (items64 > INT32_MAX) { set_error("field too large for one launch"); return EC_ERR_UNSUPPORTED; }
    const int items = (int)items64;
    size_t smem = hist_smem_bytes(ha, ba.L) + binner_smem_bytes<T>(ba.L, ba.thr != nullptr) +
                  (vertex ? 256 * sizeof(int4) : 0) + kRing * RS3 * sizeof(uint16_t);
    int grid = 0;
    if (vertex) {
        int rc = prepare_kernel(k_vertex3d<T>, smem, num_sms, items, grid_override, &grid);
        if (rc) return rc;
        k_vertex3d<T><<<grid, kThreads, smem, s>>>((const T *)field, g, ba, ha, conn6);
    } else {
        int rc = prepare_kernel(k_voxel3d<T>, smem, num_sms, items, grid_override, &grid);
        if (rc) return rc;
        k_voxel3d<T><<<grid, kThreads, smem, s>>>((const T *)field, g, ba, ha, conn6);
    }
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

int launch_curve_3d(const void *field, const int64_t dims[3], const BinArgs &ba, const HistArgs &ha,
                    int algo, int tile_z, int grid, int num_sms, cudaStream_t s, const int zrange[4], int conn6)
{
    switch (ba.dtype) {
    case EC_U8: return launch3<uint8_t>(field, dims, ba, ha, algo, tile_z, grid, num_sms, s, zrange, conn6);
    case EC_U16: return launch3<uint16_t>(field, dims, ba, ha, algo, tile_z, grid, num_sms, s, zrange, conn6);
    case EC_F32: return launch3<float>(field, dims, ba, ha, algo, tile_z, grid, num_sms, s, zrange, conn6);
    }
    set_error("unknown dtype %d", ba.dtype);
    return EC_ERR_DTYPE;
}

template <typename T>
static int launch2(const void *field, const int64_t dims[2], const BinArgs &ba, const HistArgs &ha,
                   int conn, int algo, int grid_override, int num_sms, cudaStream_t s)
{
    Geom2 g;
    g.H = dims[0]; g.W = dims[1];
    const bool vertex = algo == ALGO_VERTEX;
    const int64_t nx = vertex ? g.W + 1 : g.W, ny = vertex ? g.H + 1 : g.H;
    g.ty = 64;
    g.nbx = (int)((nx + TX2 - 1) / TX2);
    g.nby = (int)((ny + g.ty - 1) / g.ty);
    const int64_t items64 = (int64_t)g.nbx * g.nby;
    if (items64 > INT32_MAX) { set_error("field too large for one launch"); return EC_ERR_UNSUPPORTED; }
    const int items = (int)items64;
    size_t smem = hist_smem_bytes(ha, ba.L) + binner_smem_bytes<T>(ba.L, ba.thr != nullptr) +
                  (vertex ? 16 * sizeof(int4) : 0) + kRing * RW2 * sizeof(uint16_t);
    int grid = 0;
    const int conn4 = conn == 4 ? 1 : 0;
    if (vertex) {
        int rc = prepare_kernel(k_vertex2d<T>, smem, num_sms, items, grid_override, &grid);
        if (rc) return rc;
        k_vertex2d<T><<<grid, kThreads, smem, s>>>((const T *)field, g, ba, ha, conn4);
    } else {
        int rc = prepare_kernel(k_pixel2d<T>, smem, num_sms, items, grid_override, &grid);
        if (rc) return rc;
        k_pixel2d<T><<<grid, kThreads, smem, s>>>((const T *)field, g, ba, ha, conn4);
    }
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

int launch_curve_2d(const void *field, const int64_t dims[2], const BinArgs &ba, const HistArgs &ha,
                    int connectivity, int algo, int grid, int num_sms, cudaStream_t s)
{
    switch (ba.dtype) {
    case EC_U8: return launch2<uint8_t>(field, dims, ba, ha, connectivity, algo, grid, num_sms, s);
    case EC_U16: return launch2<uint16_t>(field, dims, ba, ha, connectivity, algo, grid, num_sms, s);
    case EC_F32: return launch2<float>(field, dims, ba, ha, connectivity, algo, grid, num_sms, s);
    }
    set_error("unknown dtype %d", ba.dtype);
    return EC_ERR_DTYPE;
}

int launch_scan(const long long *hist, int nd, int32_t L, const int32_t scale[kMaxDesc], int64_t *out,
                int *err_flag, cudaStream_t s)
{
    Scales sc;
    for (int i = 0; i < kMaxDesc; i++) sc.s[i] = scale[i] > 0 ? scale[i] : 1;
    // one thread per level up to 1024 (short curves start fewer idle warps)
    const int threads = (int)std::min<int64_t>(1024, std::max<int64_t>(32, ((int64_t)L + 31) / 32 * 32));
    k_scan<<<nd, threads, 0, s>>>(hist, L, sc, out, err_flag);
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

int launch_check_sorted(const void *thr, int dtype, int32_t L, int *flag, cudaStream_t s)
{
    const int blocks = (L + 255) / 256;
    if (dtype == EC_F32) k_check_sorted_f32<<<blocks, 256, 0, s>>>((const float *)thr, L, flag);
    else if (dtype == EC_U16) k_check_sorted_int<uint16_t><<<blocks, 256, 0, s>>>((const uint16_t *)thr, L, flag);
    else k_check_sorted_int<uint8_t><<<blocks, 256, 0, s>>>((const uint8_t *)thr, L, flag);
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

void row_scales(int ndim, int algo, uint32_t desc, int32_t out[kMaxDesc])
{
    // per-vertex tables are scaled; the per-top-cell closed forms are not
    static const int32_t s2[kMaxDesc] = {4, 2, 4, 1};
    static const int32_t s3[kMaxDesc] = {8, 2, 4, 8};
    int r = 0;
    for (int i = 0; i < kMaxDesc; i++) out[i] = 1;
    for (int i = 0; i < kMaxDesc; i++) {
        if (!(desc & (1u << i))) continue;
        out[r++] = algo == ALGO_VERTEX ? (ndim == 2 ? s2[i] : s3[i]) : 1;
    }
}

// Host copies of the tables for inspection and self-checks.
const Table2D &host_table_2d()
{
    static const Table2D t = make_table_2d();
    return t;
}
const Table3D &host_table_3d()
{
    static const Table3D t = make_table_3d();
    return t;
}

}  // namespace ec

// ec_gen.cu -- on-device generator of the hash-box field used as the
// low-memory (streaming) workload.  This is input generation, not part of
// the EC computation.
//
//   m(u)     = MurmurHash3's 32-bit finaliser (Appleby): u ^= u >> 16;
//              u *= 0x85EBCA6B; u ^= u >> 13; u *= 0xC2B2AE35; u ^= u >> 16
//   a        = m(lo32(seed) ^ m(hi32(seed)))
//   u(p,y,z) = m(m(m(a ^ z) ^ y) ^ p)                   (p, y, z mod 2^32)
//   h(x,y,z) = low 16 bits of u(floor(x/2), y, z) for even x, its high
//              16 bits for odd x (one finaliser serves two neighbours)
//   v(x,y,z) = floor( sum over the 5x5x5 box around (x,y,z) of h / 2000 )
// (4096 / (125 * 65536) = 1 / 2000, so v lies in [0, 4095]).  The field is
// defined for every integer coordinate, so any sub-box can be generated.
//
// One block of 288 threads produces a 64 x 32 column of outputs and walks it
// along z with one barrier per input plane.  Per input plane: eight threads
// per row of the 68 x 36 neighbourhood each form nine consecutive hashes
// (five finalisers, halves picked by the run's parity; the per-row keys
// m(m(a ^ z) ^ y) are formed one plane ahead by 36 threads), take the next
// thread's first four hashes by a warp shuffle (a row's eight threads are
// consecutive lanes of one warp) and write their nine 5-wide sums along x
// into one of two x-sum buffers; after the barrier each of the first 256
// threads sums 5 rows of those for its 4 x 2 outputs, and a running sum
// over the last five planes (a register ring indexed at compile time: the
// plane loop is unrolled by five) gives the sum along z.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ec_internal.h"

namespace {

constexpr int GX = 64, GY = 32, HY = GY + 4;
constexpr int SEG = 9, NSEG = 8;          // hashes per thread, threads per row (columns 0..71 of the 68 needed)
constexpr int kGenThreads = HY * NSEG;    // 288 = 9 warps, four rows per warp
// x-sum row pitch: 72 words put the four rows of a warp's nine-wide stores on
// distinct banks (rows 64 words apart would share 8 banks four times over)
constexpr int XP = GX + 8;
static_assert(32 % NSEG == 0, "a row's threads share one warp");

__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t u)
{
    u ^= u >> 16;
    u *= 0x85EBCA6Bu;
    u ^= u >> 13;
    u *= 0xC2B2AE35u;
    u ^= u >> 16;
    return u;
}

struct GenCtx {
    uint32_t a;
    int64_t ox, oy, oz, nx, ny, nz, bx0, by0;
    int tx, ty;
    int hrow, hseg;          // this thread's hash row and 9-wide run
    uint16_t *out[2];        // output rows 2ty, 2ty+1 of plane 0 at x = bx0 + 4tx (nullptr: past the box)
    int64_t plane;           // elements per output plane
    bool vec;                // four outputs as one 8-byte store
};

// Row keys of input plane k (relative to oz) into rk: threads 0..HY-1.
__device__ __forceinline__ void row_keys(const GenCtx &g, int64_t k, uint32_t *rk)
{
    if (threadIdx.x < HY) {
        const uint32_t pk = fmix32(g.a ^ (uint32_t)(g.oz + k));
        rk[threadIdx.x] = fmix32(pk ^ (uint32_t)(g.oy + g.by0 - 2 + (int64_t)threadIdx.x));
    }
}

// One input plane k: hashes and sums along x (all threads), then, after the
// block's barrier, sums along y, the running sum along z (ring slot J holds
// this plane's sums until five planes later), and the output plane k - 2 once
// its five-plane window is complete (the first 256 threads).
template <int J>
__device__ __forceinline__ void gen_plane(const GenCtx &g, int64_t k, uint32_t (*xs)[HY][XP], uint32_t (*rk)[HY],
                                          uint32_t (&ring)[5][8], uint32_t (&zs)[8])
{
    {
        row_keys(g, k + 1, rk[(k + 1) & 1]);   // read after this plane's barrier
        const uint32_t key = rk[k & 1][g.hrow];
        const int64_t x0 = g.ox + g.bx0 - 2 + SEG * g.hseg;
        const int64_t pe = (x0 - (x0 & 1)) / 2;   // floor(x0 / 2)
        const bool odd = (x0 & 1) != 0;
        uint32_t u[5];
#pragma unroll
        for (int i = 0; i < 5; i++) u[i] = fmix32(key ^ (uint32_t)(pe + i));
        // hash of x0 + j: half ((j + odd) & 1) of u[(j + odd) >> 1]
        uint32_t h[SEG + 4];
#pragma unroll
        for (int j = 0; j < SEG; j++) {
            const uint32_t ev = (j & 1) ? (u[j >> 1] >> 16) : (u[j >> 1] & 0xFFFFu);
            const uint32_t od = ((j + 1) & 1) ? (u[(j + 1) >> 1] >> 16) : (u[(j + 1) >> 1] & 0xFFFFu);
            h[j] = odd ? od : ev;
        }
        // the next run's first four hashes (the row's last thread needs none)
#pragma unroll
        for (int j = 0; j < 4; j++) h[SEG + j] = __shfl_down_sync(0xffffffffu, h[j], 1);
        uint32_t *xr = xs[k & 1][g.hrow];
        const int c0 = SEG * g.hseg;
        uint32_t sum = h[0] + h[1] + h[2] + h[3] + h[4];
        xr[c0] = sum;   // c0 <= 63
        if (g.hseg < NSEG - 1) {
#pragma unroll
            for (int i = 1; i < SEG; i++) {
                sum += h[i + 4] - h[i - 1];
                xr[c0 + i] = sum;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x >= 256) return;   // no outputs of its own
    uint4 r[6];
#pragma unroll
    for (int j = 0; j < 6; j++) r[j] = *(const uint4 *)&xs[k & 1][2 * g.ty + j][4 * g.tx];
    uint32_t s[8];
    s[0] = r[0].x + r[1].x + r[2].x + r[3].x + r[4].x;
    s[1] = r[0].y + r[1].y + r[2].y + r[3].y + r[4].y;
    s[2] = r[0].z + r[1].z + r[2].z + r[3].z + r[4].z;
    s[3] = r[0].w + r[1].w + r[2].w + r[3].w + r[4].w;
    s[4] = s[0] - r[0].x + r[5].x;
    s[5] = s[1] - r[0].y + r[5].y;
    s[6] = s[2] - r[0].z + r[5].z;
    s[7] = s[3] - r[0].w + r[5].w;
#pragma unroll
    for (int b = 0; b < 8; b++) {
        zs[b] += s[b] - ring[J][b];   // the plane five back leaves the window
        ring[J][b] = s[b];
    }
    const int64_t zo = k - 2;   // output plane whose 5-plane window just completed
    if (zo < 0) return;
    const int64_t x = g.bx0 + 4 * g.tx;
#pragma unroll
    for (int yy = 0; yy < 2; yy++) {
        if (!g.out[yy]) continue;
        uint32_t v[4];
#pragma unroll
        for (int b = 0; b < 4; b++) v[b] = zs[4 * yy + b] / 2000u;
        uint16_t *o = g.out[yy] + zo * g.plane;
        if (g.vec) {
            *(uint2 *)o = make_uint2(v[0] | (v[1] << 16), v[2] | (v[3] << 16));
        } else {
#pragma unroll
            for (int b = 0; b < 4; b++)
                if (x + b < g.nx) o[b] = (uint16_t)v[b];
        }
    }
}

__global__ void __launch_bounds__(kGenThreads, 2) k_hashbox(uint64_t seed, int64_t ox, int64_t oy, int64_t oz,
                                                         int64_t nx, int64_t ny, int64_t nz,
                                                         uint16_t *__restrict__ dst)
{
    __shared__ __align__(16) uint32_t xs[2][HY][XP];   // 5-wide sums along x, this plane and the next
    __shared__ uint32_t rk[2][HY];                     // row keys of this plane and the next
    GenCtx g;
    g.a = fmix32((uint32_t)seed ^ fmix32((uint32_t)(seed >> 32)));
    g.ox = ox; g.oy = oy; g.oz = oz; g.nx = nx; g.ny = ny; g.nz = nz;
    g.bx0 = (int64_t)blockIdx.x * GX;
    g.by0 = (int64_t)blockIdx.y * GY;
    g.tx = threadIdx.x & 15;   // outputs x 4tx .. 4tx+3
    g.ty = threadIdx.x >> 4;   // outputs y 2ty, 2ty+1
    g.hrow = threadIdx.x / NSEG;
    g.hseg = threadIdx.x - g.hrow * NSEG;
    g.plane = ny * nx;
    const int64_t x = g.bx0 + 4 * g.tx;
    for (int yy = 0; yy < 2; yy++) {
        const int64_t y = g.by0 + 2 * g.ty + yy;
        g.out[yy] = (y < ny && x < nx) ? dst + y * nx + x : nullptr;
    }
    // rows, planes and x all keep 8-byte alignment when nx is a multiple of 4
    g.vec = x + 3 < nx && (nx & 3) == 0 && ((uintptr_t)dst & 7u) == 0;
    uint32_t ring[5][8], zs[8];
#pragma unroll
    for (int b = 0; b < 8; b++) {
        zs[b] = 0;
#pragma unroll
        for (int a = 0; a < 5; a++) ring[a][b] = 0;
    }
    row_keys(g, -2, rk[(-2) & 1]);
    __syncthreads();   // the first plane's keys
    // input planes -2 .. nz+1; ring slot = (k + 2) mod 5
    const int64_t kend = nz + 2;
    for (int64_t k = -2; k < kend; k += 5) {
        gen_plane<0>(g, k, xs, rk, ring, zs);
        if (k + 1 < kend) gen_plane<1>(g, k + 1, xs, rk, ring, zs);
        if (k + 2 < kend) gen_plane<2>(g, k + 2, xs, rk, ring, zs);
        if (k + 3 < kend) gen_plane<3>(g, k + 3, xs, rk, ring, zs);
        if (k + 4 < kend) gen_plane<4>(g, k + 4, xs, rk, ring, zs);
    }
}

}  // namespace

using namespace ec;

extern "C" int ec_gen_hashbox_u16(uint64_t seed, int64_t x0, int64_t y0, int64_t z0, int64_t nx, int64_t ny,
                                  int64_t nz, void *dst_dev, void *stream)
{
    clear_error();
    if (nx < 1 || ny < 1 || nz < 1 || !dst_dev) { set_error("bad hash-box request"); return EC_ERR_ARG; }
    if ((nx + GX - 1) / GX > INT32_MAX || (ny + GY - 1) / GY > 65535) { set_error("hash box too wide"); return EC_ERR_ARG; }
    dim3 grid((unsigned)((nx + GX - 1) / GX), (unsigned)((ny + GY - 1) / GY));
    k_hashbox<<<grid, kGenThreads, 0, (cudaStream_t)stream>>>(seed, x0, y0, z0, nx, ny, nz, (uint16_t *)dst_dev);
    EC_CUDA(cudaGetLastError());
    return EC_OK;
}

extern "C" int ec_hashbox_producer(void *user, int64_t z0, int64_t z1, void *dst_dev, void *stream)
{
    const ec_hashbox_spec *spec = (const ec_hashbox_spec *)user;
    if (!spec) return EC_ERR_ARG;
    return ec_gen_hashbox_u16(spec->seed, spec->x0, spec->y0, spec->z0 + z0, spec->nx, spec->ny, z1 - z0, dst_dev,
                              stream);
}

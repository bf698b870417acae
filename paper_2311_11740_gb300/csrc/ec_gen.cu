// ec_gen.cu -- on-device generator of the hash-box field used as the
// low-memory (streaming) workload.  This is input generation, not part of
// the EC computation.
//
//   h(x,y,z) = low 16 bits of SplitMix64(seed*2^48 ^ (z mod 2^16)*2^32
//                                        ^ (y mod 2^16)*2^16 ^ (x mod 2^16))
//   v(x,y,z) = floor( sum over the 5x5x5 box around (x,y,z) of h / 2000 )
// (4096 / (125 * 65536) = 1 / 2000, so v lies in [0, 4095]).  SplitMix64 is
// Steele, Lea and Flood's published finaliser (OOPSLA 2014).  The field is
// defined for every integer coordinate, so any sub-box can be generated.
//
// One block produces a 64 x 32 column of outputs and walks it along z.  Per
// input plane: the 68 x 36 hashes of its neighbourhood go to shared memory
// (1.2 hashes per output), 5-wide sums along x are formed four at a time as
// running sums, and each thread sums 5 rows of those for its 4 x 2 outputs
// and keeps the last five such plane sums in registers for the sum along z.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ec_internal.h"

namespace {

constexpr int GX = 64, GY = 32, HX = GX + 4, HY = GY + 4;

__device__ __forceinline__ uint32_t hash16(uint64_t seed, int64_t x, int64_t y, int64_t z)
{
    uint64_t v = (seed << 48) ^ (((uint64_t)z & 0xFFFFull) << 32) ^ (((uint64_t)y & 0xFFFFull) << 16) ^
                 ((uint64_t)x & 0xFFFFull);
    v += 0x9E3779B97F4A7C15ull;
    v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
    v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
    v ^= v >> 31;
    return (uint32_t)(v & 0xFFFFull);
}

__global__ void __launch_bounds__(256) k_hashbox(uint64_t seed, int64_t ox, int64_t oy, int64_t oz, int64_t nx,
                                                 int64_t ny, int64_t nz, uint16_t *__restrict__ dst)
{
    __shared__ __align__(16) uint32_t hs[HY][HX];   // hashes of the plane's neighbourhood
    __shared__ __align__(16) uint32_t xs[HY][GX];   // 5-wide sums along x
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // outputs x 4tx .. 4tx+3, y 2ty, 2ty+1
    const int64_t bx0 = (int64_t)blockIdx.x * GX, by0 = (int64_t)blockIdx.y * GY;
    uint32_t ring[5][8];
#pragma unroll
    for (int a = 0; a < 5; a++)
#pragma unroll
        for (int b = 0; b < 8; b++) ring[a][b] = 0;
    for (int64_t k = -2; k < nz + 2; k++) {
        const int64_t z = oz + k;
        for (int i = threadIdx.x; i < HX * HY; i += blockDim.x) {
            const int ly = i / HX, lx = i - ly * HX;
            hs[ly][lx] = hash16(seed, ox + bx0 - 2 + lx, oy + by0 - 2 + ly, z);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < HY * (GX / 4); i += blockDim.x) {
            const int ly = i >> 4, q = i & 15;
            const uint4 a = *(const uint4 *)&hs[ly][4 * q], b = *(const uint4 *)&hs[ly][4 * q + 4];
            uint4 o;
            o.x = a.x + a.y + a.z + a.w + b.x;
            o.y = o.x - a.x + b.y;
            o.z = o.y - a.y + b.z;
            o.w = o.z - a.z + b.w;
            *(uint4 *)&xs[ly][4 * q] = o;
        }
        __syncthreads();
        uint4 r[6];
#pragma unroll
        for (int j = 0; j < 6; j++) r[j] = *(const uint4 *)&xs[2 * ty + j][4 * tx];
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
            ring[0][b] = ring[1][b]; ring[1][b] = ring[2][b]; ring[2][b] = ring[3][b]; ring[3][b] = ring[4][b];
            ring[4][b] = s[b];
        }
        const int64_t zo = k - 2;   // output plane whose 5-plane window just completed
        if (zo >= 0) {
#pragma unroll
            for (int yy = 0; yy < 2; yy++) {
                const int64_t y = by0 + 2 * ty + yy, x = bx0 + 4 * tx;
                if (y >= ny) continue;
                uint16_t v[4];
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const int e = 4 * yy + b;
                    v[b] = (uint16_t)((ring[0][e] + ring[1][e] + ring[2][e] + ring[3][e] + ring[4][e]) / 2000u);
                }
                uint16_t *row = dst + (zo * ny + y) * nx;
#pragma unroll
                for (int b = 0; b < 4; b++)
                    if (x + b < nx) row[x + b] = v[b];
            }
        }
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
    k_hashbox<<<grid, 256, 0, (cudaStream_t)stream>>>(seed, x0, y0, z0, nx, ny, nz, (uint16_t *)dst_dev);
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

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
// One block produces a 32 x 8 column of outputs and walks it along z: per
// input plane it hashes the 36 x 12 neighbourhood into shared memory, sums
// 5-wide along x then y, and keeps the last five 2D sums in registers for
// the sum along z.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ec_internal.h"

namespace {

constexpr int GX = 32, GY = 8, HX = GX + 4, HY = GY + 4;

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
    __shared__ uint32_t hs[HY][HX];
    __shared__ uint32_t xs[HY][GX];
    const int tx = threadIdx.x % GX, ty = threadIdx.x / GX;
    const int64_t bx0 = (int64_t)blockIdx.x * GX, by0 = (int64_t)blockIdx.y * GY;
    uint32_t ring[5] = {0, 0, 0, 0, 0};
    for (int64_t k = -2; k < nz + 2; k++) {
        const int64_t z = oz + k;
        for (int i = threadIdx.x; i < HX * HY; i += blockDim.x) {
            const int ly = i / HX, lx = i - ly * HX;
            hs[ly][lx] = hash16(seed, ox + bx0 - 2 + lx, oy + by0 - 2 + ly, z);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < HY * GX; i += blockDim.x) {
            const int ly = i / GX, lx = i - ly * GX;
            xs[ly][lx] = hs[ly][lx] + hs[ly][lx + 1] + hs[ly][lx + 2] + hs[ly][lx + 3] + hs[ly][lx + 4];
        }
        __syncthreads();
        const uint32_t s2 = xs[ty][tx] + xs[ty + 1][tx] + xs[ty + 2][tx] + xs[ty + 3][tx] + xs[ty + 4][tx];
        ring[0] = ring[1]; ring[1] = ring[2]; ring[2] = ring[3]; ring[3] = ring[4]; ring[4] = s2;
        const int64_t zo = k - 2;   // output plane whose 5-plane window just completed
        if (zo >= 0) {
            const int64_t x = bx0 + tx, y = by0 + ty;
            if (x < nx && y < ny) {
                const uint32_t s = ring[0] + ring[1] + ring[2] + ring[3] + ring[4];
                dst[(zo * ny + y) * nx + x] = (uint16_t)(s / 2000u);
            }
        }
        __syncthreads();
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

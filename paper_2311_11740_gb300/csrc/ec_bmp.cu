// ec_bmp.cu -- grayscale BMP input (Sec. 2.3 and Table 5 read the images as
// BMP files): one image as a 2D field, or a stack of slices, one file per z
// plane, streamed as a 3D field through the low-memory path.
//
// Accepted files: uncompressed (BI_RGB) Windows bitmaps with a
// BITMAPINFOHEADER or a later header, 8 bits per pixel with a grayscale
// palette (every entry has R = G = B; the pixel's value is its entry's gray
// level), or 24 / 32 bits per pixel whose pixels all have R = G = B.  Rows are
// stored bottom-up (positive height) or top-down (negative height), each
// padded to a multiple of 4 bytes; the field's row 0 is the image's top row.
#include <cuda_runtime.h>
#include <errno.h>
#include <fcntl.h>
#include <stdint.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ec_internal.h"

using namespace ec;

namespace {

struct BmpInfo {
    int64_t w = 0, h = 0;
    int bits = 0;
    bool top_down = false;
    int64_t data_off = 0;
    int64_t row_bytes = 0;          // stored row length, padding included
    uint8_t gray[256] = {};         // 8-bit files: the gray level of each palette index
};

uint32_t le32(const uint8_t *p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24); }
uint16_t le16(const uint8_t *p) { return (uint16_t)(p[0] | (p[1] << 8)); }

bool read_at(int fd, void *dst, size_t n, int64_t off)
{
    char *p = (char *)dst;
    while (n > 0) {
        const ssize_t r = pread(fd, p, n, (off_t)off);
        if (r < 0 && errno == EINTR) continue;
        if (r <= 0) return false;
        p += r;
        off += r;
        n -= (size_t)r;
    }
    return true;
}

int parse_bmp(int fd, const char *path, BmpInfo &b)
{
    uint8_t hd[54];
    if (!read_at(fd, hd, sizeof hd, 0)) { set_error("%s: too short for a BMP header", path); return EC_ERR_ARG; }
    if (hd[0] != 'B' || hd[1] != 'M') { set_error("%s: not a BMP file", path); return EC_ERR_ARG; }
    const uint32_t data_off = le32(hd + 10), dib = le32(hd + 14);
    if (dib < 40) { set_error("%s: header of %u bytes (BITMAPINFOHEADER or later needed)", path, dib); return EC_ERR_ARG; }
    const int32_t w = (int32_t)le32(hd + 18), h = (int32_t)le32(hd + 22);
    const int bits = le16(hd + 28);
    const uint32_t comp = le32(hd + 30), used = le32(hd + 46);
    if (w <= 0 || h == 0 || h == INT32_MIN) { set_error("%s: bad dimensions %d x %d", path, w, h); return EC_ERR_ARG; }
    if (comp != 0) { set_error("%s: compressed BMP (compression %u) not supported", path, comp); return EC_ERR_DTYPE; }
    if (bits != 8 && bits != 24 && bits != 32) {
        set_error("%s: %d bits per pixel (8, 24 or 32 supported)", path, bits);
        return EC_ERR_DTYPE;
    }
    b.w = w;
    b.h = h < 0 ? -(int64_t)h : h;
    b.top_down = h < 0;
    b.bits = bits;
    b.data_off = data_off;
    b.row_bytes = ((int64_t)bits * b.w + 31) / 32 * 4;
    struct stat st;
    if (fstat(fd, &st) != 0 || (int64_t)st.st_size < b.data_off + b.row_bytes * b.h) {
        set_error("%s: pixel array runs past the end of the file", path);
        return EC_ERR_ARG;
    }
    if (bits == 8) {
        const uint32_t n = used ? std::min<uint32_t>(used, 256u) : 256u;
        uint8_t pal[1024];
        if (!read_at(fd, pal, (size_t)n * 4, 14 + (int64_t)dib)) { set_error("%s: palette missing", path); return EC_ERR_ARG; }
        for (uint32_t i = 0; i < 256; i++) b.gray[i] = 0;
        for (uint32_t i = 0; i < n; i++) {
            const uint8_t B = pal[4 * i], G = pal[4 * i + 1], R = pal[4 * i + 2];
            if (B != G || G != R) { set_error("%s: palette entry %u is not gray", path, i); return EC_ERR_DTYPE; }
            b.gray[i] = R;
        }
    }
    return EC_OK;
}

// Rows of the image into dst (h x w uint8, row 0 = top).
int read_pixels(int fd, const char *path, const BmpInfo &b, uint8_t *dst)
{
    std::vector<uint8_t> row((size_t)b.row_bytes);
    const int bpp = b.bits / 8;
    for (int64_t y = 0; y < b.h; y++) {
        const int64_t stored = b.top_down ? y : b.h - 1 - y;
        if (!read_at(fd, row.data(), row.size(), b.data_off + stored * b.row_bytes)) {
            set_error("%s: reading row %lld failed", path, (long long)y);
            return EC_ERR_ARG;
        }
        uint8_t *d = dst + y * b.w;
        if (bpp == 1) {
            for (int64_t x = 0; x < b.w; x++) d[x] = b.gray[row[(size_t)x]];
        } else {
            for (int64_t x = 0; x < b.w; x++) {
                const uint8_t *p = &row[(size_t)(x * bpp)];
                if (p[0] != p[1] || p[1] != p[2]) {
                    set_error("%s: pixel (%lld, %lld) is not gray", path, (long long)x, (long long)y);
                    return EC_ERR_DTYPE;
                }
                d[x] = p[0];
            }
        }
    }
    return EC_OK;
}

struct Fd {
    int fd;
    explicit Fd(const char *path) : fd(open(path, O_RDONLY)) {}
    ~Fd() { if (fd >= 0) close(fd); }
};

// Slices of a stack read on demand by the streaming path: planes [z0, z1)
// (halo planes outside the stack are left as they are; the kernel ignores
// them) into page-locked staging, then copied on the given stream.
struct BmpStack {
    const char *const *paths = nullptr;
    int64_t n = 0, h = 0, w = 0;
    size_t cap = 0;
    void *pinned[2] = {nullptr, nullptr};
    cudaEvent_t copied[2] = {nullptr, nullptr};
    int next = 0;
    int err = EC_OK;
    std::string msg;
    ~BmpStack()
    {
        for (int i = 0; i < 2; i++) {
            if (copied[i]) { cudaEventSynchronize(copied[i]); cudaEventDestroy(copied[i]); }
            if (pinned[i]) cudaFreeHost(pinned[i]);
        }
    }
};

int stack_producer(void *user, int64_t z0, int64_t z1, void *dst_dev, void *stream)
{
    BmpStack &S = *(BmpStack *)user;
    const int64_t a = std::max<int64_t>(z0, 0), b = std::min<int64_t>(z1, S.n);
    if (b <= a) return 0;
    const size_t plane = (size_t)S.h * (size_t)S.w, bytes = (size_t)(b - a) * plane;
    if (bytes > S.cap) return 1;
    const int i = S.next;
    S.next ^= 1;
    if (cudaEventSynchronize(S.copied[i]) != cudaSuccess) return 2;
    for (int64_t z = a; z < b; z++) {
        Fd f(S.paths[z]);
        if (f.fd < 0) {
            S.err = EC_ERR_ARG;
            S.msg = std::string("cannot open ") + S.paths[z] + ": " + strerror(errno);
            return 3;
        }
        BmpInfo info;
        int rc = parse_bmp(f.fd, S.paths[z], info);
        if (rc == EC_OK && (info.h != S.h || info.w != S.w)) {
            set_error("%s: %lld x %lld, the stack's first slice is %lld x %lld", S.paths[z], (long long)info.h,
                      (long long)info.w, (long long)S.h, (long long)S.w);
            rc = EC_ERR_ARG;
        }
        if (rc == EC_OK) rc = read_pixels(f.fd, S.paths[z], info, (uint8_t *)S.pinned[i] + (size_t)(z - a) * plane);
        if (rc) {
            S.err = rc;
            S.msg = ec_last_error();
            return 4;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync((char *)dst_dev + (size_t)(a - z0) * plane, S.pinned[i], bytes, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return 5;
    if (cudaEventRecord(S.copied[i], s) != cudaSuccess) return 6;
    return 0;
}

}  // namespace

extern "C" int ec_bmp_read(const char *path, int64_t dims_out[2], uint8_t *pixels_host)
{
    clear_error();
    if (!path || !dims_out) { set_error("path or dims_out is NULL"); return EC_ERR_ARG; }
    Fd f(path);
    if (f.fd < 0) { set_error("cannot open %s: %s", path, strerror(errno)); return EC_ERR_ARG; }
    BmpInfo b;
    int rc = parse_bmp(f.fd, path, b);
    if (rc) return rc;
    dims_out[0] = b.h;
    dims_out[1] = b.w;
    if (!pixels_host) return EC_OK;
    return read_pixels(f.fd, path, b, pixels_host);
}

extern "C" int ec_curve_2d_bmp(ec_ctx *ctx, const char *path, const void *thresholds_host, int32_t L,
                               int connectivity, uint32_t descriptors, int64_t *out_host)
{
    clear_error();
    if (!ctx || !path || !out_host) { set_error("ctx, path or out_host is NULL"); return EC_ERR_ARG; }
    int64_t dims[2];
    int rc = ec_bmp_read(path, dims, nullptr);
    if (rc) return rc;
    rc = validate_request(2, path, dims, EC_U8, thresholds_host, L, connectivity, descriptors, out_host);
    if (rc) return rc;
    if (L == 0) return EC_OK;
    std::vector<uint8_t> pix((size_t)(dims[0] * dims[1]));
    rc = ec_bmp_read(path, dims, pix.data());
    if (rc) return rc;
    const size_t nd = (size_t)row_map(descriptors).nd, out_bytes = nd * (size_t)L * sizeof(int64_t);
    DeviceGuard dg(ctx->device);
    void *buf = nullptr;
    const size_t field_bytes = (pix.size() + 255) & ~(size_t)255;
    EC_CUDA(cudaMalloc(&buf, field_bytes + 256 + out_bytes));
    uint8_t *fd = (uint8_t *)buf, *td = fd + field_bytes;
    int64_t *od = (int64_t *)(td + 256);
    cudaStream_t s = nullptr;
    cudaError_t e = cudaMemcpyAsync(fd, pix.data(), pix.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && thresholds_host) e = cudaMemcpyAsync(td, thresholds_host, (size_t)L, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(e, "ec_curve_2d_bmp copy");
    }
    rc = ec_curve_2d(ctx, fd, dims, EC_U8, thresholds_host ? td : nullptr, L, connectivity, descriptors, od, s);
    if (rc == EC_OK) {
        e = cudaMemcpy(out_host, od, out_bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "ec_curve_2d_bmp result");
    } else {
        cudaDeviceSynchronize();
    }
    cudaFree(buf);
    return rc;
}

extern "C" int ec_curve_3d_bmp(ec_ctx *ctx, const char *const *paths, int64_t nslices, const void *thresholds_host,
                               int32_t L, int connectivity, uint32_t descriptors, int64_t slab_planes,
                               size_t device_mem_cap, int64_t *out_host)
{
    clear_error();
    if (!ctx || !paths || nslices < 1) { set_error("ctx or paths is NULL, or no slices"); return EC_ERR_ARG; }
    if (slab_planes < 1) { set_error("slab_planes must be >= 1"); return EC_ERR_ARG; }
    int64_t d2[2];
    int rc = ec_bmp_read(paths[0], d2, nullptr);
    if (rc) return rc;
    const int64_t dims[3] = {nslices, d2[0], d2[1]};
    rc = validate_request(3, paths, dims, EC_U8, thresholds_host, L, connectivity, descriptors, out_host);
    if (rc) return rc;
    if (L == 0) return EC_OK;
    BmpStack S;
    S.paths = paths;
    S.n = nslices;
    S.h = d2[0];
    S.w = d2[1];
    S.cap = (size_t)(std::min<int64_t>(slab_planes, nslices) + 2) * (size_t)(S.h * S.w);
    {
        DeviceGuard dg(ctx->device);
        for (int i = 0; i < 2; i++) {
            if (cudaMallocHost(&S.pinned[i], S.cap) != cudaSuccess) {
                cudaGetLastError();
                S.pinned[i] = nullptr;
                set_error("cannot allocate %zu bytes of page-locked staging", S.cap);
                return EC_ERR_OOM;
            }
            EC_CUDA(cudaEventCreateWithFlags(&S.copied[i], cudaEventDisableTiming));
        }
    }
    rc = ec_curve_3d_stream(ctx, nullptr, stack_producer, &S, dims, EC_U8, thresholds_host, L, connectivity,
                            descriptors, slab_planes, device_mem_cap, out_host);
    if (rc && S.err) {
        set_error("%s", S.msg.c_str());
        return S.err;
    }
    return rc;
}

// lbm_images.cu -- copies of the nodes next to a periodic seam into the
// image rows / columns of the state planes, after the step kernels (see
// lbm_images.h).  Pure data movement: one thread per image position, each
// copying that node's value in every plane of the destination state.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lbm_images.h"
#include "lbm_kernels.h"

namespace lbm {

namespace {

template <int BYTES>
struct Raw;
template <>
struct Raw<2> {
    using T = uint16_t;
};
template <>
struct Raw<4> {
    using T = uint32_t;
};
template <>
struct Raw<8> {
    using T = uint64_t;
};

__device__ __forceinline__ int wrap_axis(int g, int n) {
    const int w = g % n;
    return w < 0 ? w + n : w;
}

// ES: bytes of a stored population; EC: bytes of a carry element; UP:
// planes per u-carry component.
template <int ES, int EC, int UP>
__global__ void __launch_bounds__(kImageThreads) image_kernel(const StepParams* __restrict__ params,
                                                               const ImageTile* __restrict__ tiles) {
    using TS = typename Raw<ES>::T;
    using TC = typename Raw<EC>::T;
    const ImageTile tl = tiles[blockIdx.x];
    const int w = tl.x1 - tl.x0;
    const int k = int(threadIdx.x);
    if (w <= 0 || k >= w * (tl.y1 - tl.y0)) return;
    const StepParams& p = params[tl.inst];
    const int xi = tl.x0 + k % w, yi = tl.y0 + k / w;
    const int xs = wrap_axis(xi, p.nx), ys = wrap_axis(yi, p.ny);
    const int64_t pitch = p.pitch, plane = p.plane;
    const int64_t di = int64_t(yi + kPadRows) * pitch + xi + kPadCols;
    const int64_t si = int64_t(ys + kPadRows) * pitch + xs + kPadCols;
    TS* f = static_cast<TS*>(p.f_dst);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i * plane + di] = f[i * plane + si];
    TC* a = static_cast<TC*>(p.a_dst);
#pragma unroll
    for (int c = 0; c < 2 * UP; ++c) a[c * plane + di] = a[c * plane + si];
    TC* s = static_cast<TC*>(p.s_dst);
    const int ns = p.scheme == 2 ? 4 : 2;  // the extrapolated scheme carries two more planes
    for (int c = 0; c < ns; ++c) s[c * plane + di] = s[c * plane + si];
}

// Tiles of at most kImageThreads positions over the box [x0, x1) x [y0, y1).
int tile_box(int x0, int x1, int y0, int y1, int inst, ImageTile* out, int cap, int n) {
    const int w = x1 - x0, h = y1 - y0;
    if (w <= 0 || h <= 0) return n;
    if (w <= h) {
        const int th = std::max(1, kImageThreads / w);
        for (int y = y0; y < y1; y += th, ++n)
            if (out && n < cap) out[n] = ImageTile{inst, x0, x1, y, std::min(y1, y + th), {0, 0, 0}};
    } else {
        const int tw = std::max(1, kImageThreads / h);
        for (int x = x0; x < x1; x += tw, ++n)
            if (out && n < cap) out[n] = ImageTile{inst, x, std::min(x1, x + tw), y0, y1, {0, 0, 0}};
    }
    return n;
}

}  // namespace

int image_tiles_of_body(int nx, int ny, bool perx, bool pery, const int rect[4], int inst, ImageTile* out,
                        int cap) {
    int n = 0;
    if (perx) {  // the columns across the x seam, over the rows the interior kernel advances
        n = tile_box(-3, 0, rect[2], rect[3], inst, out, cap, n);
        n = tile_box(nx, nx + 3, rect[2], rect[3], inst, out, cap, n);
    }
    if (pery) {  // the rows across the y seam (with the corners when x is periodic too)
        const int xa = perx ? -3 : rect[0], xb = perx ? nx + 3 : rect[1];
        n = tile_box(xa, xb, -3, 0, inst, out, cap, n);
        n = tile_box(xa, xb, ny, ny + 3, inst, out, cap, n);
    }
    return n;
}

cudaError_t launch_images(int fmt, const StepParams* params, const ImageTile* tiles, int ntiles, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    switch (fmt) {
        case kFmtF64: image_kernel<8, 8, 1><<<ntiles, kImageThreads, 0, s>>>(params, tiles); break;
        case kFmtF32: image_kernel<4, 4, 1><<<ntiles, kImageThreads, 0, s>>>(params, tiles); break;
        case kFmtF32C: image_kernel<4, 4, 2><<<ntiles, kImageThreads, 0, s>>>(params, tiles); break;
        case kFmtF16:
        case kFmtBF16: image_kernel<2, 4, 2><<<ntiles, kImageThreads, 0, s>>>(params, tiles); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbm

// lbm_edge.cu -- the fused step on the edge bands of a body, and the
// initialisation of the whole body, as small two-dimensional tiles (the tile
// itself is edge_tile_body of lbm_edge_tile.cuh).
//
// The bands hold few nodes, so what bounds their cost is latency, not
// bandwidth.  Each CTA of 256 threads runs one tile of (tw - 4) x (th - 4)
// output nodes (tw x th <= 256: tiles exactly as thick as a band, 28 x 4 over
// larger areas), one thread per node of the tile and its 2-node halo, and
// hundreds of tiles run at once.
//
// Tiles come from a list (instance, output rectangle, shape), and each
// instance's parameters from a table in device memory, so one launch serves
// one body or a batch of bodies alike.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"
#include "lbm_kernels.h"
#include "lbm_edge_tile.cuh"
#include "lbm_images.cuh"
#include "lbm_init_grid.h"
#include "lbm_pipeline.cuh"

namespace lbm {

static_assert(sizeof(StepParams) % 16 == 0, "StepParams is copied to shared memory in 16-byte words");

template <class TS, class TC, class UT, int MODE, bool HOLE, bool XJ>
__global__ void __launch_bounds__(kEdgeThreads, 3)
    edge_tile_kernel(const __grid_constant__ EdgeLaunch L, const __grid_constant__ ImageLaunch I) {
    constexpr int N = kEdgeThreads;
    static_assert(kImageThreads <= N, "an image tile fits an edge CTA");
    if (I.tiles != nullptr && int(blockIdx.x) >= I.n_edge) {  // a seam-image CTA (uniform per CTA)
        if (int(threadIdx.x) < kImageThreads)
            image_copy<int(sizeof(TS)), int(sizeof(TC)), UT::layout>(L.params, I.tiles[blockIdx.x - I.n_edge],
                                                                    int(threadIdx.x));
        return;
    }
    __shared__ __align__(16) StepParams sp;
    __shared__ EdgeNow<TC, UT> s_edge[5];
    __shared__ UT su[2 * N];                      // u*: [th][2 comps][tw]
    __shared__ TC sq[4 * N];                      // Q:  [th][4 comps][tw]
    __shared__ TC sinit[MODE == 1 ? 4 * N : 1];  // initialisation: r0, Pbar0 / c^2

    EdgeTile tile;
    if (L.tiles != nullptr) {
        tile = L.tiles[blockIdx.x];
    } else {  // implicit grid of square tiles over L.rect (last tiles shifted back)
        const int b = int(blockIdx.x);
        const int bx = b % L.rtiles_x, by = b / L.rtiles_x;
        constexpr int ow = kInitOutW, oh = kInitOutH;
        tile.inst = 0;
        tile.x0 = max(L.rect[0], min(L.rect[0] + bx * ow, L.rect[1] - ow));
        tile.x1 = min(L.rect[1], tile.x0 + ow);
        tile.y0 = max(L.rect[2], min(L.rect[2] + by * oh, L.rect[3] - oh));
        tile.y1 = min(L.rect[3], tile.y0 + oh);
        tile.tw = kInitTileW;
        tile.th = uint8_t(N / kInitTileW);
        tile.hx = 2;
        tile.hy = 2;
        tile.lead = b == 0;
    }
    {
        const int4* src = reinterpret_cast<const int4*>(L.params + tile.inst);
        int4* dst = reinterpret_cast<int4*>(&sp);
        for (int q = int(threadIdx.x); q < int(sizeof(StepParams) / 16); q += N) dst[q] = src[q];
    }
    __syncthreads();
    edge_tile_body<TS, TC, UT, MODE, HOLE, XJ>(tile, sp, L.fields != 0, su, sq, MODE == 1 ? sinit : nullptr,
                                                s_edge);
}

// ---------------------------------------------------------------- launchers

// ntiles edge tiles, then n_img image tiles (I.tiles, mode 0 only)
template <class TS, class TC, class UT>
cudaError_t launch_edge_t(const EdgeLaunch& L, int ntiles, const ImageTile* img, int n_img, cudaStream_t s, int mode,
                          bool holed, bool xj) {
    if (mode != 0 || !img) n_img = 0;
    const ImageLaunch I = {n_img > 0 ? img : nullptr, ntiles, 0};
    const int64_t total = int64_t(ntiles) + n_img;
    if (total <= 0) return cudaSuccess;
    if (total > 0x7fffffff) return cudaErrorInvalidConfiguration;
    const int grid = int(total);
    // the initialisation runs once: one variant, which handles a hole and
    // reads the scheme
    if (mode == 1)
        edge_tile_kernel<TS, TC, UT, 1, true, false><<<grid, kEdgeThreads, 0, s>>>(L, I);
    else if (xj)
        edge_tile_kernel<TS, TC, UT, 0, true, true><<<grid, kEdgeThreads, 0, s>>>(L, I);
    else if (holed)
        edge_tile_kernel<TS, TC, UT, 0, true, false><<<grid, kEdgeThreads, 0, s>>>(L, I);
    else
        edge_tile_kernel<TS, TC, UT, 0, false, false><<<grid, kEdgeThreads, 0, s>>>(L, I);
    return cudaGetLastError();
}

static cudaError_t launch_edge_fmt(int fmt, const EdgeLaunch& L, int ntiles, const ImageTile* img, int n_img,
                                   cudaStream_t s, int mode, bool holed, bool xj) {
    switch (fmt) {
        case kFmtF64: return launch_edge_t<double, double, UPlain<double>>(L, ntiles, img, n_img, s, mode, holed, xj);
        case kFmtF32: return launch_edge_t<float, float, UPlain<float>>(L, ntiles, img, n_img, s, mode, holed, xj);
        case kFmtF32C: return launch_edge_t<float, float, UComp>(L, ntiles, img, n_img, s, mode, holed, xj);
        case kFmtF32H: return launch_edge_t<float, float, UCompH>(L, ntiles, img, n_img, s, mode, holed, xj);
        case kFmtF16: return launch_edge_t<__half, float, UComp>(L, ntiles, img, n_img, s, mode, holed, xj);
        case kFmtBF16: return launch_edge_t<__nv_bfloat16, float, UComp>(L, ntiles, img, n_img, s, mode, holed, xj);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_edge(int fmt, const EdgeLaunch& L, int ntiles, cudaStream_t s, int mode, bool holed, bool xj) {
    return launch_edge_fmt(fmt, L, ntiles, nullptr, 0, s, mode, holed, xj);
}

cudaError_t launch_edge_images(int fmt, const EdgeLaunch& L, int n_edge, const ImageTile* img, int n_img,
                               cudaStream_t s, bool holed, bool xj) {
    return launch_edge_fmt(fmt, L, n_edge, img, n_img, s, 0, holed, xj);
}

// Tiles of one rectangle for CTAs of nthreads threads.  A band at most 3
// nodes thick gets tiles exactly as thick (th = thickness + 4 rows of
// threads, 2 fewer for each side on a bounded edge of the body, where the
// halo would lie outside it; tw = nthreads / th columns), so few threads
// compute halo only; a larger rectangle gets wide tiles (32 x 8 threads for
// 256, 16 x 8 for 128).  Every tile has the full extent min(rectangle, tile)
// along both axes (the last one of a row or column is shifted back,
// recomputing its neighbour's nodes bit for bit), so each output node on a
// bounded edge (bodies and bands are at least 2 nodes thick) finds the Q of
// its two inward neighbours, which stage B computes for the output nodes and
// their 1-node ring, inside the tile.  Returns the number of tiles (written
// to out, at most cap, when out is not NULL).
int edge_tiles_of_rect(const int rect[4], int inst, EdgeTile* out, int cap, bool lead_first, int nthreads,
                       unsigned bounded) {
    const int w = rect[1] - rect[0], h = rect[3] - rect[2];
    if (w <= 0 || h <= 0 || nthreads < 128) return 0;
    int tw, th, hx = 2, hy = 2, ow, oh;
    if (h <= 3) {
        hy = (bounded & 4) ? 0 : 2;
        th = h + hy + ((bounded & 8) ? 0 : 2);
        tw = nthreads / th < 255 ? nthreads / th : 255;
        ow = tw - 4;
        oh = h;
    } else if (w <= 3) {
        hx = (bounded & 1) ? 0 : 2;
        tw = w + hx + ((bounded & 2) ? 0 : 2);
        th = nthreads / tw < 255 ? nthreads / tw : 255;
        ow = w;
        oh = th - 4;
    } else {
        th = 8;
        tw = nthreads / th >= 32 ? 32 : nthreads / th;
        ow = tw - 4;
        oh = th - 4;
    }
    int n = 0;
    for (int y = rect[2]; y < rect[3]; y += oh)
        for (int x = rect[0]; x < rect[1]; x += ow) {
            if (out && n < cap) {
                const int xs = x + ow <= rect[1] ? x : (rect[1] - ow > rect[0] ? rect[1] - ow : rect[0]);
                const int ys = y + oh <= rect[3] ? y : (rect[3] - oh > rect[2] ? rect[3] - oh : rect[2]);
                EdgeTile& e = out[n];
                e.inst = inst;
                e.x0 = xs;
                e.x1 = xs + ow < rect[1] ? xs + ow : rect[1];
                e.y0 = ys;
                e.y1 = ys + oh < rect[3] ? ys + oh : rect[3];
                e.tw = uint8_t(tw);
                e.th = uint8_t(th);
                e.hx = uint8_t(hx);
                e.hy = uint8_t(hy);
                e.lead = int16_t(lead_first && n == 0);
            }
            ++n;
        }
    return n;
}

}  // namespace lbm

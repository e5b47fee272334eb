// lbm_images.cu -- the tile lists of the seam images (lbm_images.h); the
// copies themselves run as CTAs of the edge launch after the interior
// launch (lbm_images.cuh, launch_edge_images in lbm_edge.cu).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lbm_images.h"

namespace lbm {

namespace {

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

}  // namespace lbm

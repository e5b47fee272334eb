// lbm_init_grid.h -- the initialisation's implicit grid of edge-kernel tiles
// over the whole body (lbm_edge.cu launches it, lbm_api.cu sizes it).
#pragma once

#include "lbm_kernels.h"

namespace lbm {

// Tiles of kInitTileW x (kEdgeThreads / kInitTileW) threads: 12 x 12 output
// nodes per CTA (144 of 256 threads, against 112 for 32 x 8).
constexpr int kInitTileW = 16;
constexpr int kInitOutW = kInitTileW - 4, kInitOutH = kEdgeThreads / kInitTileW - 4;

}  // namespace lbm

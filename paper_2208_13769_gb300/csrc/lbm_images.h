// lbm_images.h -- periodic images of the nodes next to a seam, for bodies
// whose interior kernel runs across a periodic axis.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_params.h"

namespace lbm {

// Along a periodic axis the 3 outer rows / columns of every state plane hold
// copies of the nodes across the seam (lbm_params.h).  The edge kernel
// writes the copies of the nodes it advances; where the interior kernel
// advances the nodes next to a seam, CTAs of the edge launch that follows
// the interior launch copy them.  A tile is a box of image positions [x0, x1) x [y0, y1) of one
// instance (entry of the parameter table), at most kImageThreads positions,
// each copied from the node (x mod nx, y mod ny) in every plane of the
// instance's destination state (populations, u-carry, source carry).
constexpr int kImageThreads = 256;

struct ImageTile {
    int32_t inst;
    int32_t x0, x1, y0, y1;
    int32_t pad[3];
};

// The image tiles of one instance whose interior kernel covers the
// rectangle rect (x_lo, x_hi, y_lo, y_hi): the images of its nodes within 3
// nodes of a periodic seam.  Count only when out is NULL.
int image_tiles_of_body(int nx, int ny, bool perx, bool pery, const int rect[4], int inst, ImageTile* out,
                        int cap);

// Image tiles appended to an edge launch: CTAs n_edge and on copy
// tiles[blockIdx.x - n_edge] (tiles NULL: none).
struct ImageLaunch {
    const ImageTile* tiles;
    int32_t n_edge;
    int32_t pad;
};

struct EdgeLaunch;
// A step's edge tiles (n_edge of them, as launch_edge with mode 0) and its
// seam images (n_img tiles, a device list indexing the same parameter table
// as the edge tiles, whose f_dst / a_dst / s_dst are the state being
// written) in one launch, for a step whose interior kernel ran across a
// periodic seam: it follows the interior launch on the same stream (the
// images copy what the interior launch wrote), and the small CTAs of both
// kinds share the SMs.
cudaError_t launch_edge_images(int fmt, const EdgeLaunch& L, int n_edge, const ImageTile* img, int n_img,
                               cudaStream_t s, bool holed, bool xj);

}  // namespace lbm

// lbm_kernels.h -- host-visible launchers of the solver's kernels.
#pragma once

#include <cuda_runtime.h>

#include "lbm_params.h"

namespace lbm {

// Number formats of a context: population storage / arithmetic / u-carry.
enum Format : int {
    kFmtF64 = 0,   // FP64 / FP64 / FP64
    kFmtF32 = 1,   // FP32 / FP32 / FP32
    kFmtF32C = 2,  // FP32 / FP32 / compensated FP32 pair
    kFmtF16 = 3,   // FP16 / FP32 / compensated FP32 pair
    kFmtBF16 = 4,  // BF16 / FP32 / compensated FP32 pair
    kFmtF32H = 5   // FP32 / FP32 / FP32 + 16-bit low word (UCompH)
};


// The interior kernel (lbm_interior.cu): nodes of p.rect[0] only, which must
// lie at least 2 nodes from bounded edges and 3 from periodic seams.  A CTA
// has kInteriorThreads threads, one per column of its strip and halo.
constexpr int kInteriorThreads = 128;
size_t interior_smem(int fmt, int ring_slots);
// CTAs of the interior kernel resident per SM with this ring (0 on error);
// also sets the kernel's dynamic shared-memory limit, so call it before any
// stream capture.
int interior_occupancy(int fmt, int ring_slots);
// Rows of the interior kernel's bulk-copy ring by default, all of them in
// flight (4 measured fastest for single bodies and for batches).
constexpr int kInteriorRing = 4;
constexpr int kBatchRing = 4;
// The strip grid of the interior kernel over columns [rx0, rx1): origin of
// strip 0, output columns per strip, number of strips.  aligned 1: the
// fewest strips of equal width (at most 120 columns, 112 for 16-bit storage)
// on 32-byte sector boundaries (for CTAs of one body that may run in
// different waves); 2: the same on 16-byte boundaries (at most 124 columns,
// 120 for 16-bit storage); otherwise 124-column strips from rx0 (one wave).
void interior_strips(int fmt, int rx0, int rx1, int aligned, int* strip_x0, int* strip_w, int* nstrips);

// One interior rectangle of a launch: its nodes [rect[0], rect[1]) x
// [rect[2], rect[3]), the strip grid over its columns and the rows per tile.
struct TileGeom {
    int32_t rect[4];
    int32_t strip_x0, strip_w, chunk_rows;
};
// The rectangles of one interior launch (a hole splits the interior into up
// to 4): tiles_x x tiles_y tiles each, numbered from first[q] in one 1-D grid
// of total tiles.
struct InteriorRects {
    TileGeom g[4];
    int32_t tiles_x[4];
    int32_t first[4];  // unused entries: INT32_MAX
    int32_t total;
};
// One step of the interior: a launch of R.total CTAs over the rectangles.
cudaError_t launch_interior(int fmt, const StepParams& p, const InteriorRects& R, cudaStream_t s, bool fields);

// The interiors of a batch of bodies for one time step: one CTA of
// kInteriorThreads threads per item, the interior tile (strip a, chunk b) of
// the parameter-table entry inst (a member's rectangle, with its strip grid
// and rows per chunk).
struct BatchItem {
    int32_t inst, a, b;
    int32_t pad;
};
struct BatchInteriorLaunch {
    const StepParams* params;  // device table, indexed by BatchItem::inst
    const BatchItem* items;    // device list of interior tiles, one per CTA
    int32_t fields;            // also write u, v, r to params.fields
    int32_t nitems;            // tiles in the list
};
// The setting of the dynamic shared-memory limit happens on the first call
// (also with nitems == 0), which must precede any stream capture; resident
// (may be NULL) receives the kernel's CTAs per SM with this ring.
cudaError_t launch_batch_interior(int fmt, const BatchInteriorLaunch& L, int ring_slots, cudaStream_t s,
                                  int* resident);

// The edge kernel (lbm_edge.cu): small 2-D tiles with every boundary rule.
// A tile's threads cover its output nodes and a 2-node halo, except beyond a
// side that lies on a bounded edge of the body, where there are no nodes:
// tw x th nodes (tw x th <= kEdgeThreads), from (x0 - hx, y0 - hy).
constexpr int kEdgeThreads = 256;

struct EdgeTile {
    int32_t inst;    // entry of the parameter table
    int32_t x0, y0;  // first output node
    int32_t x1, y1;  // one past the last output node
    uint8_t tw, th;  // threads along x and y
    uint8_t hx, hy;  // halo nodes before the first output node (2, or 0 on a bounded edge)
    int16_t lead;    // this tile advances the instance's step counter
};

struct EdgeLaunch {
    const StepParams* params;  // device table, indexed by EdgeTile::inst
    const EdgeTile* tiles;     // device tile list; NULL: wide tiles over rect
    int32_t fields;            // also write u, v, r to params.fields
    int32_t rtiles_x;          // implicit grid: tiles per row of rect
    int32_t rect[4];           // implicit grid: x_lo, x_hi, y_lo, y_hi
};

// One step (mode 0) or the initialisation (mode 1) over ntiles tiles.
// holed: the body has a hole; xj: the extrapolated scheme (mode 0; the
// initialisation reads the scheme from the parameters).
cudaError_t launch_edge(int fmt, const EdgeLaunch& L, int ntiles, cudaStream_t s, int mode, bool holed, bool xj);

// Tiles of one band rectangle for CTAs of `nthreads` threads (kEdgeThreads
// for the edge kernel); count only when out is NULL.  bounded: the sides of
// rect that lie on a bounded edge of the body (bit 0: x low, 1: x high,
// 2: y low, 3: y high), beyond which a band's tiles need no halo.
int edge_tiles_of_rect(const int rect[4], int inst, EdgeTile* out, int cap, bool lead_first, int nthreads,
                       unsigned bounded);

// Read-out parameters: stresses from the FP64 displacement field.
struct ReadoutParams {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y;
    double dX, lambda, mu, rho0, t;
    const double* fields;  // 5 planes [ny][nx]: u_x, u_y, v_x, v_y, r
    EdgeBC bc[4];
    int32_t hole[4];  // removed nodes of a hole (x0 >= x1: none)
};

// Writes the fields selected by mask (LBM_FIELD_* bits) into out, each block
// [ny][nx][ncomp] in bit order.
cudaError_t launch_readout(const ReadoutParams& rp, unsigned mask, double* out, cudaStream_t s);

// Diagnostics: per-CTA partial sums into `partials` (nblocks x 8 doubles),
// then a single-CTA fixed-order pass into out8 (device, 8 doubles):
// sum j_x, sum j_y, kinetic energy, strain energy, min J, non-finite flag.
int diagnostics_blocks(int64_t nodes);
cudaError_t launch_diagnostics(const ReadoutParams& rp, double* partials, int nblocks, double* out8,
                               cudaStream_t s);

}  // namespace lbm

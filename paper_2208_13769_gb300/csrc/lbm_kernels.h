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
    kFmtBF16 = 4   // BF16 / FP32 / compensated FP32 pair
};

// Output columns per strip: general kernel at initialisation, general
// kernel on the edge bands, interior kernel.
void strip_widths(int* init_w, int* band_w, int* interior_w);


// The interior kernel (lbm_interior.cu): nodes of p.rect[0] only, which must
// lie at least 2 nodes from bounded edges and 3 from periodic seams.
size_t interior_smem(int fmt, int ring_slots);
cudaError_t launch_interior(int fmt, const StepParams& p, cudaStream_t s, bool fields);

// One fused step (mode 0) or the initialisation (mode 1); fields: also write
// u, v, r to p.fields.
cudaError_t launch_fused_step(int fmt, const StepParams& p, cudaStream_t s, int mode, bool fields);

// Read-out parameters: stresses from the FP64 displacement field.
struct ReadoutParams {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y;
    double dX, lambda, mu, rho0, t;
    const double* fields;  // 5 planes [ny][nx]: u_x, u_y, v_x, v_y, r
    EdgeBC bc[4];
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

// lbm_context.h -- the solver context behind the C ABI's lbm_ctx handle, and
// the context helpers that the single-body and the batched entry points share
// (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "lbm.h"
#include "lbm_images.h"
#include "lbm_kernels.h"

namespace lbm {

// An NVTX range named after the entry point, for the scope: profilers
// (nsys, ncu --nvtx-include) attribute the launches to the call; without a
// profiler attached it costs a check of a function pointer.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Makes `dev` current for the scope, restoring the previous device after.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace lbm

struct lbm_ctx {
    int device = 0;
    int num_sms = 1;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    // the edge-band launch of a step runs on a side stream, concurrently with
    // the interior launch on the main stream (fork / join by events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaError_t last_error = cudaSuccess;
    int fmt = lbm::kFmtF32;
    int scheme = 1;
    int32_t nx = 0, ny = 0;
    double dX = 1.0;
    int32_t f16_scale_log2 = 10;
    int32_t lo_log2 = 0;  // the u-carry's 16-bit low words hold lo 2^lo_log2 (kFmtF32H)
    // layout
    int64_t pitch = 0, plane = 0;
    // device memory
    void* f[2] = {nullptr, nullptr};
    void* a[2] = {nullptr, nullptr};
    void* s[2] = {nullptr, nullptr};
    double* fields = nullptr;
    double* u0 = nullptr;
    double* v0 = nullptr;
    int32_t* flag = nullptr;
    int64_t* counter = nullptr;
    double* partials = nullptr;
    double* diag = nullptr;
    double* readout = nullptr;
    size_t readout_cap = 0;
    int diag_blocks = 1;
    int64_t device_bytes = 0;
    // problem
    bool material_set = false;
    bool bc_set[4] = {false, false, false, false};
    lbm::EdgeBC bc[4];
    double lambda = 0, mu = 0, rho0 = 0, omega = 1, body[2] = {0, 0};
    double dt = 0, c = 0, cs2 = 0;
    // progress
    bool initialized = false;
    int parity = 0;
    int64_t steps = 0;
    bool sticky = false;
    bool variant_warm = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // a rectangular hole: removed nodes x0 <= x < x1, y0 <= y < y1 (none
    // while x0 >= x1), and the traction on its faces at x0, x1, y0, y1
    int32_t hole[4] = {0, 0, 0, 0};
    double hole_T[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // launch plan (built at initialisation, once the boundaries are known):
    // the interior as up to 4 rectangles (a hole splits it), each with its
    // strip grid and row chunks; the bands around the body and the hole
    bool planned = false;
    bool has_interior = false;  // n_irect > 0
    int n_irect = 0;
    int irect[4][4];
    int i_tiles_x[4], i_tiles_y[4], i_chunk[4], i_strip_x0[4], i_strip_w[4];
    int i_ring = 0;
    // requested decomposition of the interior launch (lbm_set_tuning); 0 / -1:
    // the library's defaults
    int tune_ring = 0, tune_chunk = 0, tune_aligned = -1, tune_plan = 0;
    int nband = 0;
    int brect[12][4];
    lbm::StepParams* dparams = nullptr;  // device: make_params(parity 0), make_params(parity 1)
    lbm::EdgeTile* dtiles = nullptr;     // device: tiles of the edge bands
    int n_etiles = 0;
    // with a hole, the initialisation runs over the bands' tiles and tiles of
    // the interior rectangles (then after the band tiles in dtiles), so that
    // every face of the hole sees a tile as thick as its band
    int n_itiles = 0;
    // images of the nodes next to a periodic seam that the interior kernel
    // advances, copied after each step (lbm_images.h)
    lbm::ImageTile* dimg = nullptr;
    int n_img = 0;
};

namespace lbm {

// Host-side fault injection for tests of failure handling (nothing faults on
// the GPU): true when the environment variable LBM_FAULT names `call`
// ("alloc": lbm_create fails as if device memory were exhausted, before any
// CUDA call; "step": lbm_step fails as if a launch had failed, leaving the
// context unusable; "batch_step": the same for lbm_batch_step).
bool fault_injected(const char* call);
// Marks the context unusable after a CUDA error; returns LBM_E_CUDA.
lbm_status ctx_fail_cuda(lbm_ctx* c, cudaError_t e);
// Parameters of one step from parity `parity` (source buffers of that parity).
StepParams make_params(const lbm_ctx* c, int parity);
// LBM_OK once material and all four boundaries are set and no CUDA error
// occurred; LBM_E_STATE / LBM_E_CUDA / LBM_E_INVALID otherwise.
lbm_status ctx_ready(const lbm_ctx* c);
// Nodes the interior launches advance (all interior rectangles).
int64_t interior_nodes(const lbm_ctx* c);
// The rectangles of a step: the interior kernel's (n_irect, up to 4: a hole
// splits the interior; none for a body too small for it) and the edge
// tiles' (nband, up to 12).  edge_only: everything as edge tiles.
// seams_inside: the interior kernel also runs across periodic seams (their
// images then come from an image launch after each step), else a 3-node
// band on each side of a seam goes to the edge kernel.
void plan_rects(const lbm_ctx* c, bool edge_only, bool seams_inside, int irect[4][4], int* n_irect,
                int brect[12][4], int* nband);
// The sides of rect on a bounded edge of the body (bit 0: x low, 1: x high,
// 2: y low, 3: y high), for edge_tiles_of_rect.
unsigned bounded_sides(const lbm_ctx* c, const int rect[4]);
// The box of image sources of a body whose interior kernel runs across its
// periodic seams: the whole axis where periodic, nodes 2 .. n - 3 where bounded.
void seam_box(const lbm_ctx* c, int box[4]);
// Plans the launches and runs the initialisation of Algorithm 1 once.
lbm_status ctx_ensure_initialized(lbm_ctx* c);
// Synchronises the context's stream and maps its device flag to a status.
lbm_status ctx_check_flag(lbm_ctx* c);

}  // namespace lbm

// lbm_api.cu -- the C ABI of include/lbm.h: contexts, device memory, launch
// sequencing, CUDA-graph replay of step chunks, read-out and diagnostics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "lbm.h"
#include "lbm_context.h"
#include "lbm_init_grid.h"
#include "lbm_kernels.h"

using namespace lbm;

namespace {

constexpr int kGraphChunk = 64;  // steps per captured graph (even: keeps the ping-pong parity)
constexpr int kSegMax = 144;  // widest row segment the interior kernel copies in bulk (elements)

size_t elem_size_storage(int fmt) {
    switch (fmt) {
        case kFmtF64: return 8;
        case kFmtF32:
        case kFmtF32C:
        case kFmtF32H: return 4;
        default: return 2;
    }
}
size_t elem_size_compute(int fmt) { return fmt == kFmtF64 ? 8 : 4; }
// planes of the source carry: the last source, or D and G of the
// extrapolated scheme
int source_planes(int scheme) { return scheme == LBM_SCHEME_EXTRAPOLATED ? 4 : 2; }
// bytes of the u-carry per node, both components (the layouts of
// UPlain / UPair in lbm_device.cuh)
size_t ucarry_bytes(int fmt) {
    switch (fmt) {
        case kFmtF32: return 8;
        case kFmtF32H: return 12;
        default: return 16;  // FP64, or a pair of FP32 words
    }
}

}  // namespace

bool lbm::fault_injected(const char* call) {
    const char* v = getenv("LBM_FAULT");
    return v != nullptr && strcmp(v, call) == 0;
}

lbm_status lbm::ctx_fail_cuda(lbm_ctx* ctx, cudaError_t e) {
    if (ctx) {
        ctx->sticky = true;
        ctx->last_error = e;
    }
    return LBM_E_CUDA;
}

#define LBM_CUDA(ctx, call)                          \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return ctx_fail_cuda((ctx), e_); \
    } while (0)

StepParams lbm::make_params(const lbm_ctx* c, int parity) {
    StepParams p;
    memset(&p, 0, sizeof(p));
    p.nx = c->nx;
    p.ny = c->ny;
    p.periodic_x = c->bc[0].kind == kPeriodic;
    p.periodic_y = c->bc[2].kind == kPeriodic;
    p.scheme = c->scheme;
    p.pitch = c->pitch;
    p.plane = c->plane;
    p.f_src = c->f[parity];
    p.f_dst = c->f[parity ^ 1];
    p.a_src = c->a[parity];
    p.a_dst = c->a[parity ^ 1];
    p.s_src = c->s[parity];
    p.s_dst = c->s[parity ^ 1];
    p.fields = c->fields;
    p.u0 = c->u0;
    p.v0 = c->v0;
    p.flag = c->flag;
    p.counter = c->counter;
    p.parity = parity;
    p.dX = c->dX;
    p.dt = c->dt;
    p.c = c->c;
    p.cs2 = c->cs2;
    p.omega = c->omega;
    p.rho0 = c->rho0;
    p.lambda = c->lambda;
    p.mu = c->mu;
    p.body[0] = c->body[0];
    p.body[1] = c->body[1];
    for (int i = 0; i < 9; ++i) {
        const double w = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        const double dec = w * ldexp(1.0, -c->f16_scale_log2);
        p.dec_scale[i] = float(dec);
        p.enc_scale[i] = float(1.0 / dec);
    }
    p.lo_scale[0] = float(ldexp(1.0, c->lo_log2));
    p.lo_scale[1] = float(ldexp(1.0, -c->lo_log2));
    for (int e = 0; e < 4; ++e) p.bc[e] = c->bc[e];
    // lattice constants in FP64, and rounded to FP32
    double* L = p.lat_d;
    L[kLatOmega] = p.omega;
    L[kLatOneMOmega] = 1.0 - p.omega;
    L[kLatForcePref] = 1.0 - 0.5 * p.omega;
    L[kLatKu] = p.dX / (2.0 * p.rho0);
    L[kLatInv2dX] = 1.0 / (2.0 * p.dX);
    L[kLatSqScale] = p.dt * p.dt / (2.0 * p.dX * p.dX);
    L[kLatSb0] = p.dt * p.dt / p.dX * p.rho0 * p.body[0];
    L[kLatSb1] = p.dt * p.dt / p.dX * p.rho0 * p.body[1];
    L[kLatLambda] = p.lambda;
    L[kLatMu] = p.mu;
    L[kLatInvC2] = 1.0 / (p.c * p.c);
    L[kLatCOverRho0] = p.c / p.rho0;
    L[kLatRho0OverC] = p.rho0 / p.c;
    L[kLatRho0] = p.rho0;
    for (int k = 0; k < kLatCount; ++k) p.lat_f[k] = float(L[k]);
    for (int k = 0; k < 4; ++k) p.hole[k] = c->hole[k];
    for (int k = 0; k < 8; ++k) p.hole_T[k] = c->hole_T[k];
    return p;
}

static ReadoutParams make_readout(const lbm_ctx* c) {
    ReadoutParams r;
    memset(&r, 0, sizeof(r));
    r.nx = c->nx;
    r.ny = c->ny;
    r.periodic_x = c->bc[0].kind == kPeriodic;
    r.periodic_y = c->bc[2].kind == kPeriodic;
    r.dX = c->dX;
    r.lambda = c->lambda;
    r.mu = c->mu;
    r.rho0 = c->rho0;
    r.t = double(c->steps) * c->dt;
    r.fields = c->fields;
    for (int e = 0; e < 4; ++e) r.bc[e] = c->bc[e];
    for (int k = 0; k < 4; ++k) r.hole[k] = c->hole[k];
    return r;
}

lbm_status lbm::ctx_ready(const lbm_ctx* c) {
    if (!c) return LBM_E_INVALID;
    if (c->sticky) return LBM_E_CUDA;
    if (!c->material_set) return LBM_E_STATE;
    for (int e = 0; e < 4; ++e)
        if (!c->bc_set[e]) return LBM_E_STATE;
    return LBM_OK;
}

int64_t lbm::interior_nodes(const lbm_ctx* c) {
    int64_t n = 0;
    for (int k = 0; k < c->n_irect; ++k)
        n += int64_t(c->irect[k][1] - c->irect[k][0]) * (c->irect[k][3] - c->irect[k][2]);
    return n;
}

void lbm::seam_box(const lbm_ctx* c, int box[4]) {
    const bool perx = c->bc[0].kind == kPeriodic, pery = c->bc[2].kind == kPeriodic;
    box[0] = perx ? 0 : 2;
    box[1] = perx ? c->nx : c->nx - 2;
    box[2] = pery ? 0 : 2;
    box[3] = pery ? c->ny : c->ny - 2;
}

unsigned lbm::bounded_sides(const lbm_ctx* c, const int rect[4]) {
    const bool perx = c->bc[0].kind == kPeriodic, pery = c->bc[2].kind == kPeriodic;
    return (!perx && rect[0] == 0 ? 1u : 0u) | (!perx && rect[1] == c->nx ? 2u : 0u) |
           (!pery && rect[2] == 0 ? 4u : 0u) | (!pery && rect[3] == c->ny ? 8u : 0u);
}

void lbm::plan_rects(const lbm_ctx* c, bool edge_only, bool seams_inside, int irect[4][4], int* n_irect,
                     int brect[12][4], int* nband) {
    const bool perx = c->bc[0].kind == kPeriodic, pery = c->bc[2].kind == kPeriodic;
    // a bounded edge keeps a 2-node band for the edge kernel's boundary
    // rules; a periodic seam a 3-node band on each side (the interior
    // kernel writes no images), unless the interior kernel runs across the
    // seam, reading the images of the nodes beyond it, which the image
    // launch refreshes after every step
    const int bx = perx ? (seams_inside ? 0 : 3) : 2, by = pery ? (seams_inside ? 0 : 3) : 2;
    const int nx = c->nx, ny = c->ny;
    const int32_t* H = c->hole;
    const bool hole = H[0] < H[1];
    // too small for the interior kernel
    const bool small = edge_only || !(nx - 2 * bx >= 8 && ny - 2 * by >= 8);
    *nband = 0;
    *n_irect = 0;
    const int bands[4][4] = {{0, nx, 0, by}, {0, nx, ny - by, ny}, {0, bx, by, ny - by}, {nx - bx, nx, by, ny - by}};
    if (!hole) {
        if (small) {
            const int all[4] = {0, nx, 0, ny};
            for (int k = 0; k < 4; ++k) brect[0][k] = all[k];
            *nband = 1;
        } else {
            const int R[4] = {bx, nx - bx, by, ny - by};
            for (int k = 0; k < 4; ++k) irect[0][k] = R[k];
            *n_irect = 1;
            for (int b = 0; b < 4; ++b)
                for (int k = 0; k < 4; ++k) brect[b][k] = bands[b][k];
            *nband = 4;
        }
    } else {
        // the bands of the edges and the 2-node band around the hole (the
        // hole keeps clear of the edges' bands, lbm_set_hole); the rest of
        // the body below, above, left and right of the hole's band goes to
        // the interior kernel, or, for a body too small for it, to tiles of
        // the edge kernel as well
        for (int b = 0; b < 4; ++b)
            for (int k = 0; k < 4; ++k) brect[b][k] = bands[b][k];
        const int hb[4][4] = {{H[0] - 2, H[0], H[2] - 2, H[3] + 2},
                              {H[1], H[1] + 2, H[2] - 2, H[3] + 2},
                              {H[0], H[1], H[2] - 2, H[2]},
                              {H[0], H[1], H[3], H[3] + 2}};
        for (int b = 0; b < 4; ++b)
            for (int k = 0; k < 4; ++k) brect[4 + b][k] = hb[b][k];
        *nband = 8;
        const int R[4] = {bx, nx - bx, by, ny - by};
        const int B[4] = {H[0] - 2, H[1] + 2, H[2] - 2, H[3] + 2};
        const int parts[4][4] = {{R[0], R[1], R[2], B[2]},
                                 {R[0], R[1], B[3], R[3]},
                                 {R[0], B[0], std::max(R[2], B[2]), std::min(R[3], B[3])},
                                 {B[1], R[1], std::max(R[2], B[2]), std::min(R[3], B[3])}};
        for (int q = 0; q < 4; ++q) {
            if (!(parts[q][0] < parts[q][1] && parts[q][2] < parts[q][3])) continue;
            int* dst = small ? brect[(*nband)++] : irect[(*n_irect)++];
            for (int k = 0; k < 4; ++k) dst[k] = parts[q][k];
        }
    }
}

// The interior (nodes >= 2 from bounded edges and from a hole's faces, >= 3
// from periodic seams, or across them) as up to 4 rectangles for the lean
// kernel; the bands around the body and around the hole as tiles of the
// edge kernel; the seam images; the parameter table of both parities and the
// tile lists go to the device.
static cudaError_t build_plan(lbm_ctx* c) {
    // edge tiles only for a body that the interior kernel's per-launch
    // latency floor would slow down (plan 0), or on request (plan 1)
    const int64_t nodes = int64_t(c->nx) * c->ny;
    const int64_t edge_only_below = c->fmt == kFmtF64 ? (int64_t(3) << 17) : (int64_t(1) << 17);
    const bool edge_only = c->tune_plan == 1 || (c->tune_plan == 0 && nodes < edge_only_below);
    // periodic seams inside the interior kernel under plan 2 (as in a
    // batch, whose one image launch serves every member); by size (plan 0)
    // the seams keep their bands, whose edge launch runs beside the
    // interior's instead of after it
    const bool seams_inside = c->tune_plan == 2;
    plan_rects(c, edge_only, seams_inside, c->irect, &c->n_irect, c->brect, &c->nband);
    const bool hole = c->hole[0] < c->hole[1];
    if (c->n_irect > 0) {
        c->i_ring = c->tune_ring ? c->tune_ring : kInteriorRing;
        const int per_sm = std::max(1, interior_occupancy(c->fmt, c->i_ring));
        const int64_t slots = int64_t(c->num_sms) * per_sm;
        const int64_t all_area = interior_nodes(c);
        for (int q = 0; q < c->n_irect; ++q) {
            const int* r = c->irect[q];
            const int h = r[3] - r[2];
            interior_strips(c->fmt, r[0], r[1], c->tune_aligned > 0 ? c->tune_aligned : 0, &c->i_strip_x0[q], &c->i_strip_w[q],
                            &c->i_tiles_x[q]);
            int64_t rows;
            if (c->tune_chunk > 0) {
                rows = c->tune_chunk;
            } else {
                // one wave of CTAs per launch (strips x chunks <= SMs x
                // per_sm), the rectangles of a hole sharing it by area, at
                // least 8 rows each (shorter tiles of mid-size bodies cut the
                // row pipeline's latency: 512 x 512 FP32 in 17 us with 8-row
                // tiles against 25 us with 16)
                const int64_t area = int64_t(r[1] - r[0]) * h;
                const int64_t share = std::max<int64_t>(1, slots * area / std::max<int64_t>(1, all_area));
                const int64_t chunks = std::max<int64_t>(1, share / c->i_tiles_x[q]);
                rows = std::max<int64_t>((h + chunks - 1) / chunks, 8);
            }
            rows = std::min<int64_t>(rows, h);
            c->i_chunk[q] = int(rows);
            c->i_tiles_y[q] = int((h + rows - 1) / rows);
        }
    }
    c->has_interior = c->n_irect > 0;  // a hole may leave the bands only
    int n = 0;
    for (int b = 0; b < c->nband; ++b)
        n += edge_tiles_of_rect(c->brect[b], 0, nullptr, 0, false, kEdgeThreads, bounded_sides(c, c->brect[b]));
    int ni = n;  // the initialisation's tiles: with a hole, the interior rectangles' too
    if (hole)
        for (int q = 0; q < c->n_irect; ++q)
            ni += edge_tiles_of_rect(c->irect[q], 0, nullptr, 0, false, kEdgeThreads, 0);
    EdgeTile* h = new (std::nothrow) EdgeTile[size_t(ni)];
    if (!h) return cudaErrorMemoryAllocation;
    int m = 0;
    for (int b = 0; b < c->nband; ++b)
        m += edge_tiles_of_rect(c->brect[b], 0, h + m, n - m, m == 0, kEdgeThreads, bounded_sides(c, c->brect[b]));
    if (hole)
        for (int q = 0; q < c->n_irect; ++q)
            m += edge_tiles_of_rect(c->irect[q], 0, h + m, ni - m, false, kEdgeThreads, 0);
    // the images of the interior's nodes next to a periodic seam
    const bool perx = c->bc[0].kind == kPeriodic, pery = c->bc[2].kind == kPeriodic;
    int nimg = 0;
    ImageTile* himg = nullptr;
    if (c->has_interior && seams_inside && (perx || pery)) {
        int box[4];
        seam_box(c, box);
        nimg = image_tiles_of_body(c->nx, c->ny, perx, pery, box, 0, nullptr, 0);
        himg = new (std::nothrow) ImageTile[size_t(nimg)];
        if (!himg) {
            delete[] h;
            return cudaErrorMemoryAllocation;
        }
        image_tiles_of_body(c->nx, c->ny, perx, pery, box, 0, himg, nimg);
    }
    StepParams hp[2] = {make_params(c, 0), make_params(c, 1)};
    cudaError_t e = cudaMalloc(&c->dtiles, sizeof(EdgeTile) * size_t(ni));
    if (e == cudaSuccess) e = cudaMalloc(&c->dparams, sizeof(hp));
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->dtiles, h, sizeof(EdgeTile) * size_t(ni), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->dparams, hp, sizeof(hp), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && nimg > 0) e = cudaMalloc(&c->dimg, sizeof(ImageTile) * size_t(nimg));
    if (e == cudaSuccess && nimg > 0)
        e = cudaMemcpyAsync(c->dimg, himg, sizeof(ImageTile) * size_t(nimg), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // h and himg are freed below
    delete[] h;
    delete[] himg;
    if (e != cudaSuccess) return e;
    c->n_img = nimg;
    c->n_etiles = n;
    c->n_itiles = hole ? ni : 0;
    c->planned = true;
    return cudaSuccess;
}

// The interior launches of one time step, one per interior rectangle
// (nothing if the body has no interior).
static cudaError_t launch_interior_part(lbm_ctx* c, const StepParams& p, bool fields) {
    if (c->n_irect < 1) return cudaSuccess;
    // one launch over every interior rectangle
    InteriorRects R;
    memset(&R, 0, sizeof(R));
    int64_t total = 0;
    for (int q = 0; q < 4; ++q) {
        if (q < c->n_irect) {
            for (int k = 0; k < 4; ++k) R.g[q].rect[k] = c->irect[q][k];
            R.g[q].strip_x0 = c->i_strip_x0[q];
            R.g[q].strip_w = c->i_strip_w[q];
            R.g[q].chunk_rows = c->i_chunk[q];
            R.tiles_x[q] = c->i_tiles_x[q];
            R.first[q] = int32_t(total);
            total += int64_t(c->i_tiles_x[q]) * c->i_tiles_y[q];
        } else {
            R.tiles_x[q] = 1;
            R.first[q] = INT32_MAX;
        }
    }
    if (total > INT32_MAX - 1) return cudaErrorInvalidConfiguration;
    R.total = int32_t(total);
    StepParams pi = p;
    pi.ring_slots = c->i_ring;
    return launch_interior(c->fmt, pi, R, c->stream, fields);
}

// The edge-band launch of one time step (the whole body without an interior).
static cudaError_t launch_band_part(lbm_ctx* c, int parity, bool fields, cudaStream_t st) {
    EdgeLaunch L;
    memset(&L, 0, sizeof(L));
    L.params = c->dparams + parity;
    L.tiles = c->dtiles;
    L.fields = fields ? 1 : 0;
    return launch_edge(c->fmt, L, c->n_etiles, st, 0, c->hole[0] < c->hole[1], c->scheme == LBM_SCHEME_EXTRAPOLATED);
}

// The edge-band tiles and the seam images of one step in one launch on the
// context's stream.
static cudaError_t launch_band_images_part(lbm_ctx* c, int parity, bool fields) {
    EdgeLaunch L;
    memset(&L, 0, sizeof(L));
    L.params = c->dparams + parity;
    L.tiles = c->dtiles;
    L.fields = fields ? 1 : 0;
    return launch_edge_images(c->fmt, L, c->n_etiles, c->dimg, c->n_img, c->stream, c->hole[0] < c->hole[1],
                              c->scheme == LBM_SCHEME_EXTRAPOLATED);
}

// Launches of one time step (mode 0) or the initialisation (mode 1).
static cudaError_t launch_step_kernels(lbm_ctx* c, int mode, bool fields, int parity) {
    if (mode == 1 && c->n_itiles > 0) {  // a holed body: the plan's tiles
        EdgeLaunch L;
        memset(&L, 0, sizeof(L));
        L.params = c->dparams + parity;
        L.tiles = c->dtiles;
        L.fields = fields ? 1 : 0;
        return launch_edge(c->fmt, L, c->n_itiles, c->stream, 1, true, false);
    }
    if (mode == 1) {
        EdgeLaunch L;
        memset(&L, 0, sizeof(L));
        L.params = c->dparams + parity;
        L.tiles = nullptr;
        L.fields = fields ? 1 : 0;
        L.rect[0] = 0;
        L.rect[1] = c->nx;
        L.rect[2] = 0;
        L.rect[3] = c->ny;
        L.rtiles_x = (c->nx + kInitOutW - 1) / kInitOutW;
        const int64_t ntiles = int64_t(L.rtiles_x) * ((c->ny + kInitOutH - 1) / kInitOutH);
        if (ntiles > 0x7fffffff) return cudaErrorInvalidConfiguration;
        return launch_edge(c->fmt, L, int(ntiles), c->stream, 1, true, false);
    }
    if (!c->has_interior) return launch_band_part(c, parity, fields, c->stream);
    if (c->n_img > 0) {
        // the interior across a periodic seam: then the band tiles and the
        // seam images in one launch after it (the images copy what it wrote)
        cudaError_t e = launch_interior_part(c, make_params(c, parity), fields);
        if (e == cudaSuccess) e = launch_band_images_part(c, parity, fields);
        return e;
    }
    // interior first on the main stream, then the edge tiles on the side
    // stream: the small edge CTAs fill the room the interior CTAs leave
    cudaError_t e = cudaEventRecord(c->ev_fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    if (e == cudaSuccess) e = launch_interior_part(c, make_params(c, parity), fields);
    if (e == cudaSuccess) e = launch_band_part(c, parity, fields, c->side);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    return e;
}

static lbm_status launch(lbm_ctx* c, int mode, bool fields) {
    if (!c->planned) LBM_CUDA(c, build_plan(c));
    LBM_CUDA(c, launch_step_kernels(c, mode, fields, c->parity));
    c->parity ^= 1;
    if (mode == 0) c->steps += 1;
    return LBM_OK;
}

lbm_status lbm::ctx_ensure_initialized(lbm_ctx* c) {
    if (c->initialized) return LBM_OK;
    lbm_status st = launch(c, 1, true);
    if (st != LBM_OK) return st;
    c->initialized = true;
    // the initial fields are read only by the initialisation: give them back
    if (c->u0 || c->v0) {
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
        const int64_t ubytes = int64_t(2) * c->nx * c->ny * int64_t(sizeof(double));
        if (c->u0) c->device_bytes -= ubytes;
        if (c->v0) c->device_bytes -= ubytes;
        cudaFree(c->u0);
        cudaFree(c->v0);
        c->u0 = c->v0 = nullptr;
    }
    return LBM_OK;
}

// A graph of kGraphChunk plain steps starting at parity `par`.
static lbm_status get_graph(lbm_ctx* c, int par, cudaGraphExec_t* out) {
    if (c->graph[par]) {
        *out = c->graph[par];
        return LBM_OK;
    }
    cudaGraph_t g = nullptr;
    LBM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < kGraphChunk && err == cudaSuccess; ++k) err = launch_step_kernels(c, 0, false, par ^ (k & 1));
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return ctx_fail_cuda(c, err);
    }
    if (e2 != cudaSuccess) return ctx_fail_cuda(c, e2);
    cudaGraphExec_t ex = nullptr;
    err = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return ctx_fail_cuda(c, err);
    c->graph[par] = ex;
    *out = ex;
    return LBM_OK;
}

// Device flag bits: 1 non-finite value or J <= 0; 4 a bounded wait gave up;
// 8 a bulk copy was refused for misalignment (an internal error).
lbm_status lbm::ctx_check_flag(lbm_ctx* c) {
    int32_t h = 0;
    LBM_CUDA(c, cudaMemcpyAsync(&h, c->flag, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h & 8) return ctx_fail_cuda(c, cudaErrorMisalignedAddress);
    if (h & 4) return LBM_E_TIMEOUT;
    return (h & 1) ? LBM_E_UNSTABLE : LBM_OK;
}

static void free_all(lbm_ctx* c) {
    for (int k = 0; k < 2; ++k) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        cudaFree(c->f[k]);
        cudaFree(c->a[k]);
        cudaFree(c->s[k]);
    }
    cudaFree(c->fields);
    cudaFree(c->u0);
    cudaFree(c->v0);
    cudaFree(c->flag);
    cudaFree(c->counter);
    cudaFree(c->partials);
    cudaFree(c->diag);
    cudaFree(c->readout);
    cudaFree(c->dparams);
    cudaFree(c->dtiles);
    cudaFree(c->dimg);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->owns_stream && c->stream) cudaStreamDestroy(c->stream);
}

static bool finite_pair(const double* v) { return v == nullptr || (isfinite(v[0]) && isfinite(v[1])); }



extern "C" {

lbm_status lbm_create(const lbm_desc* d, lbm_ctx** out) {
    NvtxRange range_("lbm_create");
    if (!out) return LBM_E_INVALID;
    *out = nullptr;
    if (!d) return LBM_E_INVALID;
    if (d->nx < 3 || d->ny < 3 || !(d->dX > 0) || !isfinite(d->dX)) return LBM_E_INVALID;
    if (d->storage < LBM_F64 || d->storage > LBM_BF16) return LBM_E_INVALID;
    if (d->u_carry != LBM_UCARRY_NATIVE && d->u_carry != LBM_UCARRY_COMPENSATED &&
        d->u_carry != LBM_UCARRY_COMPENSATED16)
        return LBM_E_INVALID;
    if (d->scheme != LBM_SCHEME_EXPLICIT && d->scheme != LBM_SCHEME_PREDICTOR &&
        d->scheme != LBM_SCHEME_EXTRAPOLATED)
        return LBM_E_INVALID;
    if (d->f16_scale_log2 < -60 || d->f16_scale_log2 > 60) return LBM_E_INVALID;
    // sizes: 64-bit element counts, 32-bit node coordinates
    const int64_t nodes = int64_t(d->nx) * d->ny;
    if (d->nx > (1 << 30) || d->ny > (1 << 30) || nodes > (int64_t(1) << 40)) return LBM_E_INVALID;
    if (fault_injected("alloc")) return LBM_E_OOM;  // before any CUDA call

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_E_OOM;
    c->device = d->device;
    DeviceGuard guard(c->device);
    if (!guard.ok) {
        delete c;
        return LBM_E_INVALID;
    }
    c->stream = static_cast<cudaStream_t>(d->cuda_stream);
    if (!c->stream) {
        // graphs cannot be captured on the legacy default stream: own one
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return LBM_E_CUDA;
        }
        c->owns_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return LBM_E_CUDA;
    }
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        c->num_sms < 1) {
        cudaGetLastError();
        c->num_sms = 1;
    }
    c->nx = d->nx;
    c->ny = d->ny;
    c->dX = d->dX;
    c->scheme = d->scheme;
    c->f16_scale_log2 = d->f16_scale_log2 ? d->f16_scale_log2 : 10;
    {
        // the 16-bit low words of the u-carry: |u| < 2^b = 8 max(nx, ny) dX
        // rounded up keeps |lo| 2^k below 2^15 for k = 40 - b
        int b = 0;
        frexp(8.0 * double(std::max(d->nx, d->ny)) * d->dX, &b);
        c->lo_log2 = std::min(100, std::max(-100, 40 - b));
    }
    switch (d->storage) {
        case LBM_F64: c->fmt = kFmtF64; break;
        case LBM_F32:
            c->fmt = d->u_carry == LBM_UCARRY_COMPENSATED ? kFmtF32C
                     : d->u_carry == LBM_UCARRY_COMPENSATED16 ? kFmtF32H : kFmtF32;
            break;
        case LBM_F16: c->fmt = kFmtF16; break;
        default: c->fmt = kFmtBF16; break;
    }
    for (int e = 0; e < 4; ++e) {
        memset(&c->bc[e], 0, sizeof(EdgeBC));
        c->bc[e].times[2] = INFINITY;
    }
    // plane layout: kPadCols columns / kPadRows rows of padding on each side,
    // pitch a multiple of 64 elements covering the widest bulk-copied row
    // segment of the interior kernel (a strip starting as far right as
    // column nx - 1 reads a segment of up to kSegMax elements from 8 columns
    // left of it)
    const int64_t need = kPadCols + int64_t(d->nx) + kSegMax + 16;
    c->pitch = (need + 63) / 64 * 64;
    c->plane = c->pitch * (int64_t(d->ny) + 2 * kPadRows);
    if (c->plane > 0x7fffffffLL) {  // the interior kernel indexes a plane with 32-bit offsets
        free_all(c);
        delete c;
        return LBM_E_INVALID;
    }

    const size_t fbytes = size_t(9) * c->plane * elem_size_storage(c->fmt);
    const size_t abytes = ucarry_bytes(c->fmt) * c->plane;
    const size_t sbytes = size_t(source_planes(d->scheme)) * c->plane * elem_size_compute(c->fmt);
    const size_t fldbytes = size_t(5) * nodes * sizeof(double);
    const size_t ubytes = size_t(2) * nodes * sizeof(double);
    c->diag_blocks = diagnostics_blocks(nodes);
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < 2 && err == cudaSuccess; ++k) {
        err = cudaMalloc(&c->f[k], fbytes);
        if (err == cudaSuccess) err = cudaMalloc(&c->a[k], abytes);
        if (err == cudaSuccess) err = cudaMalloc(&c->s[k], sbytes);
    }
    if (err == cudaSuccess) err = cudaMalloc(&c->fields, fldbytes);
    if (err == cudaSuccess && d->u0) err = cudaMalloc(&c->u0, ubytes);
    if (err == cudaSuccess && d->v0) err = cudaMalloc(&c->v0, ubytes);
    if (err == cudaSuccess) err = cudaMalloc(&c->flag, sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMalloc(&c->counter, 2 * sizeof(int64_t));
    if (err == cudaSuccess) err = cudaMalloc(&c->partials, size_t(c->diag_blocks) * 8 * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&c->diag, 8 * sizeof(double));
    if (err != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return err == cudaErrorMemoryAllocation ? LBM_E_OOM : LBM_E_CUDA;
    }
    c->device_bytes = int64_t(2 * (fbytes + abytes + sbytes) + fldbytes + (d->u0 ? ubytes : 0) + (d->v0 ? ubytes : 0));
    // the state is cleared on the side stream while the initial fields are
    // uploaded on the main one (the copy engines and the SMs work at once)
    for (int k = 0; k < 2 && err == cudaSuccess; ++k) {
        err = cudaMemsetAsync(c->f[k], 0, fbytes, c->side);
        if (err == cudaSuccess) err = cudaMemsetAsync(c->a[k], 0, abytes, c->side);
        if (err == cudaSuccess) err = cudaMemsetAsync(c->s[k], 0, sbytes, c->side);
    }
    if (err == cudaSuccess) err = cudaMemsetAsync(c->fields, 0, fldbytes, c->side);
    if (err == cudaSuccess) err = cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->side);
    if (err == cudaSuccess) err = cudaMemsetAsync(c->counter, 0, 2 * sizeof(int64_t), c->side);
    if (err == cudaSuccess && d->u0) err = cudaMemcpyAsync(c->u0, d->u0, ubytes, cudaMemcpyHostToDevice, c->stream);
    if (err == cudaSuccess && d->v0) err = cudaMemcpyAsync(c->v0, d->v0, ubytes, cudaMemcpyHostToDevice, c->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->side);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    if (err != cudaSuccess) {
        free_all(c);
        delete c;
        return LBM_E_CUDA;
    }
    *out = c;
    return LBM_OK;
}

lbm_status lbm_set_material(lbm_ctx* c, double lambda, double mu, double rho0, double omega,
                            const double body_force[2]) {
    if (!c) return LBM_E_INVALID;
    if (c->sticky) return LBM_E_CUDA;
    if (c->initialized) return LBM_E_STATE;
    if (!(mu > 0) || !(rho0 > 0) || !(lambda > -mu) || !(omega > 0) || !(omega < 2)) return LBM_E_INVALID;
    if (!isfinite(mu) || !isfinite(rho0) || !isfinite(lambda) || !finite_pair(body_force)) return LBM_E_INVALID;
    c->lambda = lambda;
    c->mu = mu;
    c->rho0 = rho0;
    c->omega = omega;
    c->body[0] = body_force ? body_force[0] : 0.0;
    c->body[1] = body_force ? body_force[1] : 0.0;
    // dt = dX / (sqrt(3) C_s), C_s = sqrt(mu / rho0); lattice speed c = dX / dt
    const double Cs = sqrt(mu / rho0);
    c->dt = c->dX / (sqrt(3.0) * Cs);
    c->c = c->dX / c->dt;
    c->cs2 = Cs * Cs;
    c->material_set = true;
    return LBM_OK;
}

lbm_status lbm_set_boundary(lbm_ctx* c, int32_t edge, int32_t kind, const double value[2],
                            const double rate[2], const double times[3]) {
    if (!c) return LBM_E_INVALID;
    if (c->sticky) return LBM_E_CUDA;
    if (c->initialized) return LBM_E_STATE;
    if (edge < 0 || edge > 3 || kind < LBM_PERIODIC || kind > LBM_NEUMANN) return LBM_E_INVALID;
    if (!finite_pair(value) || !finite_pair(rate)) return LBM_E_INVALID;
    EdgeBC e;
    memset(&e, 0, sizeof(e));
    e.kind = kind;
    for (int a = 0; a < 2; ++a) {
        e.value[a] = value ? value[a] : 0.0;
        e.rate[a] = rate ? rate[a] : 0.0;
    }
    e.times[0] = times ? times[0] : 0.0;
    e.times[1] = times ? times[1] : 0.0;
    e.times[2] = times ? times[2] : INFINITY;
    if (times && (isnan(times[0]) || isnan(times[1]) || isnan(times[2]) || times[1] < 0)) return LBM_E_INVALID;
    // a periodic edge must pair with a periodic opposite edge
    const int other = edge ^ 1;
    if (c->bc_set[other] && ((c->bc[other].kind == kPeriodic) != (kind == LBM_PERIODIC))) return LBM_E_INVALID;
    c->bc[edge] = e;
    c->bc_set[edge] = true;
    return LBM_OK;
}

lbm_status lbm_set_hole(lbm_ctx* c, const int32_t hole[4], const double traction[8]) {
    if (!c || !hole) return LBM_E_INVALID;
    if (c->sticky) return LBM_E_CUDA;
    if (c->initialized) return LBM_E_STATE;
    if (!c->bc_set[0] || !c->bc_set[2]) return LBM_E_STATE;  // the margins depend on the axes' kinds
    // the hole's 2-node band must clear the bands of the body's edges (2
    // nodes at a bounded edge, 3 at a periodic seam) and its images
    const int mx = c->bc[0].kind == kPeriodic ? 5 : 4, my = c->bc[2].kind == kPeriodic ? 5 : 4;
    if (!(hole[0] < hole[1] && hole[2] < hole[3]) || hole[0] < mx || hole[1] > c->nx - mx || hole[2] < my ||
        hole[3] > c->ny - my)
        return LBM_E_INVALID;
    double T[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (traction)
        for (int k = 0; k < 8; ++k) {
            if (!isfinite(traction[k])) return LBM_E_INVALID;
            T[k] = traction[k];
        }
    for (int k = 0; k < 4; ++k) c->hole[k] = hole[k];
    for (int k = 0; k < 8; ++k) c->hole_T[k] = T[k];
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int64_t nsteps) {
    NvtxRange range_("lbm_step");
    lbm_status st = ctx_ready(c);
    if (st != LBM_OK) return st;
    if (nsteps < 0) return LBM_E_INVALID;
    if (fault_injected("step")) return ctx_fail_cuda(c, cudaErrorLaunchFailure);
    DeviceGuard guard(c->device);
    if (!guard.ok) return ctx_fail_cuda(c, cudaErrorInvalidDevice);
    st = ctx_ensure_initialized(c);
    if (st != LBM_OK || nsteps == 0) return st;
    int64_t left = nsteps;
    // plain launches until the variant is warm (attributes set outside capture)
    if (!c->variant_warm && left > 1) {
        st = launch(c, 0, false);
        if (st != LBM_OK) return st;
        --left;
        c->variant_warm = true;
    }
    while (left > kGraphChunk) {
        cudaGraphExec_t g;
        st = get_graph(c, c->parity, &g);
        if (st != LBM_OK) return st;
        LBM_CUDA(c, cudaGraphLaunch(g, c->stream));
        c->steps += kGraphChunk;  // kGraphChunk is even: parity unchanged
        left -= kGraphChunk;
    }
    while (left > 1) {
        st = launch(c, 0, false);
        if (st != LBM_OK) return st;
        --left;
    }
    return launch(c, 0, true);
}

lbm_status lbm_profile_steps(lbm_ctx* c, int64_t nsteps, double out[4]) {
    lbm_status st = ctx_ready(c);
    if (st != LBM_OK) return st;
    if (nsteps < 1 || nsteps > 4096 || !out) return LBM_E_INVALID;
    DeviceGuard guard(c->device);
    if (!guard.ok) return ctx_fail_cuda(c, cudaErrorInvalidDevice);
    st = ctx_ensure_initialized(c);
    if (st != LBM_OK) return st;
    if (!c->planned) LBM_CUDA(c, build_plan(c));
    // events e[2k] before step k's interior launch, e[2k+1] between it and
    // the band launch, e[2k+2] after the band launch (and the image launch
    // of a periodic body, timed with it)
    const int64_t nev = 2 * nsteps + 1;
    cudaEvent_t* ev = new (std::nothrow) cudaEvent_t[size_t(nev)];
    if (!ev) return LBM_E_OOM;
    int64_t made = 0;
    cudaError_t err = cudaSuccess;
    for (; made < nev && err == cudaSuccess; ++made) err = cudaEventCreate(&ev[made]);
    if (err != cudaSuccess) --made;
    if (err == cudaSuccess) err = cudaEventRecord(ev[0], c->stream);
    for (int64_t k = 0; k < nsteps && err == cudaSuccess; ++k) {
        const bool fields = k + 1 == nsteps;  // the last step refreshes the read-out fields
        const StepParams p = make_params(c, c->parity);
        err = launch_interior_part(c, p, fields);
        if (err == cudaSuccess) err = cudaEventRecord(ev[2 * k + 1], c->stream);
        if (err == cudaSuccess)
            err = c->n_img > 0 ? launch_band_images_part(c, c->parity, fields)
                               : launch_band_part(c, c->parity, fields, c->stream);
        if (err == cudaSuccess) err = cudaEventRecord(ev[2 * k + 2], c->stream);
        if (err == cudaSuccess) {
            c->parity ^= 1;
            c->steps += 1;
        }
    }
    if (err == cudaSuccess) err = cudaEventSynchronize(ev[nev - 1]);
    double sum[3] = {0, 0, 0};
    const int64_t counted = nsteps > 1 ? nsteps - 1 : 1;  // the last step also writes the fields
    for (int64_t k = 0; k < counted && err == cudaSuccess; ++k) {
        float a = 0, b = 0;
        err = cudaEventElapsedTime(&a, ev[2 * k], ev[2 * k + 1]);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&b, ev[2 * k + 1], ev[2 * k + 2]);
        sum[0] += a;
        sum[1] += b;
        sum[2] += double(a) + double(b);
    }
    for (int64_t q = 0; q < made; ++q) cudaEventDestroy(ev[q]);
    delete[] ev;
    if (err != cudaSuccess) return ctx_fail_cuda(c, err);
    for (int q = 0; q < 3; ++q) out[q] = sum[q] / double(counted);
    out[3] = double(interior_nodes(c));
    return ctx_check_flag(c);
}

lbm_status lbm_profile_interior(lbm_ctx* c, int64_t nlaunches, double out[2]) {
    lbm_status st = ctx_ready(c);
    if (st != LBM_OK) return st;
    if (nlaunches < 1 || nlaunches > 4096 || !out) return LBM_E_INVALID;
    DeviceGuard guard(c->device);
    if (!guard.ok) return ctx_fail_cuda(c, cudaErrorInvalidDevice);
    st = ctx_ensure_initialized(c);
    if (st != LBM_OK) return st;
    if (!c->planned) LBM_CUDA(c, build_plan(c));
    if (!c->has_interior) return LBM_E_INVALID;
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    // the state the next step reads, and the device flag, saved on the device
    const int q = c->parity;
    const size_t fb = size_t(9) * size_t(c->plane) * elem_size_storage(c->fmt);
    const size_t ab = ucarry_bytes(c->fmt) * size_t(c->plane);
    const size_t sb = size_t(source_planes(c->scheme)) * size_t(c->plane) * elem_size_compute(c->fmt);
    unsigned char* save = nullptr;
    cudaError_t err = cudaMalloc(&save, fb + ab + sb + sizeof(int32_t));
    if (err != cudaSuccess) {
        cudaGetLastError();
        return err == cudaErrorMemoryAllocation ? LBM_E_OOM : ctx_fail_cuda(c, err);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    err = cudaMemcpyAsync(save, c->f[q], fb, cudaMemcpyDeviceToDevice, c->stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(save + fb, c->a[q], ab, cudaMemcpyDeviceToDevice, c->stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(save + fb + ab, c->s[q], sb, cudaMemcpyDeviceToDevice, c->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(save + fb + ab + sb, c->flag, sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = launch_interior_part(c, make_params(c, q), false);  // warm
    if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
    for (int64_t k = 0; k < nlaunches && err == cudaSuccess; ++k)
        err = launch_interior_part(c, make_params(c, q ^ int((k + 1) & 1)), false);
    if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
    // restore: the context continues from the saved state
    if (err == cudaSuccess) err = cudaMemcpyAsync(c->f[q], save, fb, cudaMemcpyDeviceToDevice, c->stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(c->a[q], save + fb, ab, cudaMemcpyDeviceToDevice, c->stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(c->s[q], save + fb + ab, sb, cudaMemcpyDeviceToDevice, c->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(c->flag, save + fb + ab + sb, sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    float ms = 0;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    if (err != cudaSuccess) return ctx_fail_cuda(c, err);
    out[0] = double(ms) / double(nlaunches);
    out[1] = double(interior_nodes(c));
    return ctx_check_flag(c);
}

lbm_status lbm_set_tuning(lbm_ctx* c, const lbm_tuning* t) {
    if (!c || !t) return LBM_E_INVALID;
    if (c->sticky) return LBM_E_CUDA;
    if (c->planned) return LBM_E_STATE;
    if ((t->ring_slots != 0 && (t->ring_slots < 4 || t->ring_slots > 8)) ||
        (t->chunk_rows != 0 && (t->chunk_rows < 8 || t->chunk_rows > (1 << 20))) || t->aligned < -1 ||
        t->aligned > 2 || t->plan < 0 || t->plan > 2)
        return LBM_E_INVALID;
    c->tune_ring = t->ring_slots;
    c->tune_chunk = t->chunk_rows;
    c->tune_aligned = t->aligned;
    c->tune_plan = t->plan;
    return LBM_OK;
}

lbm_status lbm_get_tuning(const lbm_ctx* c, lbm_tuning* t) {
    if (!c || !t) return LBM_E_INVALID;
    if (c->planned && c->has_interior) {
        t->ring_slots = c->i_ring;
        t->chunk_rows = c->i_chunk[0];
        t->aligned = c->tune_aligned > 0 ? c->tune_aligned : 0;
        t->plan = 2;
    } else {
        t->ring_slots = c->tune_ring;
        t->chunk_rows = c->tune_chunk;
        t->aligned = c->tune_aligned;
        t->plan = c->planned ? 1 : c->tune_plan;
    }
    return LBM_OK;
}

lbm_status lbm_autotune(const lbm_desc* d, const int32_t edge_kind[4], int64_t steps, lbm_tuning* best,
                        double* best_ms) {
    NvtxRange range_("lbm_autotune");
    if (!d || !edge_kind || !best || steps < 1 || steps > 100000) return LBM_E_INVALID;
    for (int e = 0; e < 4; ++e)
        if (edge_kind[e] < LBM_PERIODIC || edge_kind[e] > LBM_NEUMANN) return LBM_E_INVALID;
    if ((edge_kind[0] == LBM_PERIODIC) != (edge_kind[1] == LBM_PERIODIC) ||
        (edge_kind[2] == LBM_PERIODIC) != (edge_kind[3] == LBM_PERIODIC))
        return LBM_E_INVALID;
    lbm_desc sd = *d;  // the same body shape and format, zero initial fields
    sd.u0 = nullptr;
    sd.v0 = nullptr;
    // candidates: the interior kernel with ring depth x rows per CTA (0: one
    // wave) x strip grid, and edge tiles only
    const int rings[3] = {4, 5, 6};
    const int chunks[4] = {0, 32, 96, 256};
    lbm_tuning cand[25];
    int ncand = 0;
    for (int a = 0; a < 2; ++a)
        for (int ri = 0; ri < 3; ++ri)
            for (int ci = 0; ci < 4; ++ci) {
                if (chunks[ci] > 0 && chunks[ci] >= d->ny) continue;  // the same as one chunk of all rows
                cand[ncand++] = lbm_tuning{rings[ri], chunks[ci], a, 2};
            }
    cand[ncand++] = lbm_tuning{0, 0, -1, 1};
    double best_t = INFINITY;
    lbm_tuning bt = {0, 0, -1, 0};
    lbm_status last = LBM_OK;
    for (int k = 0; k < ncand; ++k) {
        lbm_ctx* c = nullptr;
        lbm_status st = lbm_create(&sd, &c);
        if (st != LBM_OK) return st;
        const lbm_tuning t = cand[k];
        st = lbm_set_tuning(c, &t);
        if (st == LBM_OK) st = lbm_set_material(c, 0.3, 0.3, 1.0, 1.0, nullptr);
        for (int e = 0; e < 4 && st == LBM_OK; ++e)
            st = lbm_set_boundary(c, e, edge_kind[e], nullptr, nullptr, nullptr);
        // warm: initialisation, a plain step, the graphs of both parities
        if (st == LBM_OK) st = lbm_step(c, 2 * kGraphChunk + 2);
        double ms = INFINITY;
        if (st == LBM_OK) {
            DeviceGuard guard(c->device);
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            cudaError_t err = cudaEventCreate(&e0);
            if (err == cudaSuccess) err = cudaEventCreate(&e1);
            if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
            if (err == cudaSuccess) st = lbm_step(c, steps);
            if (err == cudaSuccess && st == LBM_OK) err = cudaEventRecord(e1, c->stream);
            if (err == cudaSuccess && st == LBM_OK) err = cudaEventSynchronize(e1);
            float f = 0;
            if (err == cudaSuccess && st == LBM_OK && cudaEventElapsedTime(&f, e0, e1) == cudaSuccess)
                ms = double(f) / double(steps);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            if (err != cudaSuccess) st = LBM_E_CUDA;
        }
        lbm_destroy(c);
        if (st != LBM_OK) {
            last = st;
            continue;
        }
        if (ms < best_t) {
            best_t = ms;
            bt = t;
        }
    }
    if (!(best_t < INFINITY)) return last != LBM_OK ? last : LBM_E_CUDA;
    *best = bt;
    if (best_ms) *best_ms = best_t;
    return LBM_OK;
}

int64_t lbm_fields_size(const lbm_ctx* c, uint32_t mask) {
    if (!c || mask == 0 || (mask & ~127u)) return 0;
    static const int comps[7] = {2, 2, 4, 3, 1, 3, 1};
    int64_t n = 0;
    for (int b = 0; b < 7; ++b)
        if (mask & (1u << b)) n += comps[b];
    return n * int64_t(c->nx) * c->ny;
}

lbm_status lbm_read_fields(lbm_ctx* c, uint32_t mask, double* out, int64_t out_len, double* t_out) {
    NvtxRange range_("lbm_read_fields");
    lbm_status st = ctx_ready(c);
    if (st != LBM_OK) return st;
    const int64_t need = lbm_fields_size(c, mask);
    if (need == 0 || !out || out_len < need) return LBM_E_INVALID;
    DeviceGuard guard(c->device);
    if (!guard.ok) return ctx_fail_cuda(c, cudaErrorInvalidDevice);
    st = ctx_ensure_initialized(c);
    if (st != LBM_OK) return st;
    const size_t bytes = size_t(need) * sizeof(double);
    if (bytes > c->readout_cap) {
        cudaFree(c->readout);
        c->readout = nullptr;
        c->readout_cap = 0;
        cudaError_t e = cudaMalloc(&c->readout, bytes);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return LBM_E_OOM;
        }
        LBM_CUDA(c, e);
        c->readout_cap = bytes;
    }
    ReadoutParams rp = make_readout(c);
    LBM_CUDA(c, launch_readout(rp, mask, c->readout, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync(out, c->readout, bytes, cudaMemcpyDeviceToHost, c->stream));
    if (t_out) *t_out = double(c->steps) * c->dt;
    return ctx_check_flag(c);
}

lbm_status lbm_diagnostics(lbm_ctx* c, double out[6]) {
    NvtxRange range_("lbm_diagnostics");
    lbm_status st = ctx_ready(c);
    if (st != LBM_OK) return st;
    if (!out) return LBM_E_INVALID;
    DeviceGuard guard(c->device);
    if (!guard.ok) return ctx_fail_cuda(c, cudaErrorInvalidDevice);
    st = ctx_ensure_initialized(c);
    if (st != LBM_OK) return st;
    ReadoutParams rp = make_readout(c);
    LBM_CUDA(c, launch_diagnostics(rp, c->partials, c->diag_blocks, c->diag, c->stream));
    double h[8];
    LBM_CUDA(c, cudaMemcpyAsync(h, c->diag, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    st = ctx_check_flag(c);
    for (int q = 0; q < 6; ++q) out[q] = h[q];
    return st;
}

lbm_status lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_E_INVALID;
    if (c->sticky) return LBM_E_CUDA;
    DeviceGuard guard(c->device);
    if (!guard.ok) return ctx_fail_cuda(c, cudaErrorInvalidDevice);
    return ctx_check_flag(c);
}

// ---------------------------------------------------------------- checkpoint
// A saved state: this header, then the population planes, the u-carry
// planes and the source-carry planes of the current parity (whole planes:
// their ghost rows and columns hold the populations the boundary rules sent
// back and the periodic images), then the five read-out planes.
namespace {

struct StateHeader {
    char magic[8];
    int32_t fmt, nx, ny, scheme;
    int32_t lo_log2, pad;
    int64_t pitch, plane, steps;
    double dt;
    int64_t bytes;  // the whole state, header included
};
constexpr char kStateMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', '2'};

struct StateParts {
    size_t f, a, s, fields;
};

StateParts state_parts(const lbm_ctx* c) {
    StateParts p;
    p.f = size_t(9) * size_t(c->plane) * elem_size_storage(c->fmt);
    p.a = ucarry_bytes(c->fmt) * size_t(c->plane);
    p.s = size_t(source_planes(c->scheme)) * size_t(c->plane) * elem_size_compute(c->fmt);
    p.fields = size_t(5) * size_t(c->nx) * size_t(c->ny) * sizeof(double);
    return p;
}

StateHeader state_header(const lbm_ctx* c) {
    StateHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kStateMagic, sizeof(h.magic));
    h.fmt = c->fmt;
    h.nx = c->nx;
    h.ny = c->ny;
    h.scheme = c->scheme;
    h.lo_log2 = c->lo_log2;
    h.pitch = c->pitch;
    h.plane = c->plane;
    h.steps = c->steps;
    h.dt = c->dt;
    const StateParts p = state_parts(c);
    h.bytes = int64_t(sizeof(StateHeader) + p.f + p.a + p.s + p.fields);
    return h;
}

}  // namespace

int64_t lbm_state_size(const lbm_ctx* c) {
    if (!c) return 0;
    return state_header(c).bytes;
}

lbm_status lbm_read_state(lbm_ctx* c, void* out, int64_t out_len) {
    NvtxRange range_("lbm_read_state");
    lbm_status st = ctx_ready(c);
    if (st != LBM_OK) return st;
    const StateHeader h = state_header(c);
    if (!out || out_len < h.bytes) return LBM_E_INVALID;
    DeviceGuard guard(c->device);
    if (!guard.ok) return ctx_fail_cuda(c, cudaErrorInvalidDevice);
    st = ctx_ensure_initialized(c);
    if (st != LBM_OK) return st;
    const StateParts p = state_parts(c);
    unsigned char* o = static_cast<unsigned char*>(out);
    memcpy(o, &h, sizeof(h));
    size_t at = sizeof(h);
    const int q = c->parity;
    LBM_CUDA(c, cudaMemcpyAsync(o + at, c->f[q], p.f, cudaMemcpyDeviceToHost, c->stream));
    at += p.f;
    LBM_CUDA(c, cudaMemcpyAsync(o + at, c->a[q], p.a, cudaMemcpyDeviceToHost, c->stream));
    at += p.a;
    LBM_CUDA(c, cudaMemcpyAsync(o + at, c->s[q], p.s, cudaMemcpyDeviceToHost, c->stream));
    at += p.s;
    LBM_CUDA(c, cudaMemcpyAsync(o + at, c->fields, p.fields, cudaMemcpyDeviceToHost, c->stream));
    return ctx_check_flag(c);  // synchronises: out is complete
}

lbm_status lbm_write_state(lbm_ctx* c, const void* in, int64_t in_len) {
    NvtxRange range_("lbm_write_state");
    lbm_status st = ctx_ready(c);
    if (st != LBM_OK) return st;
    if (!in || in_len < int64_t(sizeof(StateHeader))) return LBM_E_INVALID;
    StateHeader h;
    memcpy(&h, in, sizeof(h));
    const StateHeader mine = state_header(c);
    if (memcmp(h.magic, kStateMagic, sizeof(h.magic)) != 0 || h.fmt != mine.fmt || h.nx != mine.nx ||
        h.ny != mine.ny || h.scheme != mine.scheme || h.lo_log2 != mine.lo_log2 || h.pitch != mine.pitch ||
        h.plane != mine.plane ||
        h.dt != mine.dt || h.bytes != mine.bytes || in_len < h.bytes || h.steps < 0)
        return LBM_E_INVALID;
    DeviceGuard guard(c->device);
    if (!guard.ok) return ctx_fail_cuda(c, cudaErrorInvalidDevice);
    if (!c->planned) LBM_CUDA(c, build_plan(c));
    // the work queued so far is done before its buffers are overwritten, and
    // the copies are done before `in` may be released
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    const StateParts p = state_parts(c);
    const unsigned char* src = static_cast<const unsigned char*>(in);
    size_t at = sizeof(h);
    const int q = c->parity;
    LBM_CUDA(c, cudaMemcpyAsync(c->f[q], src + at, p.f, cudaMemcpyHostToDevice, c->stream));
    at += p.f;
    LBM_CUDA(c, cudaMemcpyAsync(c->a[q], src + at, p.a, cudaMemcpyHostToDevice, c->stream));
    at += p.a;
    LBM_CUDA(c, cudaMemcpyAsync(c->s[q], src + at, p.s, cudaMemcpyHostToDevice, c->stream));
    at += p.s;
    LBM_CUDA(c, cudaMemcpyAsync(c->fields, src + at, p.fields, cudaMemcpyHostToDevice, c->stream));
    // the edge kernel evaluates the boundary data at the step counter of
    // this parity
    LBM_CUDA(c, cudaMemcpyAsync(c->counter + q, &h.steps, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->steps = h.steps;
    if (!c->initialized) {  // the restored state replaces the initialisation
        c->initialized = true;
        const int64_t ubytes = int64_t(2) * c->nx * c->ny * int64_t(sizeof(double));
        if (c->u0) c->device_bytes -= ubytes;
        if (c->v0) c->device_bytes -= ubytes;
        cudaFree(c->u0);
        cudaFree(c->v0);
        c->u0 = c->v0 = nullptr;
    }
    return LBM_OK;
}

lbm_status lbm_get_info(const lbm_ctx* c, int64_t* steps, double* dt) {
    if (!c) return LBM_E_INVALID;
    if (steps) *steps = c->steps;
    if (dt) *dt = c->dt;
    return LBM_OK;
}

lbm_status lbm_memory_info(const lbm_ctx* c, int64_t* device_bytes, int64_t* bytes_per_node_update) {
    if (!c) return LBM_E_INVALID;
    if (device_bytes) *device_bytes = c->device_bytes;
    if (bytes_per_node_update) {
        const int64_t per = int64_t(9 * elem_size_storage(c->fmt)) +
                            int64_t(ucarry_bytes(c->fmt)) +
                            int64_t(source_planes(c->scheme) * elem_size_compute(c->fmt));
        *bytes_per_node_update = 2 * per;
    }
    return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx* c) {
    if (!c) return LBM_OK;
    {
        DeviceGuard guard(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        else cudaDeviceSynchronize();
        free_all(c);
    }
    delete c;
    return LBM_OK;
}

const char* lbm_last_cuda_error(const lbm_ctx* c) {
    if (!c) return "no context";
    return c->last_error == cudaSuccess ? "none" : cudaGetErrorString(c->last_error);
}

const char* lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_E_INVALID: return "invalid argument";
        case LBM_E_OOM: return "out of memory";
        case LBM_E_CUDA: return "CUDA error (context unusable)";
        case LBM_E_UNSTABLE: return "unstable: non-finite value or J <= 0 met";
        case LBM_E_TIMEOUT: return "device-side wait timed out";
        case LBM_E_STATE: return "call out of order";
    }
    return "unknown status";
}

}  // extern "C"

// lbm_batch.cu -- many bodies advanced by shared launches (the C ABI's
// lbm_batch_* entry points).
//
// Each time step of a batch is two launches, as for a single body: the
// interior tiles of every member (one CTA per tile, longest first) on the
// batch's stream, and the edge tiles of every member, each CTA reading its
// member's parameters from a device table.  The edge launch runs on a side
// stream at the same time, or, when some member's interior runs across a
// periodic seam, after the interior launch with the seam-image copies
// appended to it.
// So small and uneven bodies share the GPU instead of each paying launches
// per step, and chunks of 64 steps replay as one CUDA graph.  Every node of
// every member goes through the same tile code and arithmetic as when the
// member is stepped alone (with the interior kernel: plan 2), so the results
// are bit-identical.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_context.h"
#include "lbm_kernels.h"

using namespace lbm;

namespace {

constexpr int kBatchGraphChunk = 64;  // steps per captured graph (even)

// An interior tile of a member while the work list is built.
struct InteriorWork {
    int32_t inst, bx, by;
};

}  // namespace

struct lbm_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    cudaStream_t side = nullptr;  // the edge tiles' stream
    cudaEvent_t ev_sync = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<lbm_ctx*> m;
    std::vector<int> base_parity;  // member parity when the batch step count is even
    int fmt = 0;
    int n_entries = 0;           // parameter-table entries per parity
    StepParams* dtab = nullptr;  // [2][n_entries]: entry q * n_entries + e at parity base_parity ^ q
    BatchItem* ditems = nullptr;  // interior tiles, longest first
    EdgeTile* dtiles = nullptr;   // edge tiles of every member
    ImageTile* dimg = nullptr;    // seam images of the members with a periodic axis
    int32_t** dflagptr = nullptr;  // device: each member's status flag
    int32_t* dflagval = nullptr;   // device: the flags gathered by lbm_batch_sync
    std::vector<int32_t> hflag;    // host copy of dflagval
    int n_work = 0;               // interior tiles
    int n_edge = 0;               // edge tiles
    int n_img = 0;                // image tiles
    int chunk_rows = 0;
    int ring = kBatchRing;
    int aligned = 1;  // strip grid of the interior tiles (interior_strips)
    bool holed = false;           // some member has a hole
    int64_t steps = 0;
    bool warm = false;
    bool sticky = false;
    cudaError_t last_error = cudaSuccess;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

namespace {

lbm_status batch_fail(lbm_batch* b, cudaError_t e) {
    b->sticky = true;
    b->last_error = e;
    return LBM_E_CUDA;
}

#define BATCH_CUDA(b, call)                              \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return batch_fail((b), e_); \
    } while (0)

void batch_free(lbm_batch* b) {
    for (int k = 0; k < 2; ++k)
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    cudaFree(b->dtab);
    cudaFree(b->ditems);
    cudaFree(b->dtiles);
    cudaFree(b->dimg);
    cudaFree(b->dflagptr);
    cudaFree(b->dflagval);
    if (b->ev_sync) cudaEventDestroy(b->ev_sync);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->owns_stream && b->stream) cudaStreamDestroy(b->stream);
}

// One batch time step from table parity q: the interior tiles on the batch's
// stream and the edge tiles on the side stream, forked from and joined to
// the batch's stream (the small edge CTAs fill the room the interior CTAs
// leave), or, with seam images, the edge tiles and the images after the
// interior on the batch's stream.
cudaError_t batch_launch(lbm_batch* b, int q, bool fields) {
    const StepParams* tab = b->dtab + size_t(q) * size_t(b->n_entries);
    BatchInteriorLaunch I;
    memset(&I, 0, sizeof(I));
    I.params = tab;
    I.items = b->ditems;
    I.fields = fields ? 1 : 0;
    I.nitems = b->n_work;
    EdgeLaunch E;
    memset(&E, 0, sizeof(E));
    E.params = tab;
    E.tiles = b->dtiles;
    E.fields = fields ? 1 : 0;
    if (b->n_img > 0) {
        // members across periodic seams: the interior, then every member's
        // edge tiles and seam images in one launch after it (the images copy
        // what the interior launch wrote; the two launches barely overlapped
        // anyway, six interior CTAs filling an SM's registers)
        cudaError_t e = launch_batch_interior(b->fmt, I, b->ring, b->stream, nullptr);
        if (e == cudaSuccess) e = launch_edge_images(b->fmt, E, b->n_edge, b->dimg, b->n_img, b->stream, b->holed, false);
        return e;
    }
    cudaError_t e = cudaEventRecord(b->ev_fork, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->ev_fork, 0);
    if (e == cudaSuccess) e = launch_batch_interior(b->fmt, I, b->ring, b->stream, nullptr);
    if (e == cudaSuccess) e = launch_edge(b->fmt, E, b->n_edge, b->side, 0, b->holed, false);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_join, b->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_join, 0);
    return e;
}

void advance_members(lbm_batch* b, int64_t k) {
    for (lbm_ctx* c : b->m) {
        c->steps += k;
        if (k & 1) c->parity ^= 1;
    }
    b->steps += k;
}

lbm_status batch_graph(lbm_batch* b, int q, cudaGraphExec_t* out) {
    if (b->graph[q]) {
        *out = b->graph[q];
        return LBM_OK;
    }
    cudaGraph_t g = nullptr;
    BATCH_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < kBatchGraphChunk && err == cudaSuccess; ++k) err = batch_launch(b, q ^ (k & 1), false);
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return batch_fail(b, err);
    }
    if (e2 != cudaSuccess) return batch_fail(b, e2);
    cudaGraphExec_t ex = nullptr;
    err = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return batch_fail(b, err);
    b->graph[q] = ex;
    *out = ex;
    return LBM_OK;
}

// The batch's default strip grid: 124-column strips for 16-bit storage
// (measured on the 256-body workload: 40 900 MLUPS against 38 700 with
// strips on 32-byte sectors, which are at most 112 columns wide in a 2-byte
// plane), sector-aligned strips otherwise (FP32: 36 700 against 36 100).
int batch_default_aligned(int fmt) { return fmt == kFmtF16 || fmt == kFmtBF16 ? 0 : 1; }

// Copies every member's status flag into one array (one launch and one
// copy for the whole batch instead of one round trip per member).
__global__ void gather_flags(int32_t* const* flags, int32_t* out, int n) {
    const int i = int(blockIdx.x * blockDim.x + threadIdx.x);
    if (i < n) out[i] = *flags[i];
}

// Orders `waiter` after the work enqueued so far on `s`.
cudaError_t stream_after(cudaStream_t waiter, cudaStream_t s, cudaEvent_t ev) {
    if (waiter == s) return cudaSuccess;
    cudaError_t e = cudaEventRecord(ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(waiter, ev, 0);
    return e;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(lbm_ctx* const* members, int32_t n, void* cuda_stream, lbm_batch** out) {
    return lbm_batch_create_tuned(members, n, cuda_stream, nullptr, out);
}

lbm_status lbm_batch_create_tuned(lbm_ctx* const* members, int32_t n, void* cuda_stream, const lbm_tuning* tuning,
                                  lbm_batch** out) {
    NvtxRange range_("lbm_batch_create");
    if (!out) return LBM_E_INVALID;
    *out = nullptr;
    if (!members || n < 1) return LBM_E_INVALID;
    if (tuning && ((tuning->ring_slots != 0 && (tuning->ring_slots < 4 || tuning->ring_slots > 8)) ||
                   (tuning->chunk_rows != 0 && (tuning->chunk_rows < 8 || tuning->chunk_rows > (1 << 20))) ||
                   tuning->aligned < -1 || tuning->aligned > 2))
        return LBM_E_INVALID;
    for (int i = 0; i < n; ++i) {
        if (!members[i]) return LBM_E_INVALID;
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return LBM_E_INVALID;
        if (members[i]->device != members[0]->device || members[i]->fmt != members[0]->fmt) return LBM_E_INVALID;
        if (members[i]->scheme == LBM_SCHEME_EXTRAPOLATED) return LBM_E_INVALID;  // single bodies only
        const lbm_status st = ctx_ready(members[i]);
        if (st != LBM_OK) return st;
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_E_OOM;
    b->device = members[0]->device;
    b->fmt = members[0]->fmt;
    DeviceGuard guard(b->device);
    if (!guard.ok) {
        delete b;
        return LBM_E_INVALID;
    }
    try {
        b->m.assign(members, members + n);
        b->base_parity.resize(size_t(n));
        b->hflag.resize(size_t(n));
    } catch (...) {
        delete b;
        return LBM_E_OOM;
    }
    // every member initialised (its initialisation is ordered before the
    // batch's first step by the streams; its flag is read by lbm_batch_sync)
    for (int i = 0; i < n; ++i) {
        lbm_status st = ctx_ensure_initialized(members[i]);
        if (st != LBM_OK) {
            delete b;
            return st;
        }
        b->base_parity[size_t(i)] = members[i]->parity;
    }
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSuccess;
    if (!b->stream) {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->owns_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_sync, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);

    // each member's rectangles: the interior kernel wherever the body allows
    // it (plan 2), whatever plan the member runs alone with (plan 0 gives
    // small bodies edge tiles only; in a batch their interior tiles share the
    // launch with the others'), unless the member asked for edge tiles only
    struct Rects {
        int irect[4][4];
        int n_irect;
        int brect[12][4];
        int nband;
    };
    std::vector<Rects> mr;
    try {
        mr.resize(size_t(n));
    } catch (...) {
        batch_free(b);
        delete b;
        return LBM_E_OOM;
    }
    // interior tiles: rows per chunk so that the batch holds about eight
    // waves of resident CTAs (at least 32 rows, at most 256)
    int64_t all_interior = 0;
    for (int i = 0; i < n; ++i) {
        const lbm_ctx* c = b->m[size_t(i)];
        Rects& r = mr[size_t(i)];
        plan_rects(c, c->tune_plan == 1, true, r.irect, &r.n_irect, r.brect, &r.nband);
        for (int k = 0; k < r.n_irect; ++k)
            all_interior += int64_t(r.irect[k][1] - r.irect[k][0]) * (r.irect[k][3] - r.irect[k][2]);
        b->holed = b->holed || c->hole[0] < c->hole[1];
    }
    b->ring = tuning && tuning->ring_slots ? tuning->ring_slots : kBatchRing;
    b->aligned = tuning && tuning->aligned >= 0 ? tuning->aligned : batch_default_aligned(b->fmt);
    // the interior kernel's CTAs per SM with this ring (the first call also
    // sets its shared-memory limit, outside any capture)
    int resident = 0;
    {
        BatchInteriorLaunch L;
        memset(&L, 0, sizeof(L));
        if (e == cudaSuccess) e = launch_batch_interior(b->fmt, L, b->ring, b->stream, &resident);
    }
    const int64_t wave = int64_t(b->m[0]->num_sms) * std::max(1, resident);
    b->chunk_rows = tuning && tuning->chunk_rows
                        ? tuning->chunk_rows
                        : int(std::min<int64_t>(256, std::max<int64_t>(32, all_interior / (int64_t(120) * wave * 8))));
    std::vector<StepParams> tab;
    std::vector<InteriorWork> work;
    std::vector<EdgeTile> tiles;
    std::vector<ImageTile> imgs;
    std::vector<BatchItem> items;
    try {
        // parameter table: one entry per interior rectangle of each member
        // (at least one per member; its edge tiles use the first), for both
        // parities: entry e of parity q at q * b->n_entries + e
        std::vector<int> first_entry(size_t(n), 0), strips, owner;
        std::vector<StepParams> ent;
        for (int i = 0; i < n; ++i) {
            lbm_ctx* c = b->m[size_t(i)];
            const Rects& mri = mr[size_t(i)];
            first_entry[size_t(i)] = int(ent.size());
            const int nr = std::max(1, mri.n_irect);
            for (int q = 0; q < nr; ++q) {
                StepParams p = make_params(c, b->base_parity[size_t(i)]);
                int ns = 0;
                if (q < mri.n_irect) {
                    for (int k = 0; k < 4; ++k) p.rect[k] = mri.irect[q][k];
                    interior_strips(b->fmt, p.rect[0], p.rect[1], b->aligned, &p.strip_x0, &p.strip_w, &ns);
                }
                p.chunk_rows = b->chunk_rows;
                p.ring_slots = b->ring;
                ent.push_back(p);
                strips.push_back(ns);
                owner.push_back(i);
                if (q < mri.n_irect) {
                    const int e = int(ent.size()) - 1;
                    const int h = p.rect[3] - p.rect[2];
                    const int sy = (h + b->chunk_rows - 1) / b->chunk_rows;
                    for (int by = 0; by < sy; ++by)
                        for (int bx = 0; bx < ns; ++bx) work.push_back(InteriorWork{e, bx, by});
                }
            }
        }
        b->n_entries = int(ent.size());
        tab.resize(size_t(2) * ent.size());
        for (size_t e = 0; e < ent.size(); ++e) {
            tab[e] = ent[e];
            // the other parity: the member's parameters of that parity with
            // this entry's plan
            const int i = owner[e];
            StepParams p = make_params(b->m[size_t(i)], b->base_parity[size_t(i)] ^ 1);
            for (int k = 0; k < 4; ++k) p.rect[k] = ent[e].rect[k];
            p.strip_x0 = ent[e].strip_x0;
            p.strip_w = ent[e].strip_w;
            p.chunk_rows = ent[e].chunk_rows;
            p.ring_slots = ent[e].ring_slots;
            tab[ent.size() + e] = p;
        }
        for (int i = 0; i < n; ++i) {
            const Rects& mri = mr[size_t(i)];
            bool first = true;
            const int e = first_entry[size_t(i)];
            for (int r = 0; r < mri.nband; ++r) {
                const unsigned bs = bounded_sides(b->m[size_t(i)], mri.brect[r]);
                const int cnt = edge_tiles_of_rect(mri.brect[r], e, nullptr, 0, false, kEdgeThreads, bs);
                const size_t at = tiles.size();
                tiles.resize(at + size_t(cnt));
                edge_tiles_of_rect(mri.brect[r], e, tiles.data() + at, cnt, first, kEdgeThreads, bs);
                first = first && cnt == 0;
            }
            // the images of its interior's nodes next to a periodic seam
            const lbm_ctx* c = b->m[size_t(i)];
            const bool perx = c->bc[0].kind == kPeriodic, pery = c->bc[2].kind == kPeriodic;
            if (mri.n_irect > 0 && (perx || pery)) {
                int box[4];
                seam_box(c, box);
                const int cnt = image_tiles_of_body(c->nx, c->ny, perx, pery, box, e, nullptr, 0);
                const size_t at = imgs.size();
                imgs.resize(at + size_t(cnt));
                image_tiles_of_body(c->nx, c->ny, perx, pery, box, e, imgs.data() + at, cnt);
            }
        }
        // longest tiles first: the short tiles of small bodies fill the tail
        // of the last wave
        auto rows_of = [&](const InteriorWork& w) {
            const StepParams& p = tab[size_t(w.inst)];
            return std::min(b->chunk_rows, p.rect[3] - p.rect[2]);
        };
        std::stable_sort(work.begin(), work.end(),
                         [&](const InteriorWork& x, const InteriorWork& y) { return rows_of(x) > rows_of(y); });
        items.reserve(work.size());
        for (const InteriorWork& w : work) items.push_back(BatchItem{w.inst, w.bx, w.by, 0});
    } catch (...) {
        batch_free(b);
        delete b;
        return LBM_E_OOM;
    }
    if (items.size() > 0x7fffffff || tiles.size() > 0x7fffffff || imgs.size() > 0x7fffffff)
        e = cudaErrorInvalidValue;
    b->n_work = int(work.size());
    b->n_edge = int(tiles.size());
    b->n_img = int(imgs.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->dtab, sizeof(StepParams) * tab.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->dflagptr, sizeof(int32_t*) * size_t(n));
    if (e == cudaSuccess) e = cudaMalloc(&b->dflagval, sizeof(int32_t) * size_t(n));
    std::vector<int32_t*> flagptr;
    try {
        for (lbm_ctx* c : b->m) flagptr.push_back(c->flag);
    } catch (...) {
        e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->dflagptr, flagptr.data(), sizeof(int32_t*) * size_t(n), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && !items.empty()) e = cudaMalloc(&b->ditems, sizeof(BatchItem) * items.size());
    if (e == cudaSuccess && !tiles.empty()) e = cudaMalloc(&b->dtiles, sizeof(EdgeTile) * tiles.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->dtab, tab.data(), sizeof(StepParams) * tab.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(b->ditems, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && !tiles.empty())
        e = cudaMemcpyAsync(b->dtiles, tiles.data(), sizeof(EdgeTile) * tiles.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && !imgs.empty()) e = cudaMalloc(&b->dimg, sizeof(ImageTile) * imgs.size());
    if (e == cudaSuccess && !imgs.empty())
        e = cudaMemcpyAsync(b->dimg, imgs.data(), sizeof(ImageTile) * imgs.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host tables die with this scope
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? LBM_E_OOM : LBM_E_CUDA;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps) {
    NvtxRange range_("lbm_batch_step");
    if (!b) return LBM_E_INVALID;
    if (b->sticky) return LBM_E_CUDA;
    if (nsteps < 0) return LBM_E_INVALID;
    if (fault_injected("batch_step")) return batch_fail(b, cudaErrorLaunchFailure);
    const int n = int(b->m.size());
    for (int i = 0; i < n; ++i) {
        lbm_ctx* c = b->m[size_t(i)];
        if (c->sticky) return LBM_E_CUDA;
        // a member stepped on its own since the batch was made is out of phase
        if (c->parity != (b->base_parity[size_t(i)] ^ int(b->steps & 1))) return LBM_E_STATE;
    }
    if (nsteps == 0) return LBM_OK;
    DeviceGuard guard(b->device);
    if (!guard.ok) return batch_fail(b, cudaErrorInvalidDevice);
    // the batch stream waits for work the members enqueued on their streams
    for (lbm_ctx* c : b->m) BATCH_CUDA(b, stream_after(b->stream, c->stream, c->ev_join));
    int64_t left = nsteps;
    if (!b->warm && left > 1) {
        BATCH_CUDA(b, batch_launch(b, int(b->steps & 1), false));
        advance_members(b, 1);
        --left;
        b->warm = true;
    }
    while (left > kBatchGraphChunk) {
        cudaGraphExec_t g;
        const lbm_status st = batch_graph(b, int(b->steps & 1), &g);
        if (st != LBM_OK) return st;
        BATCH_CUDA(b, cudaGraphLaunch(g, b->stream));
        advance_members(b, kBatchGraphChunk);
        left -= kBatchGraphChunk;
    }
    while (left > 0) {
        BATCH_CUDA(b, batch_launch(b, int(b->steps & 1), left == 1));
        advance_members(b, 1);
        --left;
    }
    // members' own streams wait for the batch before their next calls
    BATCH_CUDA(b, cudaEventRecord(b->ev_sync, b->stream));
    for (lbm_ctx* c : b->m)
        if (c->stream != b->stream) BATCH_CUDA(b, cudaStreamWaitEvent(c->stream, b->ev_sync, 0));
    return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b, int32_t* status) {
    if (!b) return LBM_E_INVALID;
    if (b->sticky) return LBM_E_CUDA;
    DeviceGuard guard(b->device);
    if (!guard.ok) return batch_fail(b, cudaErrorInvalidDevice);
    // every member's flag in one launch and one copy (the members' streams
    // wait for the batch's, so nothing of a member is pending elsewhere);
    // bits as for one context: 8 a refused copy (the member becomes
    // unusable), 4 a bounded wait gave up, 1 a non-finite value or J <= 0
    const int n = int(b->m.size());
    gather_flags<<<(n + 255) / 256, 256, 0, b->stream>>>(b->dflagptr, b->dflagval, n);
    BATCH_CUDA(b, cudaGetLastError());
    BATCH_CUDA(b, cudaMemcpyAsync(b->hflag.data(), b->dflagval, sizeof(int32_t) * size_t(n), cudaMemcpyDeviceToHost,
                                  b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    lbm_status worst = LBM_OK;
    for (int i = 0; i < n; ++i) {
        lbm_ctx* c = b->m[size_t(i)];
        const int32_t h = b->hflag[size_t(i)];
        lbm_status st = LBM_OK;
        if (c->sticky) st = LBM_E_CUDA;
        else if (h & 8) st = ctx_fail_cuda(c, cudaErrorMisalignedAddress);
        else if (h & 4) st = LBM_E_TIMEOUT;
        else if (h & 1) st = LBM_E_UNSTABLE;
        if (status) status[i] = st;
        if (worst == LBM_OK) worst = st;
    }
    return worst;
}

lbm_status lbm_batch_get_info(const lbm_batch* b, int64_t* steps, int32_t* interior_ctas, int32_t* edge_ctas) {
    if (!b) return LBM_E_INVALID;
    if (steps) *steps = b->steps;
    if (interior_ctas) *interior_ctas = b->n_work;
    if (edge_ctas) *edge_ctas = b->n_edge;
    return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b) {
    if (!b) return LBM_OK;
    {
        DeviceGuard guard(b->device);
        if (b->stream) cudaStreamSynchronize(b->stream);
        batch_free(b);
    }
    delete b;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_ctx* const* members, int32_t n, int64_t steps, lbm_tuning* best,
                              double* best_ms) {
    NvtxRange range_("lbm_batch_autotune");
    if (!members || n < 1 || !best || steps < 1 || steps > 100000) return LBM_E_INVALID;
    for (int i = 0; i < n; ++i)
        if (!members[i] || members[i]->scheme == LBM_SCHEME_EXTRAPOLATED) return LBM_E_INVALID;
    DeviceGuard guard(members[0]->device);
    if (!guard.ok) return LBM_E_INVALID;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    // scratch members: the same shapes and formats, zero fields
    std::vector<lbm_ctx*> scratch;
    lbm_status status = LBM_OK;
    try {
        scratch.assign(size_t(n), nullptr);
    } catch (...) {
        cudaStreamDestroy(st);
        return LBM_E_OOM;
    }
    for (int i = 0; i < n && status == LBM_OK; ++i) {
        const lbm_ctx* c = members[i];
        lbm_desc d;
        memset(&d, 0, sizeof(d));
        d.nx = c->nx;
        d.ny = c->ny;
        d.dX = c->dX;
        d.storage = c->fmt == kFmtF64 ? LBM_F64 : (c->fmt == kFmtF16 ? LBM_F16 : (c->fmt == kFmtBF16 ? LBM_BF16 : LBM_F32));
        d.u_carry = c->fmt == kFmtF32 ? LBM_UCARRY_NATIVE
                    : (c->fmt == kFmtF32H ? LBM_UCARRY_COMPENSATED16 : LBM_UCARRY_COMPENSATED);
        d.scheme = c->scheme;
        d.f16_scale_log2 = c->f16_scale_log2;
        d.cuda_stream = st;
        d.device = c->device;
        status = lbm_create(&d, &scratch[size_t(i)]);
        if (status == LBM_OK) status = lbm_set_material(scratch[size_t(i)], 0.3, 0.3, 1.0, 1.0, nullptr);
        for (int e = 0; e < 4 && status == LBM_OK; ++e)
            status = lbm_set_boundary(scratch[size_t(i)], e, c->bc[e].kind, nullptr, nullptr, nullptr);
        if (status == LBM_OK && c->hole[0] < c->hole[1])  // the same plan: bands around the hole
            status = lbm_set_hole(scratch[size_t(i)], c->hole, c->hole_T);
    }
    // candidates: ring depth x rows per interior tile (0: the default) on the
    // format's default strip grid, then the other two strip grids at the
    // best of those
    const int rings[3] = {4, 5, 6};
    const int chunks[5] = {0, 32, 64, 128, 256};
    const int al0 = batch_default_aligned(members[0]->fmt);
    double best_t = INFINITY;
    lbm_tuning bt = {0, 0, al0, 0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (status == LBM_OK &&
        (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        cudaGetLastError();
        status = LBM_E_CUDA;
    }
    for (int k = 0; k < 3 * 5 + 2 && status == LBM_OK; ++k) {
        {
            lbm_tuning t = {0, 0, al0, 0};
            if (k < 15) {
                t.ring_slots = rings[k / 5];
                t.chunk_rows = chunks[k % 5];
            } else {  // the other strip grids
                t = bt;
                t.aligned = (al0 + 1 + (k - 15)) % 3;
            }
            lbm_batch* b = nullptr;
            status = lbm_batch_create_tuned(scratch.data(), n, st, &t, &b);
            // warm: a plain step and the graphs of both parities
            if (status == LBM_OK) status = lbm_batch_step(b, 2 * kBatchGraphChunk + 2);
            if (status == LBM_OK) status = lbm_batch_sync(b, nullptr);
            double ms = INFINITY;
            if (status == LBM_OK) {
                cudaError_t err = cudaEventRecord(e0, st);
                if (err == cudaSuccess) status = lbm_batch_step(b, steps);
                if (err == cudaSuccess && status == LBM_OK) err = cudaEventRecord(e1, st);
                if (err == cudaSuccess && status == LBM_OK) err = cudaEventSynchronize(e1);
                float f = 0;
                if (err == cudaSuccess && status == LBM_OK && cudaEventElapsedTime(&f, e0, e1) == cudaSuccess)
                    ms = double(f) / double(steps);
                if (err != cudaSuccess) status = LBM_E_CUDA;
            }
            if (b) lbm_batch_destroy(b);
            if (status == LBM_OK && ms < best_t) {
                best_t = ms;
                bt = t;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (lbm_ctx* c : scratch) lbm_destroy(c);
    cudaStreamDestroy(st);
    if (status != LBM_OK) return status;
    if (!(best_t < INFINITY)) return LBM_E_CUDA;
    *best = bt;
    if (best_ms) *best_ms = best_t;
    return LBM_OK;
}

}  // extern "C"

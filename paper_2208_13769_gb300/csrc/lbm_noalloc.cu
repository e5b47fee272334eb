// lbm_noalloc.cu -- diagnostics of caller-owned device fields without any
// allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a CUDA graph
// being captured, inside a memory pool with a fixed budget, or in a process
// whose allocator is owned by another runtime that forbids side allocations.
// lbm_diagnostics_noalloc serves them.  It runs the same two reduction kernels
// as lbm_diagnostics, but their per-CTA partial sums go to a file-scope
// static device array instead of context memory.  The array is part of the
// library image: every GPU that loads the library holds it until the process
// exits, and every call shares it.
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "lbm.h"
#include "lbm_kernels.h"

namespace {

// Partial sums of at most kMaxBlocks CTAs, 8 doubles each (64 KiB); larger
// bodies stride over them.  The reduction uses 32-bit node coordinates.
constexpr int kMaxBlocks = 1024;
constexpr int64_t kNoAllocMaxNodes = LBM_NOALLOC_MAX_NODES;
static __device__ __align__(256) double g_partials[kMaxBlocks * 8];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
// per device: the address of g_partials and the id of the CUDA context it
// belongs to (a device reset destroys the context; the module, and with it
// the array, is loaded afresh, possibly elsewhere, in the next one)
double* g_ptr[kMaxDevices] = {nullptr};
unsigned long long g_ctx[kMaxDevices] = {0};

// The unique id of the calling thread's current CUDA context (0 if there is
// none yet, or if the driver cannot tell), through the driver's entry points
// (no link against the driver library).
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || c == nullptr || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// The device address of g_partials on `device` (which must be current).
// Looked up on the first call in each CUDA context of the device and kept
// for the calls that follow in that context; the host-side name g_partials
// is only a stand-in and must never be handed to a kernel.
cudaError_t partials_address(int device, double** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_ptr[device] || ctx == 0 || ctx != g_ctx[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_ptr[device] = static_cast<double*>(p);
        g_ctx[device] = current_context_id();  // the lookup made the context current if none was
    }
    *out = g_ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_diagnostics_noalloc(const lbm_field_geometry* geo, const double* fields_dev,
                                              double* out_dev, void* cuda_stream) {
    if (!geo || !fields_dev || !out_dev) return LBM_E_INVALID;
    if (geo->nx < 3 || geo->ny < 3 || !(geo->dX > 0) || !(geo->mu > 0) || !(geo->rho0 > 0)) return LBM_E_INVALID;
    const int64_t nodes = int64_t(geo->nx) * geo->ny;
    if (nodes > kNoAllocMaxNodes) return LBM_E_INVALID;  // beyond the stated maximum
    for (int e = 0; e < 4; ++e)
        if (geo->edge_kind[e] < LBM_PERIODIC || geo->edge_kind[e] > LBM_NEUMANN) return LBM_E_INVALID;
    if ((geo->edge_kind[0] == LBM_PERIODIC) != (geo->edge_kind[1] == LBM_PERIODIC) ||
        (geo->edge_kind[2] == LBM_PERIODIC) != (geo->edge_kind[3] == LBM_PERIODIC))
        return LBM_E_INVALID;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return LBM_E_CUDA;
    double* partials = nullptr;
    if (partials_address(device, &partials) != cudaSuccess) return LBM_E_CUDA;

    lbm::ReadoutParams rp;
    memset(&rp, 0, sizeof(rp));
    rp.nx = geo->nx;
    rp.ny = geo->ny;
    rp.periodic_x = geo->edge_kind[0] == LBM_PERIODIC;
    rp.periodic_y = geo->edge_kind[2] == LBM_PERIODIC;
    rp.dX = geo->dX;
    rp.lambda = geo->lambda;
    rp.mu = geo->mu;
    rp.rho0 = geo->rho0;
    rp.t = 0.0;  // the Dirichlet displacements below are already at the fields' time
    rp.fields = fields_dev;
    for (int e = 0; e < 4; ++e) {
        rp.bc[e].kind = geo->edge_kind[e];
        rp.bc[e].value[0] = geo->edge_u[e][0];
        rp.bc[e].value[1] = geo->edge_u[e][1];
    }
    // every CTA overwrites its own partial slot before the final pass reads
    // it, so nothing left by an earlier call needs clearing
    int nblocks = lbm::diagnostics_blocks(nodes);
    if (nblocks > kMaxBlocks) nblocks = kMaxBlocks;
    const cudaError_t e = lbm::launch_diagnostics(rp, partials, nblocks, out_dev, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}

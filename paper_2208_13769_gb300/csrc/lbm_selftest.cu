// lbm_selftest.cu -- exercises, on the device, the give-up path of the
// bounded mbarrier wait that guards every bulk-copy slot of the interior
// kernel, without faulting or hanging anything: a barrier that expects two
// arrivals gets one, so its phase never completes, and the wait must return
// after its poll limit with the CTA (and the context) intact.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"
#include "lbm_pipeline.cuh"

namespace {

__global__ void bounded_wait_kernel(uint32_t limit, int32_t* result) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        lbm::mbar_init(&bar, 2);
        lbm::fence_mbar_init();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(lbm::smem_addr(&bar)) : "memory");
        // one arrival of two: phase 0 stays open; no copy is in flight, so
        // the CTA may leave with the barrier incomplete
        result[0] = lbm::mbar_wait_n(&bar, 0u, limit) ? 0 : 1;
    }
}

}  // namespace

extern "C" lbm_status lbm_selftest_bounded_wait(uint32_t polls, void* cuda_stream, int32_t* timed_out) {
    if (!timed_out || polls == 0 || polls > (1u << 22)) return LBM_E_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int32_t* d = nullptr;
    if (cudaMalloc(&d, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        return LBM_E_OOM;
    }
    cudaError_t e = cudaMemsetAsync(d, 0xff, sizeof(int32_t), s);
    if (e == cudaSuccess) {
        bounded_wait_kernel<<<1, 32, 0, s>>>(polls, d);
        e = cudaGetLastError();
    }
    int32_t h = -1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return LBM_E_CUDA;
    *timed_out = h;
    return LBM_OK;
}

// lbm_fields.cu -- read-out and diagnostics kernels.
//
// Both start from the FP64 fields (u, v, r) the last fused step wrote.  The
// stresses are evaluated from u with the same central differences and ghost
// rules as the step: H = Grad u (Eq. defgrad), P(F) of Sec. 7's neo-Hooke
// energy, Pbar(H) (Eq. Plin), sigma = J^-1 P F^T, and W(F) with ln J.
#include <cuda_runtime.h>
#include <math.h>

#include "lbm_kernels.h"

namespace lbm {

namespace {

__device__ __forceinline__ int wrapc(int g, int n) {
    int w = g % n;
    return w < 0 ? w + n : w;
}

// u_comp(x + dx, y + dy) - u_comp(x - dx, y - dy) for an axis step (dx, dy)
// in {(1,0), (0,1)}, with the ghost rules of bounded edges.
__device__ double du_fd(const ReadoutParams& p, int x, int y, int dx, int dy, int comp) {
    const double* u = p.fields + int64_t(comp) * p.nx * p.ny;
    auto U = [&](int xx, int yy) { return u[int64_t(yy) * p.nx + xx]; };
    // across a face of the hole: the linear ghost 2 u_0 - u_1 from the node
    // and the node behind it
    if (in_hole(p.hole, x + dx, y + dy)) return (2.0 * U(x, y) - U(x - dx, y - dy)) - U(x - dx, y - dy);
    if (in_hole(p.hole, x - dx, y - dy)) return U(x + dx, y + dy) - (2.0 * U(x, y) - U(x + dx, y + dy));
    const int n = dx ? p.nx : p.ny;
    const int k = dx ? x : y;
    const bool per = dx ? p.periodic_x : p.periodic_y;
    if (per || (k > 0 && k < n - 1)) {
        int xp = x + dx, yp = y + dy, xm = x - dx, ym = y - dy;
        if (dx) { xp = wrapc(xp, n); xm = wrapc(xm, n); } else { yp = wrapc(yp, n); ym = wrapc(ym, n); }
        return U(xp, yp) - U(xm, ym);
    }
    const int edge = (dx ? 0 : 2) + (k == 0 ? 0 : 1);
    const EdgeBC& e = p.bc[edge];
    const int s = (k == 0) ? 1 : -1;  // inward step
    const double u0 = U(x, y), u1 = U(x + s * dx, y + s * dy);
    double ghost;
    if (e.kind == kDirichlet)
        ghost = 2.0 * (e.value[comp] + e.rate[comp] * p.t) - u0;
    else
        ghost = 2.0 * u0 - u1;
    return (k == 0) ? (u1 - ghost) : (ghost - u1);
}

struct Local {
    double H[4], P[4], Pb[4], J, W, sig[4];
};

__device__ void local_state(const ReadoutParams& p, int x, int y, Local& L) {
    const double inv2 = 1.0 / (2.0 * p.dX);
    const bool removed = in_hole(p.hole, x, y);  // reads as undeformed
    for (int a = 0; a < 2; ++a) {
        L.H[2 * a] = removed ? 0.0 : du_fd(p, x, y, 1, 0, a) * inv2;
        L.H[2 * a + 1] = removed ? 0.0 : du_fd(p, x, y, 0, 1, a) * inv2;
    }
    const double h11 = L.H[0], h12 = L.H[1], h21 = L.H[2], h22 = L.H[3];
    const double jm1 = h11 + h22 + (h11 * h22 - h12 * h21);
    L.J = 1.0 + jm1;
    const double F[4] = {1.0 + h11, h12, h21, 1.0 + h22};
    const double FiT[4] = {F[3] / L.J, -F[2] / L.J, -F[1] / L.J, F[0] / L.J};
    const double c = 0.5 * p.lambda * jm1 * (2.0 + jm1);
    for (int q = 0; q < 4; ++q) L.P[q] = p.mu * (F[q] - FiT[q]) + c * FiT[q];
    const double tr = h11 + h22;
    L.Pb[0] = -p.mu * (2.0 * h11 + tr);
    L.Pb[1] = -p.mu * (h12 + h21);
    L.Pb[2] = L.Pb[1];
    L.Pb[3] = -p.mu * (2.0 * h22 + tr);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) L.sig[2 * a + b] = (L.P[2 * a] * F[2 * b] + L.P[2 * a + 1] * F[2 * b + 1]) / L.J;
    const double IC = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3];
    const double lnJ = log1p(jm1);
    L.W = 0.5 * p.mu * (IC - 2.0) + 0.25 * p.lambda * jm1 * (2.0 + jm1) - (0.5 * p.lambda + p.mu) * lnJ;
}

__global__ void readout_kernel(const ReadoutParams p, unsigned mask, double* out) {
    const int64_t N = int64_t(p.nx) * p.ny;
    const int64_t id = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (id >= N) return;
    const int x = int(id % p.nx), y = int(id / p.nx);
    const bool need_stress = mask & (4u | 8u | 32u | 64u);
    Local L;
    if (need_stress) local_state(p, x, y, L);
    int64_t off = 0;
    if (mask & 1u) {
        out[off + 2 * id] = p.fields[id];
        out[off + 2 * id + 1] = p.fields[N + id];
        off += 2 * N;
    }
    if (mask & 2u) {
        out[off + 2 * id] = p.fields[2 * N + id];
        out[off + 2 * id + 1] = p.fields[3 * N + id];
        off += 2 * N;
    }
    if (mask & 4u) {
        for (int q = 0; q < 4; ++q) out[off + 4 * id + q] = L.P[q];
        off += 4 * N;
    }
    if (mask & 8u) {
        out[off + 3 * id] = L.Pb[0];
        out[off + 3 * id + 1] = L.Pb[1];
        out[off + 3 * id + 2] = L.Pb[3];
        off += 3 * N;
    }
    if (mask & 16u) {
        out[off + id] = p.fields[4 * N + id];
        off += N;
    }
    if (mask & 32u) {
        out[off + 3 * id] = L.sig[0];
        out[off + 3 * id + 1] = L.sig[1];
        out[off + 3 * id + 2] = L.sig[3];
        off += 3 * N;
    }
    if (mask & 64u) {
        out[off + id] = L.J;
        off += N;
    }
}

constexpr int kDiagThreads = 256;

// Sums over the block in a fixed order: warp shuffles, then warp 0.
__device__ void block_reduce(double v[6], double* smem /* [32][6] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < 6; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_down_sync(0xffffffffu, x, o);
            if (q == 4) x = fmin(x, y);
            else if (q == 5) x = fmax(x, y);
            else x += y;
        }
        if (lane == 0) smem[warp * 6 + q] = x;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        for (int q = 0; q < 6; ++q) {
            double x = lane < nw ? smem[lane * 6 + q] : (q == 4 ? INFINITY : 0.0);
            for (int o = 16; o > 0; o >>= 1) {
                double y = __shfl_down_sync(0xffffffffu, x, o);
                if (q == 4) x = fmin(x, y);
                else if (q == 5) x = fmax(x, y);
                else x += y;
            }
            if (lane == 0) v[q] = x;
        }
    }
}

__global__ void __launch_bounds__(kDiagThreads) diag_partial_kernel(const ReadoutParams p, double* partials) {
    __shared__ double sm[32 * 6];
    const int64_t N = int64_t(p.nx) * p.ny;
    double v[6] = {0.0, 0.0, 0.0, 0.0, INFINITY, 0.0};
    for (int64_t id = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; id < N;
         id += int64_t(gridDim.x) * blockDim.x) {
        const int x = int(id % p.nx), y = int(id / p.nx);
        if (in_hole(p.hole, x, y)) continue;  // not part of the body
        Local L;
        local_state(p, x, y, L);
        const double j0 = p.rho0 * p.fields[2 * N + id], j1 = p.rho0 * p.fields[3 * N + id];
        v[0] += j0;
        v[1] += j1;
        v[2] += (j0 * j0 + j1 * j1) / (2.0 * p.rho0);
        v[3] += L.W;
        v[4] = fmin(v[4], L.J);
        const double chk = p.fields[id] + p.fields[N + id] + j0 + j1 + L.W + L.J;
        if (!isfinite(chk) || !(L.J > 0.0)) v[5] = 1.0;
    }
    block_reduce(v, sm);
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; ++q) partials[int64_t(blockIdx.x) * 8 + q] = v[q];
}

__global__ void __launch_bounds__(kDiagThreads) diag_final_kernel(const double* partials, int nblocks, double* out) {
    __shared__ double sm[32 * 6];
    double v[6] = {0.0, 0.0, 0.0, 0.0, INFINITY, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double* q = partials + int64_t(b) * 8;
        v[0] += q[0];
        v[1] += q[1];
        v[2] += q[2];
        v[3] += q[3];
        v[4] = fmin(v[4], q[4]);
        v[5] = fmax(v[5], q[5]);
    }
    block_reduce(v, sm);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 6; ++q) out[q] = v[q];
        out[6] = 0.0;
        out[7] = 0.0;
    }
}

}  // namespace

cudaError_t launch_readout(const ReadoutParams& rp, unsigned mask, double* out, cudaStream_t s) {
    const int64_t N = int64_t(rp.nx) * rp.ny;
    const int threads = 256;
    const int64_t blocks = (N + threads - 1) / threads;
    readout_kernel<<<unsigned(blocks), threads, 0, s>>>(rp, mask, out);
    return cudaGetLastError();
}

int diagnostics_blocks(int64_t nodes) {
    int64_t b = (nodes + kDiagThreads - 1) / kDiagThreads;
    if (b > 1216) b = 1216;  // 8 CTAs per SM on 152 SMs
    return int(b < 1 ? 1 : b);
}

cudaError_t launch_diagnostics(const ReadoutParams& rp, double* partials, int nblocks, double* out8,
                               cudaStream_t s) {
    diag_partial_kernel<<<nblocks, kDiagThreads, 0, s>>>(rp, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<1, kDiagThreads, 0, s>>>(partials, nblocks, out8);
    return cudaGetLastError();
}

}  // namespace lbm

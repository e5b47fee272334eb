// lbm_pipeline.cuh -- device helpers shared by the fused step kernels:
// bulk-copy and mbarrier wrappers, boundary data, the ghost-rule differences,
// lattice-unit constants and the storage geometry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"

namespace lbm {

namespace {

constexpr uint32_t kSpinLimit = 1u << 22;  // bounded mbarrier polling

__device__ __forceinline__ int wrap_coord(int g, int n) {
    int w = g % n;
    return w < 0 ? w + n : w;
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase did not complete within `limit` polls.
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    return mbar_wait_n(bar, parity, kSpinLimit);
}
// Bulk global -> shared copy; both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// T*(t) of a Neumann edge: T0 outside [t_on, t_off), ramping to T1 over t_ramp.
__device__ __forceinline__ void traction(const EdgeBC& e, double t, double& tx, double& ty) {
    double s;
    if (t < e.times[0] || t >= e.times[2])
        s = 0.0;
    else if (e.times[1] > 0.0)
        s = fmin(1.0, (t - e.times[0]) / e.times[1]);
    else
        s = 1.0;
    tx = e.value[0] + (e.rate[0] - e.value[0]) * s;
    ty = e.value[1] + (e.rate[1] - e.value[1]) * s;
}

// Boundary data of one edge at the collision time of a launch, evaluated once
// per CTA (in FP64, then rounded): the Dirichlet displacement u*(t) and wall
// momentum j*/c in lattice units, the Neumann traction T*(t).
template <class TC, class UT>
struct EdgeNow {
    int kind;
    UT us[2];
    TC jh[2];
    TC T[2];
};

template <class TC, class UT>
__device__ __forceinline__ void edge_now(EdgeNow<TC, UT>& out, const EdgeBC& e, double t, double rho0_over_c) {
    out.kind = e.kind;
    for (int c = 0; c < 2; ++c) {
        out.us[c] = UT::from_double(e.value[c] + e.rate[c] * t);
        out.jh[c] = TC(e.rate[c] * rho0_over_c);
    }
    double tx, ty;
    traction(e, t, tx, ty);
    out.T[0] = TC(tx);
    out.T[1] = TC(ty);
}

// u(+1) - u(-1) along one axis around u0 with the ghost rules of bounded
// edges (Dirichlet: u_g = 2 u*(t) - u0; Neumann: linear extrapolation,
// u_g = 2 u0 - u1).  um, up: neighbours below/above; u1: the inward
// neighbour (read only when a ghost is needed); u2 is not used by these
// rules.
template <class TC, class UT>
__device__ __forceinline__ TC du_axis(const UT& um, const UT& u0, const UT& up, const UT& u1, const UT& u2,
                                      bool ghost_lo, bool ghost_hi, const EdgeNow<TC, UT>& e, int comp) {
    if (!ghost_lo && !ghost_hi) return up.minus(um);
    if (e.kind == kDirichlet) {
        const TC v = u0.minus(e.us[comp]) + u1.minus(e.us[comp]);
        return ghost_hi ? -v : v;
    }
    const TC v = TC(2) * u1.minus(u0);
    return ghost_hi ? -v : v;
}

// Q(+1) - Q(-1) with the linear ghost of bounded edges, Q_g = 2 Q0 - Q1.
template <class TC>
__device__ __forceinline__ TC dq_axis(TC qm, TC q0, TC qp, TC q1, TC q2, bool ghost_lo, bool ghost_hi) {
    if (!ghost_lo && !ghost_hi) return qp - qm;
    const TC v = TC(2) * (q1 - q0);
    return ghost_hi ? -v : v;
}

// Lattice constants of a launch in the arithmetic type, read from the
// host-computed table (no FP64 arithmetic on the device: its FP64 units are
// slow on this part).
template <class TC>
__device__ __forceinline__ TC lat_const(const StepParams& p, int k);
template <>
__device__ __forceinline__ float lat_const<float>(const StepParams& p, int k) {
    return p.lat_f[k];
}
template <>
__device__ __forceinline__ double lat_const<double>(const StepParams& p, int k) {
    return p.lat_d[k];
}

template <class TC>
struct LatConsts {
    TC omega, one_m_omega, force_pref, ku, inv_2dx, sq_scale, sb0, sb1, lam, mu, inv_c2, c_over_rho0,
        rho0_over_c, rho0;
    __device__ __forceinline__ void load(const StepParams& p) {
        omega = lat_const<TC>(p, kLatOmega);
        one_m_omega = lat_const<TC>(p, kLatOneMOmega);
        force_pref = lat_const<TC>(p, kLatForcePref);
        ku = lat_const<TC>(p, kLatKu);
        inv_2dx = lat_const<TC>(p, kLatInv2dX);
        sq_scale = lat_const<TC>(p, kLatSqScale);
        sb0 = lat_const<TC>(p, kLatSb0);
        sb1 = lat_const<TC>(p, kLatSb1);
        lam = lat_const<TC>(p, kLatLambda);
        mu = lat_const<TC>(p, kLatMu);
        inv_c2 = lat_const<TC>(p, kLatInvC2);
        c_over_rho0 = lat_const<TC>(p, kLatCOverRho0);
        rho0_over_c = lat_const<TC>(p, kLatRho0OverC);
        rho0 = lat_const<TC>(p, kLatRho0);
    }
};

// Lattice-unit equilibrium over w_i, even part (r, Pf): used by the
// anti-bounce-back rule.
template <class T>
__device__ __forceinline__ T eq_even(int i, T r, T pxx, T pxy, T pyy) {
    const int e2 = ex(i) * ex(i) + ey(i) * ey(i);
    const T epe = T(ex(i) * ex(i)) * pxx + T(ey(i) * ey(i)) * pyy + T(2 * ex(i) * ey(i)) * pxy;
    const T rterm = (e2 == 0) ? T(2) * r : (e2 == 1 ? T(0.5) * r : -r);
    return rterm + T(1.5) * (T(3) * epe - (pxx + pyy));
}
template <class T>
__device__ __forceinline__ T eq_odd(int i, T a0, T a1) {
    return T(3) * (T(ex(i)) * a0 + T(ey(i)) * a1);
}

// Geometry of the extended state arrays.
struct Geo {
    int nx, ny;
    int64_t pitch, plane;
    bool perx, pery;
    __device__ __forceinline__ int64_t at(int x, int y) const { return int64_t(y + kPadRows) * pitch + x + kPadCols; }
};

// Stores v at (x, y) and at its periodic images (x +/- nx, y +/- ny) inside
// the 3-wide image band.  x in [-1, nx], y in [-1, ny].
template <class T>
__device__ __forceinline__ void store_img(T* base, const Geo& g, int x, int y, T v) {
    base[g.at(x, y)] = v;
    int ix = 0, iy = 0;
    if (g.perx) ix = (x < 3) ? g.nx : (x >= g.nx - 3 ? -g.nx : 0);
    if (g.pery) iy = (y < 3) ? g.ny : (y >= g.ny - 3 ? -g.ny : 0);
    if (ix) base[g.at(x + ix, y)] = v;
    if (iy) base[g.at(x, y + iy)] = v;
    if (ix && iy) base[g.at(x + ix, y + iy)] = v;
    // a periodic axis shorter than 6 nodes has a node in both bands
    if (g.perx && x < 3 && x >= g.nx - 3) {
        base[g.at(x - g.nx, y)] = v;
        if (iy) base[g.at(x - g.nx, y + iy)] = v;
    }
    if (g.pery && y < 3 && y >= g.ny - 3) {
        base[g.at(x, y - g.ny)] = v;
        if (ix) base[g.at(x + ix, y - g.ny)] = v;
        if (g.perx && x < 3 && x >= g.nx - 3) base[g.at(x - g.nx, y - g.ny)] = v;
    }
}

}  // namespace

}  // namespace lbm

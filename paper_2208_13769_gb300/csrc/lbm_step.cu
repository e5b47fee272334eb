// lbm_step.cu -- the fused per-time-step kernel of the Lagrangian LBM
// (Algorithm 1 of arXiv 2208.13769, with the paper's footnote predictor for
// u), and its initialisation variant.
//
// One launch advances the whole body from t_n to t_n+1.  1S at a node needs
// P + Pbar on its 4 neighbours, which need u on a 2-node halo, which needs the
// streamed populations there.  Each CTA owns a strip of W = NT - 4 columns and
// a chunk of rows, and walks the rows as a three-stage pipeline (one thread
// per column):
//   stage A, row a     : pull-stream, first moment, predicted u*   (W + 4 cols)
//   stage B, row a - 2 : H = Grad u*, Q = P(F) + Pbar(H)           (W + 2 cols)
//   stage C, row a - 4 : 1S = rho0 b + Div Q, corrected j and u, equilibrium,
//                        BGK collision with He forcing, store       (W cols)
// u* and Q live in 5-row rolling buffers in shared memory (a ghost rule at a
// bounded edge reaches two rows inward, so each stage lags the previous one
// by two rows).  Only 4 columns of stage A, 2 of stage B and a few warm-up
// rows per chunk are recomputed; every state value crosses HBM once per step
// in each direction (stage C re-reads its row's populations from L1).
//
// Lattice units inside the kernel: m = sum_i e_i f_i, Pf = sum_i e_i e_i f_i,
// s = (dt / c) 1S, jh = j / c, so that the equilibrium (Sec. 5) reads
//   f_i^eq = w_i [ r (2 - 3/2 |e_i|^2) + 3 e_i.jh + 3/2 (3 e_i.Pf.e_i - tr Pf) ]
// and no rounded physical constant enters the lattice dynamics.
//
// State per node (two ping-pong copies):
//   f^col_i (9 planes, storage type; a ghost row/column around the body
//            receives the populations the boundary rules of Sec. 6 send back
//            and the wrapped ones of periodic axes, so the pull never branches);
//   A = u_n + dX/(2 rho0) (jh_n + s_n / 2)   (u-carry, 2 comps);
//   s_n                                      (source carry, 2 comps);
// so that u*_n+1 = A + dX/(2 rho0) m  and  jh_n+1 = m + s_(n+1 or n) / 2.
#include <cuda_runtime.h>

#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_kernels.h"

namespace lbm {

namespace {

constexpr int kDepth = 5;  // rows held by the rolling buffers

// Strip / chunk origin, clamped so that every strip (chunk) is full when the
// axis is at least one strip long; the last one then overlaps its neighbour
// and the overlapping nodes are computed identically by both CTAs.
__device__ __forceinline__ int clamped_origin(int b, int T, int n) {
    const int o = b * T;
    const int last = n - T;
    return last <= 0 ? 0 : (o > last ? last : o);
}

__device__ __forceinline__ int wrap_coord(int g, int n) {
    int w = g % n;
    return w < 0 ? w + n : w;
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

// u(+1) - u(-1) along one axis around u0 with the ghost rules of bounded
// edges (Dirichlet: u_g = 2 u*(t) - u0; Neumann: quadratic extrapolation).
// um, up: neighbours below/above; u1, u2: first and second inward neighbours
// (used only when a ghost is needed).
template <class TC, class UT>
__device__ __forceinline__ TC du_axis(const UT& um, const UT& u0, const UT& up, const UT& u1, const UT& u2,
                                      bool ghost_lo, bool ghost_hi, const EdgeBC& e, int comp, double t) {
    if (!ghost_lo && !ghost_hi) return up.minus(um);
    if (e.kind == kDirichlet) {
        const double us = e.value[comp] + e.rate[comp] * t;
        const TC v = u0.minus_d(us) + u1.minus_d(us);
        return ghost_hi ? -v : v;
    }
    const TC v = TC(3) * u1.minus(u0) - u2.minus(u1);
    return ghost_hi ? -v : v;
}

// Q(+1) - Q(-1) with the quadratic ghost of bounded edges.
template <class TC>
__device__ __forceinline__ TC dq_axis(TC qm, TC q0, TC qp, TC q1, TC q2, bool ghost_lo, bool ghost_hi) {
    if (!ghost_lo && !ghost_hi) return qp - qm;
    const TC v = TC(4) * q1 - TC(3) * q0 - q2;
    return ghost_hi ? -v : v;
}

template <class TC>
struct LatConsts {
    TC omega, force_pref, ku, inv_2dx, sq_scale, sb0, sb1, lam, mu, inv_c2, c_over_rho0, rho0_over_c, rho0;
    __device__ __forceinline__ void load(const StepParams& p) {
        omega = TC(p.omega);
        force_pref = TC(1.0 - 0.5 * p.omega);
        ku = TC(p.dX / (2.0 * p.rho0));
        inv_2dx = TC(1.0 / (2.0 * p.dX));
        sq_scale = TC(p.dt * p.dt / (2.0 * p.dX * p.dX));
        sb0 = TC(p.dt * p.dt / p.dX * p.rho0 * p.body[0]);
        sb1 = TC(p.dt * p.dt / p.dX * p.rho0 * p.body[1]);
        lam = TC(p.lambda);
        mu = TC(p.mu);
        inv_c2 = TC(1.0 / (p.c * p.c));
        c_over_rho0 = TC(p.c / p.rho0);
        rho0_over_c = TC(p.rho0 / p.c);
        rho0 = TC(p.rho0);
    }
};

// Lattice-unit equilibrium over w_i: even part (r, Pf) and odd part (jh).
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

template <int S>
struct Slot {
    static constexpr int v = ((S % kDepth) + kDepth) % kDepth;
};

}  // namespace

template <class TS, class TC, class UT, int NT, int MODE>
__global__ void __launch_bounds__(NT) strip_step_kernel(const __grid_constant__ StepParams p) {
    constexpr int W = NT - 4;  // output columns per strip
    __shared__ UT su[kDepth][2][NT];
    __shared__ TC sq[kDepth][4][NT];
    // initialisation only: r0 and Pbar(Grad u0) / c^2 from stage B to stage C
    __shared__ TC sinit[MODE == 1 ? kDepth : 1][4][MODE == 1 ? NT : 1];

    LatConsts<TC> k;
    k.load(p);
    const int nx = p.nx, ny = p.ny;
    const int t = threadIdx.x;
    const int x0 = clamped_origin(blockIdx.x, W, nx);
    const int y_begin = clamped_origin(blockIdx.y, p.chunk_rows, ny);
    const int y_end = min(ny, y_begin + p.chunk_rows);
    const int64_t pitch = p.pitch, plane = p.plane;
    const bool perx = p.periodic_x != 0, pery = p.periodic_y != 0;
    const TS* __restrict__ fsrc = static_cast<const TS*>(p.f_src);
    TS* __restrict__ fdst = static_cast<TS*>(p.f_dst);
    const TC* __restrict__ s_src = static_cast<const TC*>(p.s_src);
    TC* __restrict__ s_dst = static_cast<TC*>(p.s_dst);

    // time of the collision this launch performs
    int64_t n_now = 0;
    if (MODE == 0) n_now = p.counter[p.parity] + 1;
    if (blockIdx.x == 0 && blockIdx.y == 0 && t == 0) p.counter[p.parity ^ 1] = n_now;
    const double t_now = double(n_now) * p.dt;

    // this thread's column (stage A at every t, stage B at t in [1, NT-2],
    // stage C at t in [2, NT-3])
    const int gx_raw = x0 - 2 + t;
    int gx = gx_raw;
    bool col_ok = true;
    if (gx < 0 || gx >= nx) {
        if (perx) gx = wrap_coord(gx, nx);
        else col_ok = false;
    }
    const bool colB = col_ok && t >= 1 && t <= NT - 2;
    const bool colC = t >= 2 && t <= NT - 3 && gx_raw < nx;
    const bool gxl = !perx && gx == 0, gxh = !perx && gx == nx - 1;
    // inward neighbours in the strip for the x ghost rules
    const int tin1 = gxl ? min(t + 1, NT - 1) : max(t - 1, 0);
    const int tin2 = gxl ? min(t + 2, NT - 1) : max(t - 2, 0);
    const int tm = t > 0 ? t - 1 : t, tp = t < NT - 1 ? t + 1 : t;
    const EdgeBC& ebx = gxl ? p.bc[0] : p.bc[1];
    const int64_t xo = int64_t(gx) + p.xoff;

    bool bad = false;
    const int niter = (y_end - y_begin) + 6;

    auto body = [&](int q, auto slot_tag) {
        constexpr int S = decltype(slot_tag)::value;
        const int a = y_begin - 2 + q;

        // ---------------- stage A: row a in [y_begin - 2, y_end + 1]
        if (a <= y_end + 1) {
            constexpr int sa = Slot<S>::v;
            int gy = a;
            bool ok = col_ok;
            if (gy < 0 || gy >= ny) {
                if (pery) gy = wrap_coord(gy, ny);
                else ok = false;
            }
            if (ok) {
                if (MODE == 0) {
                    const int64_t id = int64_t(gy + 1) * pitch + xo;
                    TC g[9];
#pragma unroll
                    for (int i = 1; i < 9; ++i)
                        g[i] = Codec<TS, TC>::ld(fsrc[i * plane + id - int64_t(ey(i)) * pitch - ex(i)], i, p);
                    const TC m0 = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
                    const TC m1 = (g[2] - g[4]) + (g[5] - g[8]) + (g[6] - g[7]);
                    const UT a0 = UT::load(p.a_src, id, plane);
                    const UT a1 = UT::load(p.a_src, id + UT::planes * plane, plane);
                    su[sa][0][t] = a0.add(k.ku * m0);
                    su[sa][1][t] = a1.add(k.ku * m1);
                } else {
                    const int64_t h = (int64_t(gy) * nx + gx) * 2;
                    su[sa][0][t] = UT::from_double(p.u0 ? p.u0[h] : 0.0);
                    su[sa][1][t] = UT::from_double(p.u0 ? p.u0[h + 1] : 0.0);
                }
            }
        }
        __syncthreads();

        // ---------------- stage B: row m = a - 2 in [y_begin - 1, y_end]
        {
            constexpr int s0 = Slot<S - 2>::v, sp = Slot<S - 1>::v, sp2 = Slot<S>::v;
            constexpr int sm = Slot<S - 3>::v, sm2 = Slot<S - 4>::v;
            const int m = a - 2;
            int gy = m;
            bool ok = colB && m >= y_begin - 1 && m <= y_end;
            if (gy < 0 || gy >= ny) {
                if (pery) gy = wrap_coord(gy, ny);
                else ok = false;
            }
            if (ok) {
                const bool gyl = !pery && gy == 0, gyh = !pery && gy == ny - 1;
                const EdgeBC& eby = gyl ? p.bc[2] : p.bc[3];
                const int r1 = gyl ? sp : sm, r2 = gyl ? sp2 : sm2;
                TC h[2][2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const UT u0 = su[s0][c][t];
                    h[c][0] = du_axis<TC, UT>(su[s0][c][tm], u0, su[s0][c][tp], su[s0][c][tin1], su[s0][c][tin2],
                                              gxl, gxh, ebx, c, t_now) * k.inv_2dx;
                    h[c][1] = du_axis<TC, UT>(su[sm][c][t], u0, su[sp][c][t], su[r1][c][t], su[r2][c][t], gyl, gyh,
                                              eby, c, t_now) * k.inv_2dx;
                }
                TC q11, q12, q21, q22;
                const TC J = stress_remainder<TC>(h[0][0], h[0][1], h[1][0], h[1][1], k.lam, k.mu, q11, q12, q21, q22);
                bad |= !(J > TC(0)) || !(fabs(q11) + fabs(q12) + fabs(q21) + fabs(q22) < TC(1e30));
                sq[s0][0][t] = q11;
                sq[s0][1][t] = q12;
                sq[s0][2][t] = q21;
                sq[s0][3][t] = q22;
                if (MODE == 1) {
                    const TC tr = h[0][0] + h[1][1];
                    sinit[s0 * (MODE == 1)][0][t * (MODE == 1)] = -k.rho0 * tr;
                    sinit[s0 * (MODE == 1)][1][t * (MODE == 1)] = -k.mu * (TC(2) * h[0][0] + tr) * k.inv_c2;
                    sinit[s0 * (MODE == 1)][2][t * (MODE == 1)] = -k.mu * (h[0][1] + h[1][0]) * k.inv_c2;
                    sinit[s0 * (MODE == 1)][3][t * (MODE == 1)] = -k.mu * (TC(2) * h[1][1] + tr) * k.inv_c2;
                }
            }
        }
        __syncthreads();

        // ---------------- stage C: row kr = a - 4 in [y_begin, y_end)
        {
            constexpr int qs0 = Slot<S - 4>::v, qsp = Slot<S - 3>::v, qsp2 = Slot<S - 2>::v;
            constexpr int qsm = Slot<S - 5>::v, qsm2 = Slot<S - 6>::v;
            const int kr = a - 4;
            if (colC && kr >= y_begin && kr < y_end) {
                const int gy = kr;
                const bool gyl = !pery && gy == 0, gyh = !pery && gy == ny - 1;
                const int64_t id = int64_t(gy + 1) * pitch + xo;
                TC f[9];
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    f[i] = Codec<TS, TC>::ld(fsrc[i * plane + id - int64_t(ey(i)) * pitch - ex(i)], i, p);

                // s = (dt / c) 1S, 1S = rho0 b + Div(P + Pbar)   (Eq. source1)
                const int r1 = gyl ? qsp : qsm, r2 = gyl ? qsp2 : qsm2;
                TC dQ[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if ((c & 1) == 0)  // Q_a1: derivative along x
                        dQ[c] = dq_axis<TC>(sq[qs0][c][tm], sq[qs0][c][t], sq[qs0][c][tp], sq[qs0][c][tin1],
                                            sq[qs0][c][tin2], gxl, gxh);
                    else  // Q_a2: derivative along y
                        dQ[c] = dq_axis<TC>(sq[qsm][c][t], sq[qs0][c][t], sq[qsp][c][t], sq[r1][c][t],
                                            sq[r2][c][t], gyl, gyh);
                }
                const TC sn0 = k.sb0 + k.sq_scale * (dQ[0] + dQ[1]);
                const TC sn1 = k.sb1 + k.sq_scale * (dQ[2] + dQ[3]);

                TC r, j0, j1, pxx, pxy, pyy;
                UT ux = su[Slot<S - 4>::v][0][t], uy = su[Slot<S - 4>::v][1][t];
                if (MODE == 0) {
                    r = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
                    const TC m0 = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
                    const TC m1 = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
                    const TC dg = (f[5] + f[6]) + (f[7] + f[8]);
                    pxx = (f[1] + f[3]) + dg;
                    pyy = (f[2] + f[4]) + dg;
                    pxy = (f[5] - f[6]) + (f[7] - f[8]);
                    const TC so0 = s_src[id], so1 = s_src[id + plane];
                    if (p.scheme == 1) {
                        j0 = m0 + TC(0.5) * sn0;
                        j1 = m1 + TC(0.5) * sn1;
                        ux = ux.add(k.ku * (TC(0.5) * (sn0 - so0)));
                        uy = uy.add(k.ku * (TC(0.5) * (sn1 - so1)));
                    } else {
                        j0 = m0 + TC(0.5) * so0;
                        j1 = m1 + TC(0.5) * so1;
                    }
                } else {
                    // initialisation of Algorithm 1: r = -rho0 Div u0,
                    // j = rho0 v0, Pbar = Pbar(Grad u0) (from stage B)
                    constexpr int si = Slot<S - 4>::v;
                    r = sinit[si * (MODE == 1)][0][t * (MODE == 1)];
                    pxx = sinit[si * (MODE == 1)][1][t * (MODE == 1)];
                    pxy = sinit[si * (MODE == 1)][2][t * (MODE == 1)];
                    pyy = sinit[si * (MODE == 1)][3][t * (MODE == 1)];
                    const int64_t hh = (int64_t(gy) * nx + gx) * 2;
                    j0 = k.rho0_over_c * TC(p.v0 ? p.v0[hh] : 0.0);
                    j1 = k.rho0_over_c * TC(p.v0 ? p.v0[hh + 1] : 0.0);
                }

                // equilibrium (Sec. 5), source populations (Eq. source), BGK
                // collision with He forcing (Eq. col)
                TC fc[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const TC w = wgt<TC>(i);
                    const TC feq = w * (eq_even<TC>(i, r, pxx, pxy, pyy) + eq_odd<TC>(i, j0, j1));
                    const TC fi = (MODE == 0) ? f[i] : feq;
                    fc[i] = fi - k.omega * (fi - feq) + k.force_pref * w * eq_odd<TC>(i, sn0, sn1);
                    fdst[i * plane + id] = Codec<TS, TC>::st(fc[i], i, p);
                }

                // links that leave the body: boundary rules of Sec. 6, or the
                // periodic wrap, into the ghost layer of the destination
                if (gx == 0 || gx == nx - 1 || gy == 0 || gy == ny - 1) {
                    const TC q11 = sq[qs0][0][t], q12 = sq[qs0][1][t], q21 = sq[qs0][2][t], q22 = sq[qs0][3][t];
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        const int dx = gx + ex(i), dy = gy + ey(i);
                        const bool cx = dx < 0 || dx >= nx, cy = dy < 0 || dy >= ny;
                        if (!cx && !cy) continue;
                        const bool bx = cx && !perx, by = cy && !pery;
                        if (!bx && !by) {
                            // periodic: the puller at wrap(D) reads wrap(D) - e_i
                            const int wx = cx ? wrap_coord(dx, nx) : dx;
                            const int wy = cy ? wrap_coord(dy, ny) : dy;
                            fdst[i * plane + int64_t(wy - ey(i) + 1) * pitch + (wx - ex(i)) + p.xoff] =
                                Codec<TS, TC>::st(fc[i], i, p);
                            continue;
                        }
                        const int oi = opp(i);
                        const EdgeBC* ea = bx ? &p.bc[dx < 0 ? 0 : 1] : nullptr;
                        const EdgeBC* eb = by ? &p.bc[dy < 0 ? 2 : 3] : nullptr;
                        int nd = 0;
                        double js0 = 0.0, js1 = 0.0;
                        if (ea && ea->kind == kDirichlet) {
                            js0 += ea->rate[0];
                            js1 += ea->rate[1];
                            ++nd;
                        }
                        if (eb && eb->kind == kDirichlet) {
                            js0 += eb->rate[0];
                            js1 += eb->rate[1];
                            ++nd;
                        }
                        TC val;
                        if (nd > 0) {
                            // Eq. (bbcon): jh* = rho0 v* / c
                            const TC a0 = TC(js0 / nd) * k.rho0_over_c, a1 = TC(js1 / nd) * k.rho0_over_c;
                            val = fc[i] - TC(2) * wgt<TC>(i) * eq_odd<TC>(i, a0, a1);
                        } else {
                            // Eq. (abbcon) with Pbar* of Sec. 6 in the wall-normal frame
                            const int sx = bx ? (dx < 0 ? -1 : 1) : 0, sy = by ? (dy < 0 ? -1 : 1) : 0;
                            const double inv_len = (sx != 0 && sy != 0) ? 0.70710678118654752440 : 1.0;
                            double T0 = 0.0, T1 = 0.0;
                            if (ea) {
                                double ta, tb;
                                traction(*ea, t_now, ta, tb);
                                T0 += ta;
                                T1 += tb;
                            }
                            if (eb) {
                                double ta, tb;
                                traction(*eb, t_now, ta, tb);
                                T0 += ta;
                                T1 += tb;
                            }
                            const TC N0 = TC(sx * inv_len), N1 = TC(sy * inv_len);
                            const TC g0 = -TC(T0 * inv_len) + q11 * N0 + q12 * N1;
                            const TC g1 = -TC(T1 * inv_len) + q21 * N0 + q22 * N1;
                            const TC t0 = -N1, t1 = N0;
                            const TC pnn = (N0 * g0 + N1 * g1) * k.inv_c2;
                            const TC pnt = (t0 * g0 + t1 * g1) * k.inv_c2;
                            const TC ptt = t0 * t0 * pxx + TC(2) * t0 * t1 * pxy + t1 * t1 * pyy;
                            const TC sxx = pnn * N0 * N0 + TC(2) * pnt * N0 * t0 + ptt * t0 * t0;
                            const TC syy = pnn * N1 * N1 + TC(2) * pnt * N1 * t1 + ptt * t1 * t1;
                            const TC sxy = pnn * N0 * N1 + pnt * (N0 * t1 + t0 * N1) + ptt * t0 * t1;
                            val = -fc[i] + TC(2) * wgt<TC>(i) * eq_even<TC>(i, r, sxx, sxy, syy);
                        }
                        fdst[oi * plane + int64_t(dy + 1) * pitch + dx + p.xoff] = Codec<TS, TC>::st(val, oi, p);
                    }
                }

                // carries for the next step
                const UT A0 = ux.add(k.ku * (j0 + TC(0.5) * sn0));
                const UT A1 = uy.add(k.ku * (j1 + TC(0.5) * sn1));
                A0.store(p.a_dst, id, plane);
                A1.store(p.a_dst, id + UT::planes * plane, plane);
                s_dst[id] = sn0;
                s_dst[id + plane] = sn1;
                if (p.fields != nullptr) {
                    const int64_t o = int64_t(gy) * nx + gx;
                    const int64_t np = int64_t(nx) * ny;
                    p.fields[o] = ux.to_double();
                    p.fields[np + o] = uy.to_double();
                    p.fields[2 * np + o] = double(j0 * k.c_over_rho0);
                    p.fields[3 * np + o] = double(j1 * k.c_over_rho0);
                    p.fields[4 * np + o] = double(r);
                    if (!(fabs(double(j0)) + fabs(double(j1)) < 1e300)) bad = true;
                }
            }
        }
    };

    for (int q = 0; q < niter; q += kDepth) {
        body(q, std::integral_constant<int, 0>{});
        if (q + 1 < niter) body(q + 1, std::integral_constant<int, 1>{});
        if (q + 2 < niter) body(q + 2, std::integral_constant<int, 2>{});
        if (q + 3 < niter) body(q + 3, std::integral_constant<int, 3>{});
        if (q + 4 < niter) body(q + 4, std::integral_constant<int, 4>{});
    }
    if (bad) atomicOr(p.flag, 1);
}

// ---------------------------------------------------------------- launchers

template <class TS, class TC, class UT, int NT, int MODE>
cudaError_t launch_one(const StepParams& p, cudaStream_t s) {
    dim3 grid(p.tiles_x, p.tiles_y);
    strip_step_kernel<TS, TC, UT, NT, MODE><<<grid, NT, 0, s>>>(p);
    return cudaGetLastError();
}

// `fields` selects at run time whether the launch also writes u, v, r (the
// same instantiation runs either way, so results are bit-identical).
template <class TS, class TC, class UT, int NT>
struct Variant {
    static constexpr int width = NT - 4;
    static cudaError_t run(const StepParams& p0, cudaStream_t s, int mode, bool fields) {
        StepParams p = p0;
        if (!fields) p.fields = nullptr;
        return mode == 1 ? launch_one<TS, TC, UT, NT, 1>(p, s) : launch_one<TS, TC, UT, NT, 0>(p, s);
    }
};

using V64 = Variant<double, double, UPlain<double>, 128>;
using V32 = Variant<float, float, UPlain<float>, 128>;
using V32c = Variant<float, float, UComp, 128>;
using V16 = Variant<__half, float, UComp, 128>;
using Vb16 = Variant<__nv_bfloat16, float, UComp, 128>;

void tile_shape(int fmt, int* tx, int* ty) {
    switch (fmt) {
        case kFmtF64: *tx = V64::width; break;
        case kFmtF32: *tx = V32::width; break;
        case kFmtF32C: *tx = V32c::width; break;
        case kFmtF16: *tx = V16::width; break;
        default: *tx = Vb16::width; break;
    }
    *ty = 128;
}

cudaError_t launch_fused_step(int fmt, const StepParams& p, cudaStream_t s, int mode, bool fields) {
    switch (fmt) {
        case kFmtF64: return V64::run(p, s, mode, fields);
        case kFmtF32: return V32::run(p, s, mode, fields);
        case kFmtF32C: return V32c::run(p, s, mode, fields);
        case kFmtF16: return V16::run(p, s, mode, fields);
        case kFmtBF16: return Vb16::run(p, s, mode, fields);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm

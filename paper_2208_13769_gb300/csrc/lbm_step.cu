// lbm_step.cu -- the fused per-time-step kernel of the Lagrangian LBM
// (Algorithm 1 of arXiv 2208.13769, with the paper's footnote predictor for
// u), and its initialisation variant.
//
// One launch advances the whole body from t_n to t_n+1.  Each CTA owns a
// TX x TY tile.  Because 1S at a node needs P + Pbar on its 4 neighbours,
// which need u on a 2-node halo, which needs the streamed populations there,
// a CTA recomputes the cheap part of the step (pull-stream, first moment,
// predicted u) on the tile plus a 2-node ring, keeps u in shared memory,
// evaluates H, P and Pbar on the tile plus a 1-node ring, and then finishes
// its own nodes: 1S, corrected j and u, equilibrium, collision, store.
// The ring costs only L2 traffic; every state value crosses HBM once per
// step in each direction.
//
// State per node (two ping-pong copies):
//   f^col_i (9 planes, storage type; one ghost row/column around the body
//            that receives the populations the boundary rules of Sec. 6
//            send back, and the wrapped ones of periodic axes, so the pull
//            is branch-free);
//   A = u_n + dt/(2 rho0) (j_n + dt/2 1S_n)   (u-carry, 2 comps);
//   1S_n                                      (source carry, 2 comps);
// so that u*_n+1 = A + dt/(2 rho0) sum_i C_i f_i  and
//         j_n+1  = sum_i C_i f_i + dt/2 1S_(n+1 or n).
#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_kernels.h"

namespace lbm {

namespace {

// Tile origin, clamped so that every tile is full when the axis is at least
// one tile long (the last tile then overlaps its neighbour; overlapping nodes
// are computed identically by both CTAs).
__device__ __forceinline__ int tile_origin(int b, int T, int n) {
    int o = b * T;
    int last = n - T;
    return (last > 0 && o > last) ? last : (last <= 0 ? 0 : o);
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

// Difference u(right) - u(left) along one axis for the node at R2-local
// index `at`, with the ghost rules of bounded edges (Dirichlet: u_g = 2u* - u;
// Neumann: quadratic extrapolation).  `stride` steps one node along the axis
// in shared memory.  ghost_hi/lo: the neighbour lies beyond a bounded edge.
template <class TC, class UT>
__device__ __forceinline__ TC du_axis(const UT* su, int at, int stride, bool ghost_lo, bool ghost_hi,
                                      const EdgeBC& e_lo, const EdgeBC& e_hi, int comp, double t) {
    const UT u0 = su[at];
    if (!ghost_lo && !ghost_hi) return su[at + stride].minus(su[at - stride]);
    if (ghost_hi) {
        const UT u1 = su[at - stride];
        if (e_hi.kind == kDirichlet) {
            double us = e_hi.value[comp] + e_hi.rate[comp] * t;
            return -(u0.minus_d(us) + u1.minus_d(us));
        }
        const UT u2 = su[at - 2 * stride];
        return TC(3) * u0.minus(u1) - u1.minus(u2);
    }
    const UT u1 = su[at + stride];
    if (e_lo.kind == kDirichlet) {
        double us = e_lo.value[comp] + e_lo.rate[comp] * t;
        return u1.minus_d(us) + u0.minus_d(us);
    }
    const UT u2 = su[at + 2 * stride];
    return TC(3) * u1.minus(u0) - u2.minus(u1);
}

// Difference Q(right) - Q(left) with the quadratic ghost of bounded edges.
template <class TC>
__device__ __forceinline__ TC dq_axis(const TC* q, int at, int stride, bool ghost_lo, bool ghost_hi) {
    if (!ghost_lo && !ghost_hi) return q[at + stride] - q[at - stride];
    if (ghost_hi) return TC(3) * q[at] - TC(4) * q[at - stride] + q[at - 2 * stride];
    return -TC(3) * q[at] + TC(4) * q[at + stride] - q[at + 2 * stride];
}

}  // namespace

template <class TS, class TC, class UT, int TX, int TY, int NT, int MODE, bool FIELDS>
__global__ void __launch_bounds__(NT) fused_step_kernel(const StepParams p) {
    constexpr int R2X = TX + 4, R2Y = TY + 4, R1X = TX + 2, R1Y = TY + 2;
    constexpr int NPT = (TX * TY) / NT;
    static_assert(NPT * NT == TX * TY, "tile must be a multiple of the block size");
    constexpr int RING = R2X * R2Y - TX * TY;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    UT* su = reinterpret_cast<UT*>(smem_raw);                    // [2][R2Y][R2X]
    TC* sq = reinterpret_cast<TC*>(smem_raw + sizeof(UT) * 2 * R2X * R2Y);  // [4][R1Y][R1X]

    Consts<TC> k;
    k.load(p);
    const int nx = p.nx, ny = p.ny;
    const int x0 = tile_origin(blockIdx.x, TX, nx);
    const int y0 = tile_origin(blockIdx.y, TY, ny);
    const int64_t pitch = p.pitch, plane = p.plane;
    const int xoff = p.xoff;
    const bool perx = p.periodic_x != 0, pery = p.periodic_y != 0;
    const TS* __restrict__ fsrc = static_cast<const TS*>(p.f_src);
    TS* __restrict__ fdst = static_cast<TS*>(p.f_dst);

    // time of the collision this launch performs
    int64_t n_now = 0;
    if (MODE == 0) {
        n_now = p.counter[p.parity] + 1;
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) p.counter[p.parity ^ 1] = n_now;
    } else {
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) p.counter[p.parity ^ 1] = 0;
    }
    const double t_now = double(n_now) * p.dt;

    auto gidx = [&](int x, int y) -> int64_t { return int64_t(y + 1) * pitch + x + xoff; };

    // ------------------------------------------------ phase 1: u* on the tile + 2 ring
    // u* (or u0 at initialisation) of a node that is not one of this CTA's
    // own: pull only the 8 moving populations for the first moment.
    auto fill_u = [&](int s2, int gx, int gy) {
        if (MODE == 0) {
            const int64_t id = gidx(gx, gy);
            TC m0 = TC(0), m1 = TC(0);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                TC fi = Codec<TS, TC>::ld(fsrc[i * plane + id - int64_t(ey(i)) * pitch - ex(i)], i, p);
                m0 += TC(ex(i)) * fi;
                m1 += TC(ey(i)) * fi;
            }
            UT a0 = UT::load(p.a_src, id, plane);
            UT a1 = UT::load(p.a_src, id + UT::planes * plane, plane);
            su[s2] = a0.add(k.k_u * (k.c * m0));
            su[R2X * R2Y + s2] = a1.add(k.k_u * (k.c * m1));
        } else {
            const int64_t h = (int64_t(gy) * nx + gx) * 2;
            su[s2] = UT::from_double(p.u0 ? p.u0[h] : 0.0);
            su[R2X * R2Y + s2] = UT::from_double(p.u0 ? p.u0[h + 1] : 0.0);
        }
    };
    // maps a halo coordinate to the body (periodic wrap); false if outside
    auto to_body = [&](int& gx, int& gy) -> bool {
        if (gx < 0 || gx >= nx) {
            if (!perx) return false;
            gx = wrap_coord(gx, nx);
        }
        if (gy < 0 || gy >= ny) {
            if (!pery) return false;
            gy = wrap_coord(gy, ny);
        }
        return true;
    };

    TC f[NPT][9];
#pragma unroll
    for (int kk = 0; kk < NPT; ++kk) {
        const int q = threadIdx.x + kk * NT;
        const int lx = q % TX, ly = q / TX;
        int gx = x0 + lx, gy = y0 + ly;
        const int s2 = (ly + 2) * R2X + (lx + 2);
        if (gx < nx && gy < ny) {
            if (MODE == 0) {
                const int64_t id = gidx(gx, gy);
                TC m0 = TC(0), m1 = TC(0);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    f[kk][i] = Codec<TS, TC>::ld(fsrc[i * plane + id - int64_t(ey(i)) * pitch - ex(i)], i, p);
                    m0 += TC(ex(i)) * f[kk][i];
                    m1 += TC(ey(i)) * f[kk][i];
                }
                UT a0 = UT::load(p.a_src, id, plane);
                UT a1 = UT::load(p.a_src, id + UT::planes * plane, plane);
                su[s2] = a0.add(k.k_u * (k.c * m0));
                su[R2X * R2Y + s2] = a1.add(k.k_u * (k.c * m1));
            } else {
                fill_u(s2, gx, gy);
            }
        } else if (to_body(gx, gy)) {
            // a periodic axis shorter than the tile: the position holds an image
            fill_u(s2, gx, gy);
        }
    }
    for (int q = threadIdx.x; q < RING; q += NT) {
        // ring enumeration: 2 top rows, 2 bottom rows, then 2 + 2 side columns
        int lx2, ly2;
        if (q < 2 * R2X) {
            lx2 = q % R2X;
            ly2 = q / R2X;
        } else if (q < 4 * R2X) {
            lx2 = (q - 2 * R2X) % R2X;
            ly2 = R2Y - 2 + (q - 2 * R2X) / R2X;
        } else {
            const int r = q - 4 * R2X;
            ly2 = 2 + r / 4;
            const int c = r % 4;
            lx2 = c < 2 ? c : TX + c;
        }
        int gx = x0 - 2 + lx2, gy = y0 - 2 + ly2;
        if (to_body(gx, gy)) fill_u(ly2 * R2X + lx2, gx, gy);
    }
    __syncthreads();

    // ------------------------------------------------ phase 2a: Q = P + Pbar on tile + 1 ring
    const EdgeBC& bxl = p.bc[0];
    const EdgeBC& bxh = p.bc[1];
    const EdgeBC& byl = p.bc[2];
    const EdgeBC& byh = p.bc[3];
    bool bad = false;
    for (int q = threadIdx.x; q < R1X * R1Y; q += NT) {
        const int l1x = q % R1X, l1y = q / R1X;
        int gx = x0 - 1 + l1x, gy = y0 - 1 + l1y;
        if (!perx && (gx < 0 || gx >= nx)) continue;
        if (!pery && (gy < 0 || gy >= ny)) continue;
        if (perx) gx = wrap_coord(gx, nx);
        if (pery) gy = wrap_coord(gy, ny);
        const int s2 = (l1y + 1) * R2X + (l1x + 1);
        const bool gxl = !perx && gx == 0, gxh = !perx && gx == nx - 1;
        const bool gyl = !pery && gy == 0, gyh = !pery && gy == ny - 1;
        TC h11 = du_axis<TC, UT>(su, s2, 1, gxl, gxh, bxl, bxh, 0, t_now) * k.inv_2dx;
        TC h21 = du_axis<TC, UT>(su + R2X * R2Y, s2, 1, gxl, gxh, bxl, bxh, 1, t_now) * k.inv_2dx;
        TC h12 = du_axis<TC, UT>(su, s2, R2X, gyl, gyh, byl, byh, 0, t_now) * k.inv_2dx;
        TC h22 = du_axis<TC, UT>(su + R2X * R2Y, s2, R2X, gyl, gyh, byl, byh, 1, t_now) * k.inv_2dx;
        TC p11, p12, p21, p22;
        TC J = piola<TC>(h11, h12, h21, h22, k.lam, k.mu, p11, p12, p21, p22);
        bad |= !(J > TC(0)) || !(fabs(p11) + fabs(p12) + fabs(p21) + fabs(p22) < TC(1e30));
        const TC tr = h11 + h22;
        sq[0 * R1X * R1Y + q] = p11 - k.mu * (TC(2) * h11 + tr);
        sq[1 * R1X * R1Y + q] = p12 - k.mu * (h12 + h21);
        sq[2 * R1X * R1Y + q] = p21 - k.mu * (h12 + h21);
        sq[3 * R1X * R1Y + q] = p22 - k.mu * (TC(2) * h22 + tr);
    }
    if (bad) atomicOr(p.flag, 1);
    __syncthreads();

    // ------------------------------------------------ phase 2b: own nodes
    const TC* __restrict__ sfrc = static_cast<const TC*>(p.s_src);
    TC* __restrict__ sdst = static_cast<TC*>(p.s_dst);
#pragma unroll
    for (int kk = 0; kk < NPT; ++kk) {
        const int q = threadIdx.x + kk * NT;
        const int lx = q % TX, ly = q / TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (!(gx < nx && gy < ny)) continue;
        const int64_t id = gidx(gx, gy);
        const int s1 = (ly + 1) * R1X + (lx + 1);
        const int s2 = (ly + 2) * R2X + (lx + 2);
        const bool gxl = !perx && gx == 0, gxh = !perx && gx == nx - 1;
        const bool gyl = !pery && gy == 0, gyh = !pery && gy == ny - 1;

        // 1S(t_now) = rho0 b + Div(P + Pbar)  (Eq. source1)
        const int R1 = R1X * R1Y;
        TC S0 = k.rho0 * k.b0 + (dq_axis<TC>(sq, s1, 1, gxl, gxh) + dq_axis<TC>(sq + R1, s1, R1X, gyl, gyh)) * k.inv_2dx;
        TC S1 = k.rho0 * k.b1 + (dq_axis<TC>(sq + 2 * R1, s1, 1, gxl, gxh) + dq_axis<TC>(sq + 3 * R1, s1, R1X, gyl, gyh)) * k.inv_2dx;

        TC r, j0, j1, pxx, pxy, pyy;
        UT u0 = su[s2], u1 = su[R2X * R2Y + s2];
        if (MODE == 0) {
            TC m0 = TC(0), m1 = TC(0);
            r = TC(0);
            pxx = TC(0);
            pxy = TC(0);
            pyy = TC(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                r += f[kk][i];
                m0 += TC(ex(i)) * f[kk][i];
                m1 += TC(ey(i)) * f[kk][i];
                pxx += TC(ex(i) * ex(i)) * f[kk][i];
                pyy += TC(ey(i) * ey(i)) * f[kk][i];
                pxy += TC(ex(i) * ey(i)) * f[kk][i];
            }
            m0 *= k.c;
            m1 *= k.c;
            const TC c2 = k.c * k.c;
            pxx *= c2;
            pyy *= c2;
            pxy *= c2;
            const TC sOld0 = sfrc[id], sOld1 = sfrc[id + plane];
            if (p.scheme == 1) {
                j0 = m0 + k.half_dt * S0;
                j1 = m1 + k.half_dt * S1;
                u0 = u0.add(k.k_u * k.half_dt * (S0 - sOld0));
                u1 = u1.add(k.k_u * k.half_dt * (S1 - sOld1));
            } else {
                j0 = m0 + k.half_dt * sOld0;
                j1 = m1 + k.half_dt * sOld1;
            }
        } else {
            // initialisation of Algorithm 1 from u0, v0
            TC h11 = du_axis<TC, UT>(su, s2, 1, gxl, gxh, bxl, bxh, 0, 0.0) * k.inv_2dx;
            TC h21 = du_axis<TC, UT>(su + R2X * R2Y, s2, 1, gxl, gxh, bxl, bxh, 1, 0.0) * k.inv_2dx;
            TC h12 = du_axis<TC, UT>(su, s2, R2X, gyl, gyh, byl, byh, 0, 0.0) * k.inv_2dx;
            TC h22 = du_axis<TC, UT>(su + R2X * R2Y, s2, R2X, gyl, gyh, byl, byh, 1, 0.0) * k.inv_2dx;
            const TC tr = h11 + h22;
            r = -k.rho0 * tr;
            pxx = -k.mu * (TC(2) * h11 + tr);
            pyy = -k.mu * (TC(2) * h22 + tr);
            pxy = -k.mu * (h12 + h21);
            const int64_t h = (int64_t(gy) * nx + gx) * 2;
            j0 = k.rho0 * TC(p.v0 ? p.v0[h] : 0.0);
            j1 = k.rho0 * TC(p.v0 ? p.v0[h + 1] : 0.0);
        }

        // equilibrium (Sec. 5), source populations (Eq. source), collision (Eq. col)
        TC fc[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const TC w = wgt<TC>(i);
            const TC feq = w * (feq_even_over_w<TC>(i, r, pxx, pxy, pyy, k.inv_cs2) +
                                feq_odd_over_w<TC>(i, j0, j1, k.inv_c));
            const TC psi = w * feq_odd_over_w<TC>(i, S0, S1, k.inv_c);
            const TC fi = (MODE == 0) ? f[kk][i] : feq;
            fc[i] = fi - k.omega * (fi - feq) + k.force_pref * psi;
            fdst[i * plane + id] = Codec<TS, TC>::st(fc[i], i, p);
        }

        // links that leave the body: boundary rules or periodic wrap into the
        // ghost layer of the destination buffer
        const bool edge = gx == 0 || gx == nx - 1 || gy == 0 || gy == ny - 1;
        if (edge) {
            const TC q11 = sq[s1], q12 = sq[R1 + s1], q21 = sq[2 * R1 + s1], q22 = sq[3 * R1 + s1];
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                int dx = gx + ex(i), dy = gy + ey(i);
                const bool cx = dx < 0 || dx >= nx, cy = dy < 0 || dy >= ny;
                if (!cx && !cy) continue;
                const bool bx = cx && !perx, by = cy && !pery;
                if (!bx && !by) {
                    // periodic wrap: the puller at wrap(D) reads wrap(D) - e_i
                    int wx = cx ? wrap_coord(dx, nx) : dx;
                    int wy = cy ? wrap_coord(dy, ny) : dy;
                    fdst[i * plane + gidx(wx - ex(i), wy - ey(i))] = Codec<TS, TC>::st(fc[i], i, p);
                    continue;
                }
                const int oi = opp(i);
                const EdgeBC* ea = bx ? &p.bc[dx < 0 ? 0 : 1] : nullptr;
                const EdgeBC* eb = by ? &p.bc[dy < 0 ? 2 : 3] : nullptr;
                int nd = 0;
                double js0 = 0.0, js1 = 0.0;
                if (ea && ea->kind == kDirichlet) {
                    js0 += p.rho0 * ea->rate[0];
                    js1 += p.rho0 * ea->rate[1];
                    ++nd;
                }
                if (eb && eb->kind == kDirichlet) {
                    js0 += p.rho0 * eb->rate[0];
                    js1 += p.rho0 * eb->rate[1];
                    ++nd;
                }
                TC val;
                if (nd > 0) {
                    // Eq. (bbcon)
                    const TC a0 = TC(js0 / nd), a1 = TC(js1 / nd);
                    val = fc[i] - TC(2) * wgt<TC>(i) * feq_odd_over_w<TC>(i, a0, a1, k.inv_c);
                } else {
                    // Eq. (abbcon) with Pbar* of Sec. 6 in the wall-normal frame
                    const int sx = bx ? (dx < 0 ? -1 : 1) : 0, sy = by ? (dy < 0 ? -1 : 1) : 0;
                    const double inv_len = (sx != 0 && sy != 0) ? 0.70710678118654752440 : 1.0;
                    double T0 = 0.0, T1 = 0.0;
                    if (ea) {
                        double a, b;
                        traction(*ea, t_now, a, b);
                        T0 += a;
                        T1 += b;
                    }
                    if (eb) {
                        double a, b;
                        traction(*eb, t_now, a, b);
                        T0 += a;
                        T1 += b;
                    }
                    const TC N0 = TC(sx * inv_len), N1 = TC(sy * inv_len);
                    const TC g0 = -TC(T0 * inv_len) + q11 * N0 + q12 * N1;
                    const TC g1 = -TC(T1 * inv_len) + q21 * N0 + q22 * N1;
                    const TC t0 = -N1, t1 = N0;
                    const TC pnn = N0 * g0 + N1 * g1;
                    const TC pnt = t0 * g0 + t1 * g1;
                    const TC ptt = t0 * t0 * pxx + TC(2) * t0 * t1 * pxy + t1 * t1 * pyy;
                    const TC sxx = pnn * N0 * N0 + TC(2) * pnt * N0 * t0 + ptt * t0 * t0;
                    const TC syy = pnn * N1 * N1 + TC(2) * pnt * N1 * t1 + ptt * t1 * t1;
                    const TC sxy = pnn * N0 * N1 + pnt * (N0 * t1 + t0 * N1) + ptt * t0 * t1;
                    val = -fc[i] + TC(2) * wgt<TC>(i) * feq_even_over_w<TC>(i, r, sxx, sxy, syy, k.inv_cs2);
                }
                fdst[oi * plane + gidx(dx, dy)] = Codec<TS, TC>::st(val, oi, p);
            }
        }

        // carries for the next step
        UT A0 = u0.add(k.k_u * (j0 + k.half_dt * S0));
        UT A1 = u1.add(k.k_u * (j1 + k.half_dt * S1));
        A0.store(p.a_dst, id, plane);
        A1.store(p.a_dst, id + UT::planes * plane, plane);
        sdst[id] = S0;
        sdst[id + plane] = S1;
        if (FIELDS) {
            const int64_t o = int64_t(gy) * nx + gx;
            const int64_t np = int64_t(nx) * ny;
            p.fields[o] = u0.to_double();
            p.fields[np + o] = u1.to_double();
            p.fields[2 * np + o] = double(j0 * k.inv_rho0);
            p.fields[3 * np + o] = double(j1 * k.inv_rho0);
            p.fields[4 * np + o] = double(r);
            if (!(fabs(double(j0)) + fabs(double(j1)) < 1e300)) atomicOr(p.flag, 1);
        }
    }
}

// ---------------------------------------------------------------- launchers

template <class TS, class TC, class UT, int TX, int TY, int NT>
size_t smem_bytes() {
    return sizeof(UT) * 2 * (TX + 4) * (TY + 4) + sizeof(TC) * 4 * (TX + 2) * (TY + 2);
}

template <class TS, class TC, class UT, int TX, int TY, int NT, int MODE, bool FIELDS>
cudaError_t launch_one(const StepParams& p, cudaStream_t s) {
    auto kern = fused_step_kernel<TS, TC, UT, TX, TY, NT, MODE, FIELDS>;
    const size_t sm = smem_bytes<TS, TC, UT, TX, TY, NT>();
    static bool configured = false;  // per instantiation, set once per process
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid(p.tiles_x, p.tiles_y);
    kern<<<grid, NT, sm, s>>>(p);
    return cudaGetLastError();
}

template <class TS, class TC, class UT, int TX, int TY, int NT>
struct Variant {
    static constexpr int tx = TX, ty = TY;
    static cudaError_t run(const StepParams& p, cudaStream_t s, int mode, bool fields) {
        if (mode == 1) return fields ? launch_one<TS, TC, UT, TX, TY, NT, 1, true>(p, s)
                                     : launch_one<TS, TC, UT, TX, TY, NT, 1, false>(p, s);
        return fields ? launch_one<TS, TC, UT, TX, TY, NT, 0, true>(p, s)
                      : launch_one<TS, TC, UT, TX, TY, NT, 0, false>(p, s);
    }
};

// Tile configurations per number format: {TX, TY} with 256 threads.
using V64 = Variant<double, double, UPlain<double>, 32, 16, 256>;
using V32 = Variant<float, float, UPlain<float>, 64, 16, 256>;
using V32c = Variant<float, float, UComp, 64, 16, 256>;
using V16 = Variant<__half, float, UComp, 64, 16, 256>;
using Vb16 = Variant<__nv_bfloat16, float, UComp, 64, 16, 256>;

void tile_shape(int fmt, int* tx, int* ty) {
    switch (fmt) {
        case kFmtF64: *tx = V64::tx; *ty = V64::ty; break;
        case kFmtF32: *tx = V32::tx; *ty = V32::ty; break;
        case kFmtF32C: *tx = V32c::tx; *ty = V32c::ty; break;
        case kFmtF16: *tx = V16::tx; *ty = V16::ty; break;
        default: *tx = Vb16::tx; *ty = Vb16::ty; break;
    }
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

// lbm_edge_tile.cuh -- one tile of the fused step on the edge bands of a
// body or of a batch's members (or of the initialisation), the body of the
// edge kernel (lbm_edge.cu).
//
// Nodes within 2 of a bounded edge (3 of a periodic seam) need the boundary
// machinery of Sec. 6: ghost values in Grad u and Div Q, bounced populations
// and periodic images.  A tile owns (tw - 4) x (th - 4) output nodes and has
// one thread per node of the tile and its 2-node halo:
//   stage A (every thread)      : pull-stream, first moment, predicted u*
//   stage B (1-node inner ring) : H = Grad u* with the ghost rules,
//                                 Q = P(F) + Pbar(H)
//   stage C (output nodes)      : 1S = rho0 b + Div Q, moments, corrected j
//                                 and u, equilibrium, BGK collision with He
//                                 forcing, stores, boundary rules of Sec. 6
// with a barrier between stages.  Every global load is issued in stage A, so
// a tile costs one memory latency plus its arithmetic.  The arithmetic is
// that of the interior kernel (lattice units, Q expanded without
// cancellation, collision by opposite pairs).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"
#include "lbm_kernels.h"
#include "lbm_pipeline.cuh"

namespace lbm {

namespace {

// Rare paths, kept out of line so the kernel's code stays small: stores of a
// node on a periodic axis shorter than 6 nodes, and the boundary rules of a
// node on a bounded edge.
template <class T>
__device__ __noinline__ void store_img_slow(T* base, Geo g, int x, int y, T v) {
    store_img(base, g, x, y, v);
}

template <class TC>
struct Pops {
    TC v[9];
};

// Eq. (abbcon) for link i with the node's post-collision population fci
// across a wall of outward normal (sx, sy) inv_len (inv_len = 1/sqrt(2) at a
// corner) carrying the traction (T0, T1) inv_len; Pbar* of Sec. 6 in the
// wall's frame from the quasi-traction g = -T* + Q N and the tangential
// entry of the populations' second moment.
template <class TS, class TC>
__device__ __forceinline__ TC abb_value(int i, TC fci, int sx, int sy, TC inv_len, TC T0, TC T1, TC r, TC pxx,
                                        TC pxy, TC pyy, TC q11, TC q12, TC q21, TC q22, TC inv_c2) {
    const TC N0 = TC(sx) * inv_len, N1 = TC(sy) * inv_len;
    const TC g0 = -T0 * inv_len + q11 * N0 + q12 * N1;
    const TC g1 = -T1 * inv_len + q21 * N0 + q22 * N1;
    const TC t0 = -N1, t1 = N0;
    const TC pnn = (N0 * g0 + N1 * g1) * inv_c2;
    const TC pnt = (t0 * g0 + t1 * g1) * inv_c2;
    const TC ptt = t0 * t0 * pxx + TC(2) * t0 * t1 * pxy + t1 * t1 * pyy;
    const TC sxx = pnn * N0 * N0 + TC(2) * pnt * N0 * t0 + ptt * t0 * t0;
    const TC syy = pnn * N1 * N1 + TC(2) * pnt * N1 * t1 + ptt * t1 * t1;
    const TC sxy = pnn * N0 * N1 + pnt * (N0 * t1 + t0 * N1) + ptt * t0 * t1;
    return -fci + wmul<TS>(TC(2) * wgt<TC>(i), eq_even<TC>(i, r, sxx, sxy, syy));
}

// Links of node (gx, gy) that leave the body through a bounded edge: the
// boundary rules of Sec. 6, written into the first ghost row/column.  fc:
// the node's post-collision populations; r, pxx, pxy, pyy: its moments;
// q: its Q = P + Pbar.  HOLE: links may also enter a hole.
template <class TS, class TC, class UT, bool HOLE>
__device__ __noinline__ void boundary_links(TS* fdst, Geo g, const StepParams& p, const EdgeNow<TC, UT>* s_edge,
                                            int gx, int gy, Pops<TC> fc, TC r, TC pxx, TC pxy, TC pyy, TC q11,
                                            TC q12, TC q21, TC q22, TC inv_c2) {
    const int nx = g.nx, ny = g.ny;
#pragma unroll 1
    for (int i = 1; i < 9; ++i) {
        const int dx = gx + ex(i), dy = gy + ey(i);
        if (HOLE && in_hole(p.hole, dx, dy)) {
            // Eq. (abbcon) across the face of the hole the link crosses, or
            // both faces at the hole's corner
            const bool cx = ex(i) != 0 && in_hole(p.hole, gx + ex(i), gy);
            const bool cy = ey(i) != 0 && in_hole(p.hole, gx, gy + ey(i));
            const int sx = (cx || !cy) ? ex(i) : 0, sy = (cy || !cx) ? ey(i) : 0;
            TC T0 = TC(0), T1 = TC(0);
            if (sx != 0) {  // the face at x0 (entered along +x) or at x1
                const int fa = sx > 0 ? 0 : 1;
                T0 += TC(p.hole_T[2 * fa]);
                T1 += TC(p.hole_T[2 * fa + 1]);
            }
            if (sy != 0) {  // the face at y0 or at y1
                const int fa = sy > 0 ? 2 : 3;
                T0 += TC(p.hole_T[2 * fa]);
                T1 += TC(p.hole_T[2 * fa + 1]);
            }
            const TC inv_len = (sx != 0 && sy != 0) ? TC(0.70710678118654752440) : TC(1);
            const TC val =
                abb_value<TS, TC>(i, fc.v[i], sx, sy, inv_len, T0, T1, r, pxx, pxy, pyy, q11, q12, q21, q22, inv_c2);
            const int oi = opp(i);
            store_img(fdst + oi * g.plane, g, dx, dy, Codec<TS, TC>::st(val, oi, p));
            continue;
        }
        const bool bx2 = !g.perx && (dx < 0 || dx >= nx);
        const bool by2 = !g.pery && (dy < 0 || dy >= ny);
        if (!bx2 && !by2) continue;
        const int oi = opp(i);
        const EdgeNow<TC, UT>* ea = bx2 ? &s_edge[dx < 0 ? 0 : 1] : nullptr;
        const EdgeNow<TC, UT>* eb = by2 ? &s_edge[dy < 0 ? 2 : 3] : nullptr;
        const bool da = ea && ea->kind == kDirichlet, db = eb && eb->kind == kDirichlet;
        TC val;
        if (da || db) {
            // Eq. (bbcon) with jh* = rho0 v* / c (averaged over the Dirichlet
            // edges of a corner link)
            TC a0c, a1c;
            if (da && db) {
                a0c = TC(0.5) * (ea->jh[0] + eb->jh[0]);
                a1c = TC(0.5) * (ea->jh[1] + eb->jh[1]);
            } else {
                const EdgeNow<TC, UT>* e = da ? ea : eb;
                a0c = e->jh[0];
                a1c = e->jh[1];
            }
            val = fc.v[i] - wmul<TS>(TC(2) * wgt<TC>(i), eq_odd<TC>(i, a0c, a1c));
        } else {
            // Eq. (abbcon) with Pbar* of Sec. 6 in the wall-normal frame; a
            // corner link: N = (N1 + N2)/sqrt(2), T* = (T1 + T2)/sqrt(2)
            const int sx = bx2 ? (dx < 0 ? -1 : 1) : 0, sy = by2 ? (dy < 0 ? -1 : 1) : 0;
            const TC inv_len = (sx != 0 && sy != 0) ? TC(0.70710678118654752440) : TC(1);
            TC T0 = TC(0), T1 = TC(0);
            if (ea) {
                T0 += ea->T[0];
                T1 += ea->T[1];
            }
            if (eb) {
                T0 += eb->T[0];
                T1 += eb->T[1];
            }
            val = abb_value<TS, TC>(i, fc.v[i], sx, sy, inv_len, T0, T1, r, pxx, pxy, pyy, q11, q12, q21, q22, inv_c2);
        }
        store_img(fdst + oi * g.plane, g, dx, dy, Codec<TS, TC>::st(val, oi, p));
    }
}

// The tile `tile` of the body whose parameters are p (mode 0: one time step;
// mode 1: the initialisation).  Every thread of the CTA calls it (threads
// beyond tw x th idle through the barriers).  Shared memory: su holds 2 x
// tw x th u-carry values, sq 4 x tw x th arithmetic values, sinit (mode 1)
// 4 x tw x th, s_edge the boundary data of the 4 edges and of a hole's faces
// (5 entries).  want_fields: also write u, v, r to p.fields.  HOLE: the
// body may have a hole (false: p.hole is not read, and the tile's code
// carries none of the hole's tests).  XJ (mode 0): the extrapolated scheme,
// whose carries are E = u(t) + F (the u* of stage A), D = ku jh(t) and
// F = ku (3 jh(t) - jh(t - dt)) (the initialisation reads p.scheme instead).
template <class TS, class TC, class UT, int MODE, bool HOLE, bool XJ>
__device__ __forceinline__ void edge_tile_body(const EdgeTile& tile, const StepParams& p, bool want_fields, UT* su,
                                               TC* sq, TC* sinit, EdgeNow<TC, UT>* s_edge) {
    const int t = threadIdx.x;

    // the collision of this launch is at t_now = n_now dt; the step counter
    // is read here and used once stage A has issued its loads, so that the
    // two memory round trips overlap
    int64_t n_now = 0;
    if (MODE == 0 && t < 4) n_now = p.counter[p.parity] + 1;

    LatConsts<TC> k;
    k.load(p);
    Geo g;
    g.nx = p.nx;
    g.ny = p.ny;
    g.pitch = p.pitch;
    g.plane = p.plane;
    g.perx = p.periodic_x != 0;
    g.pery = p.periodic_y != 0;
    const int nx = g.nx, ny = g.ny;
    const int64_t pitch = g.pitch, plane = g.plane;
    const TS* __restrict__ fsrc = static_cast<const TS*>(p.f_src);
    TS* __restrict__ fdst = static_cast<TS*>(p.f_dst);
    const void* __restrict__ a_src = p.a_src;
    void* __restrict__ a_dst = p.a_dst;
    const typename UT::CView as0 = UT::cview(a_src, 0, plane), as1 = UT::cview(a_src, 1, plane);
    const typename UT::View ad0 = UT::view(a_dst, 0, plane), ad1 = UT::view(a_dst, 1, plane);
    const TC* __restrict__ s_src = static_cast<const TC*>(p.s_src);
    TC* __restrict__ s_dst = static_cast<TC*>(p.s_dst);

    // ---- this thread's node: raw coordinates (an image beyond a periodic
    // seam) and node coordinates
    const int tw = tile.tw, th = tile.th;
    const int tx = t % tw, ty = t / tw;  // ty >= th: an idle thread
    const int nxo = tile.x1 - tile.x0, nyo = tile.y1 - tile.y0;  // output extent
    const int hx = tile.hx, hy = tile.hy;  // halo before the output nodes
    const int gxr = tile.x0 - hx + tx, gyr = tile.y0 - hy + ty;
    const bool okx = g.perx ? (gxr >= -2 && gxr < nx + 2) : (gxr >= 0 && gxr < nx);
    const bool oky = g.pery ? (gyr >= -2 && gyr < ny + 2) : (gyr >= 0 && gyr < ny);
    const int gx = g.perx ? wrap_coord(gxr, nx) : gxr;
    const int gy = g.pery ? wrap_coord(gyr, ny) : gyr;
    // a node of the hole is not part of the body: it holds nothing, and the
    // cells of the hole next to its faces receive the populations the
    // anti-bounce-back rule sends back
    const bool holed = HOLE && p.hole[0] < p.hole[1];  // the body has a hole (uniform)
    const bool removed = holed && in_hole(p.hole, gx, gy);
    const bool inA = okx && oky && ty < th && !removed;
    const bool inB = inA && tx >= hx - 1 && tx <= hx + nxo && ty >= hy - 1 && ty <= hy + nyo;
    const bool inC = tx >= hx && tx < hx + nxo && ty >= hy && ty < hy + nyo && !removed;
    // a removed neighbour along an axis is a face of the hole: a bounded edge
    // for the ghost rules
    const bool hxl = holed && in_hole(p.hole, gx - 1, gy), hxh = holed && in_hole(p.hole, gx + 1, gy);
    const bool hyl = holed && in_hole(p.hole, gx, gy - 1), hyh = holed && in_hole(p.hole, gx, gy + 1);
    const bool gxl = (!g.perx && gx == 0) || hxl, gxh = (!g.perx && gx == nx - 1) || hxh;
    const bool gyl = (!g.pery && gy == 0) || hyl, gyh = (!g.pery && gy == ny - 1) || hyh;
    // within one node of the hole (a link may enter it)
    const bool near_hole =
        holed && gx >= p.hole[0] - 1 && gx <= p.hole[1] && gy >= p.hole[2] - 1 && gy <= p.hole[3];
    // first and second inward neighbours (used only by a ghost rule)
    const int tx1 = gxl ? min(tx + 1, tw - 1) : max(tx - 1, 0);
    const int tx2 = gxl ? min(tx + 2, tw - 1) : max(tx - 2, 0);
    const int ty1 = gyl ? min(ty + 1, th - 1) : max(ty - 1, 0);
    const int ty2 = gyl ? min(ty + 2, th - 1) : max(ty - 2, 0);
    const int txm = max(tx - 1, 0), txp = min(tx + 1, tw - 1);
    const int tym = max(ty - 1, 0), typ = min(ty + 1, th - 1);
    const int64_t o = g.at(gxr, gyr);  // raw position in the planes

    // ---------------- stage A: pull-stream, first moment, predicted u*
    TC f[9];
    TC so0 = TC(0), so1 = TC(0);  // source carry (XJ: D) of the node (stage C)
    TC fo0 = TC(0), fo1 = TC(0);  // XJ: F of the node
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = TC(0);
    if (MODE == 0 && inA) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[i] = Codec<TS, TC>::ld(fsrc[int64_t(i) * plane + o - ex(i) - int64_t(ey(i)) * pitch], i, p);
        const UT A0 = UT::load(as0, o, plane, p);
        const UT A1 = UT::load(as1, o, plane, p);
        if (inC) {
            so0 = s_src[o];
            so1 = s_src[o + plane];
        }
        if (XJ) {  // u* = E
            if (inC) {
                fo0 = s_src[o + 2 * plane];
                fo1 = s_src[o + 3 * plane];
            }
            su[(ty * 2) * tw + tx] = A0;
            su[(ty * 2 + 1) * tw + tx] = A1;
        } else {
            const TC m0 = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
            const TC m1 = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
            su[(ty * 2) * tw + tx] = A0.add(k.ku * m0);
            su[(ty * 2 + 1) * tw + tx] = A1.add(k.ku * m1);
        }
    } else if (MODE == 1 && inA) {
        const int64_t hh = (int64_t(gy) * nx + gx) * 2;
        su[(ty * 2) * tw + tx] = UT::from_double(p.u0 ? p.u0[hh] : 0.0);
        su[(ty * 2 + 1) * tw + tx] = UT::from_double(p.u0 ? p.u0[hh + 1] : 0.0);
    }
    if (tile.lead && t == 0) p.counter[p.parity ^ 1] = n_now;
    if (t < 4) edge_now<TC, UT>(s_edge[t], p.bc[t], double(n_now) * p.dt, p.lat_d[kLatRho0OverC]);
    if (HOLE && t == 4) s_edge[4].kind = kNeumann;  // the faces of a hole (only the kind is read)
    __syncthreads();

    // ---------------- stage B: H = Grad u*, Q = P(F) + Pbar(H)
    bool bad = false;
    if (inB) {
        const EdgeNow<TC, UT>& ebx = s_edge[(hxl || hxh) ? 4 : (gxl ? 0 : 1)];
        const EdgeNow<TC, UT>& eby = s_edge[(hyl || hyh) ? 4 : (gyl ? 2 : 3)];
        TC hh[2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const UT* r0 = su + (ty * 2 + c) * tw;
            const UT u0 = r0[tx];
            hh[c][0] = du_axis<TC, UT>(r0[txm], u0, r0[txp], r0[tx1], r0[tx2], gxl, gxh, ebx, c) * k.inv_2dx;
            hh[c][1] = du_axis<TC, UT>(su[(tym * 2 + c) * tw + tx], u0, su[(typ * 2 + c) * tw + tx],
                                       su[(ty1 * 2 + c) * tw + tx], su[(ty2 * 2 + c) * tw + tx], gyl, gyh, eby,
                                       c) *
                       k.inv_2dx;
        }
        TC q11, q12, q21, q22;
        const TC J =
            stress_remainder<TC>(hh[0][0], hh[0][1], hh[1][0], hh[1][1], k.lam, k.mu, q11, q12, q21, q22);
        bad |= !(J > TC(0)) || !(fabs(q11) + fabs(q12) + fabs(q21) + fabs(q22) < TC(1e30));
        TC* qr = sq + (ty * 4) * tw + tx;
        qr[0] = q11;
        qr[tw] = q12;
        qr[2 * tw] = q21;
        qr[3 * tw] = q22;
        if (MODE == 1) {
            const TC tr = hh[0][0] + hh[1][1];
            TC* ir = sinit + (ty * 4) * tw + tx;
            ir[0] = -k.rho0 * tr;
            ir[tw] = -k.mu * (TC(2) * hh[0][0] + tr) * k.inv_c2;
            ir[2 * tw] = -k.mu * (hh[0][1] + hh[1][0]) * k.inv_c2;
            ir[3 * tw] = -k.mu * (TC(2) * hh[1][1] + tr) * k.inv_c2;
        }
    }
    __syncthreads();

    // ---------------- stage C: source, moments, collision, stores
    if (inC) {
        // s = (dt / c) 1S, 1S = rho0 b + Div(P + Pbar)   (Eq. source1)
        TC dQ[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const TC* r0 = sq + (ty * 4 + c) * tw;
            if ((c & 1) == 0)  // Q_a1: derivative along x
                dQ[c] = dq_axis<TC>(r0[txm], r0[tx], r0[txp], r0[tx1], r0[tx2], gxl, gxh);
            else  // Q_a2: derivative along y
                dQ[c] = dq_axis<TC>(sq[(tym * 4 + c) * tw + tx], r0[tx], sq[(typ * 4 + c) * tw + tx],
                                    sq[(ty1 * 4 + c) * tw + tx], sq[(ty2 * 4 + c) * tw + tx], gyl, gyh);
        }
        const TC sn0 = k.sb0 + k.sq_scale * (dQ[0] + dQ[1]);
        const TC sn1 = k.sb1 + k.sq_scale * (dQ[2] + dQ[3]);

        const UT ux = su[(ty * 2) * tw + tx], uy = su[(ty * 2 + 1) * tw + tx];
        TC r, j0, j1, pxx, pxy, pyy;
        TC du0 = TC(0), du1 = TC(0);  // predictor correction of u*
        if (MODE == 0) {
            r = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
            const TC m0 = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
            const TC m1 = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
            const TC dg = (f[5] + f[6]) + (f[7] + f[8]);
            pxx = (f[1] + f[3]) + dg;
            pyy = (f[2] + f[4]) + dg;
            pxy = (f[5] - f[6]) + (f[7] - f[8]);
            if (XJ) {  // u(t + dt) = u(t) + ku (jh(t) + jh) = E - (F - D) + ku jh
                j0 = m0 + TC(0.5) * sn0;
                j1 = m1 + TC(0.5) * sn1;
                du0 = k.ku * j0 - (fo0 - so0);
                du1 = k.ku * j1 - (fo1 - so1);
            } else if (p.scheme == 1) {
                j0 = m0 + TC(0.5) * sn0;
                j1 = m1 + TC(0.5) * sn1;
                du0 = k.ku * (TC(0.5) * (sn0 - so0));
                du1 = k.ku * (TC(0.5) * (sn1 - so1));
            } else {
                j0 = m0 + TC(0.5) * so0;
                j1 = m1 + TC(0.5) * so1;
            }
        } else {
            // initialisation of Algorithm 1: r = -rho0 Div u0, j = rho0 v0,
            // Pbar = Pbar(Grad u0) (from stage B), f = f^eq
            const TC* ir = sinit + (ty * 4) * tw + tx;
            r = ir[0];
            pxx = ir[tw];
            pxy = ir[2 * tw];
            pyy = ir[3 * tw];
            const int64_t hh = (int64_t(gy) * nx + gx) * 2;
            j0 = k.rho0_over_c * TC(p.v0 ? p.v0[hh] : 0.0);
            j1 = k.rho0_over_c * TC(p.v0 ? p.v0[hh + 1] : 0.0);
        }

        // equilibrium (Sec. 5), He forcing (Eq. source), BGK collision
        // (Eq. col), by opposite pairs: f^col_i = (1 - omega) f_i
        //   + w_i (omega E_i + 3 e_i.(omega jh + (1 - omega/2) s)),
        // E_i the even part of f^eq_i / w_i (equal for i and its opposite)
        const TC tr15 = TC(1.5) * (pxx + pyy);
        const TC E0 = TC(2) * r - tr15;
        const TC Ex = TC(0.5) * r + TC(4.5) * pxx - tr15;
        const TC Ey = TC(0.5) * r + TC(4.5) * pyy - tr15;
        const TC Ed = -r + TC(4.5) * (pxx + pyy) - tr15;
        const TC Ep = Ed + TC(9) * pxy, Em = Ed - TC(9) * pxy;
        const TC w0 = wgt<TC>(0), w1 = wgt<TC>(1), w5 = wgt<TC>(5);
        if (MODE == 1) {
            const TC o0 = TC(3) * j0, o1 = TC(3) * j1;
            f[0] = w0 * E0;
            f[1] = w1 * (Ex + o0);
            f[3] = w1 * (Ex - o0);
            f[2] = w1 * (Ey + o1);
            f[4] = w1 * (Ey - o1);
            f[5] = w5 * (Ep + o0 + o1);
            f[7] = w5 * (Ep - o0 - o1);
            f[6] = w5 * (Em - o0 + o1);
            f[8] = w5 * (Em + o0 - o1);
        }
        const TC b0 = TC(3) * (k.omega * j0 + k.force_pref * sn0);
        const TC b1 = TC(3) * (k.omega * j1 + k.force_pref * sn1);
        const TC ax = wmul<TS>(w1, k.omega * Ex), ay = wmul<TS>(w1, k.omega * Ey);
        const TC ap = wmul<TS>(w5, k.omega * Ep), am = wmul<TS>(w5, k.omega * Em);
        const TC bx = wmul<TS>(w1, b0), by = wmul<TS>(w1, b1);
        const TC bp = wmul<TS>(w5, b0 + b1), bm = wmul<TS>(w5, b1 - b0);
        TC fc[9];
        fc[0] = k.one_m_omega * f[0] + wmul<TS>(w0, k.omega * E0);
        fc[1] = k.one_m_omega * f[1] + (ax + bx);
        fc[3] = k.one_m_omega * f[3] + (ax - bx);
        fc[2] = k.one_m_omega * f[2] + (ay + by);
        fc[4] = k.one_m_omega * f[4] + (ay - by);
        fc[5] = k.one_m_omega * f[5] + (ap + bp);
        fc[7] = k.one_m_omega * f[7] + (ap - bp);
        fc[6] = k.one_m_omega * f[6] + (am + bm);
        fc[8] = k.one_m_omega * f[8] + (am - bm);

        // stores, with the periodic images of nodes near a seam
        const bool short_x = g.perx && nx < 6, short_y = g.pery && ny < 6;
        const int64_t img_x = (!g.perx || short_x) ? 0 : (gx < 3 ? nx : (gx >= nx - 3 ? -nx : 0));
        const int64_t img_y =
            (!g.pery || short_y) ? 0 : (gy < 3 ? int64_t(ny) * pitch : (gy >= ny - 3 ? -int64_t(ny) * pitch : 0));
        const bool slow = short_x || short_y;
        auto put = [&](auto* base, auto v) {
            if (slow) {
                store_img_slow(base, g, gx, gy, v);
                return;
            }
            base[o] = v;
            if (img_x) base[o + img_x] = v;
            if (img_y) base[o + img_y] = v;
            if (img_x && img_y) base[o + img_y + img_x] = v;
        };
#pragma unroll
        for (int i = 0; i < 9; ++i) put(fdst + i * plane, Codec<TS, TC>::st(fc[i], i, p));

        // links that leave the body through a bounded edge or enter the hole
        if (gxl || gxh || gyl || gyh || near_hole) {
            const TC* qr = sq + (ty * 4) * tw + tx;
            Pops<TC> pc;
#pragma unroll
            for (int i = 0; i < 9; ++i) pc.v[i] = fc[i];
            boundary_links<TS, TC, UT, HOLE>(fdst, g, p, s_edge, gx, gy, pc, r, pxx, pxy, pyy, qr[0], qr[tw], qr[2 * tw],
                                       qr[3 * tw], k.inv_c2);
        }

        // carries for the next step: A' = u + ku (jh + s/2), u = u* + du;
        // the extrapolated scheme: E' = E - F + 4 D', D' = ku jh,
        // F' = 3 D' - D (before the first step jh(-dt) = jh(0): D = D',
        // F = 2 D', and E' = u0 + 2 D')
        const bool xj = XJ || (MODE == 1 && p.scheme == 2);
        const TC ka0 = xj ? k.ku * j0 : k.ku * (j0 + TC(0.5) * sn0);
        const TC ka1 = xj ? k.ku * j1 : k.ku * (j1 + TC(0.5) * sn1);
        const TC f0 = MODE == 1 ? TC(2) * ka0 : fo0, f1 = MODE == 1 ? TC(2) * ka1 : fo1;
        const UT A0 = xj ? ux.add(TC(4) * ka0 - f0).renorm() : ux.add(du0 + ka0).renorm();
        const UT A1 = xj ? uy.add(TC(4) * ka1 - f1).renorm() : uy.add(du1 + ka1).renorm();
        UT::store(A0, A1, ad0, ad1, plane, p, put);
        if (xj) {
            const TC d0 = MODE == 1 ? ka0 : so0, d1 = MODE == 1 ? ka1 : so1;
            put(s_dst, ka0);
            put(s_dst + plane, ka1);
            put(s_dst + 2 * plane, TC(3) * ka0 - d0);
            put(s_dst + 3 * plane, TC(3) * ka1 - d1);
        } else {
            put(s_dst, sn0);
            put(s_dst + plane, sn1);
        }
        if (want_fields && p.fields != nullptr) {
            const int64_t fo = int64_t(gy) * nx + gx;
            const int64_t np = int64_t(nx) * ny;
            p.fields[fo] = ux.add(du0).to_double();
            p.fields[np + fo] = uy.add(du1).to_double();
            p.fields[2 * np + fo] = double(j0 * k.c_over_rho0);
            p.fields[3 * np + fo] = double(j1 * k.c_over_rho0);
            p.fields[4 * np + fo] = double(r);
            if (!(isfinite(j0) && isfinite(j1))) bad = true;  // in the arithmetic type: no FP64 work
        }
    }
    if (bad) atomicOr(p.flag, 1);
}

}  // namespace

}  // namespace lbm

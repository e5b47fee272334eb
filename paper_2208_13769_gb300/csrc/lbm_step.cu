// lbm_step.cu -- the fused per-time-step kernel of the Lagrangian LBM
// (Algorithm 1 of arXiv 2208.13769, with the paper's footnote predictor for
// u), and its initialisation variant.
//
// One launch advances the whole body from t_n to t_n+1.  1S at a node needs
// P + Pbar on its 4 neighbours, which need u on a 2-node halo, which needs the
// streamed populations there.  Each CTA owns a strip of W = NT - 4 columns and
// a chunk of rows and walks the rows as a three-stage pipeline, one thread per
// column:
//   stage A, row a     : pull-stream, first moment, predicted u*   (W + 4 cols)
//   stage B, row a - 2 : H = Grad u*, Q = P(F) + Pbar(H)           (W + 2 cols)
//   stage C, row a - 4 : 1S = rho0 b + Div Q, corrected j and u, equilibrium,
//                        BGK collision with He forcing, store       (W cols)
// (a ghost rule at a bounded edge reaches two rows inward, hence the lag of
// two rows per stage).  The input rows -- 9 population segments (each from
// the row its link comes from), the u-carry and the source carry -- are
// brought into a ring of shared-memory row slots by bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier per slot) issued D rows ahead of
// stage A, so global-memory latency overlaps the compute of the rows in
// between.  u* and Q live in 5-row rolling buffers.  Only 4 columns of stage
// A, 2 of stage B and a few warm-up rows per chunk are recomputed; every
// state value crosses HBM once per step in each direction.
//
// Periodic axes: the state arrays carry 3 image rows/columns beyond each
// periodic edge (kept current by the writes of stage C), so every row segment
// a strip needs is contiguous.  Bounded axes: the first ghost row/column
// receives the populations the boundary rules of Sec. 6 send back, so the
// pull never branches.
//
// Lattice units inside the kernel: m = sum_i e_i f_i, Pf = sum_i e_i e_i f_i,
// s = (dt / c) 1S, jh = j / c, so that the equilibrium (Sec. 5) reads
//   f_i^eq = w_i [ r (2 - 3/2 |e_i|^2) + 3 e_i.jh + 3/2 (3 e_i.Pf.e_i - tr Pf) ]
// and no rounded physical constant enters the lattice dynamics.
//
// State per node (two ping-pong copies):
//   f^col_i                                    (9 planes, storage type)
//   A = u_n + dX/(2 rho0) (jh_n + s_n / 2)     (u-carry, 2 comps)
//   s_n                                        (source carry, 2 comps)
// so that u*_n+1 = A + dX/(2 rho0) m  and  jh_n+1 = m + s_(n+1 or n) / 2.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"
#include "lbm_kernels.h"
#include "lbm_pipeline.cuh"

namespace lbm {


// Shared-memory layout: [R pair slots] x [2 rows] x [9 population segments of
// NT + kSegExtra elements] for the bulk-copy ring; u* and Q in 3 pair slots
// (6 rows) each.

template <class TS, class TC, class UT, int NT, int MODE>
__global__ void __launch_bounds__(NT) strip_step_kernel(const __grid_constant__ StepParams p) {
    using CT = typename UT::Elem;        // carry element type
    constexpr int W = NT - 4;            // output columns per strip
    constexpr int SEG = NT + kSegExtra;  // elements per row segment
    constexpr int UP = UT::planes;
    constexpr int ROW_BYTES = 9 * SEG * int(sizeof(TS));
    constexpr int PAIR_BYTES = 2 * ROW_BYTES;
    static_assert(ROW_BYTES % 16 == 0, "row segment size");
    constexpr int ALIGN_COLS = 16 / int(sizeof(TS));

    extern __shared__ __align__(128) unsigned char smem[];
    const int R = p.ring_slots;  // pair slots: lookahead + 3
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);                                 // [R]
    UT* su = reinterpret_cast<UT*>(smem + 256);                                          // [3][2 rows][2 comps][NT]
    TC* sq = reinterpret_cast<TC*>(smem + 256 + sizeof(UT) * 12 * NT);                   // [3][2 rows][4][NT]
    TC* sinit = sq + 24 * NT;                                                            // MODE 1: [3][2][4][NT]
    unsigned char* ring = smem + step_smem_fixed<UT, TC, NT>(MODE);
    __shared__ int s_abort;
    __shared__ EdgeNow<TC, UT> s_edge[4];

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
    const int t = threadIdx.x;
    // output rectangle of this CTA's launch slice, strip and chunk inside it
    // (origins clamped so the last strip / chunk is full when it fits)
    // 1-D grid over the (rectangle, strip, chunk) tiles
    int rb = 0;
    while (rb + 1 < p.nrect && int(blockIdx.x) >= p.tile_base[rb + 1]) ++rb;
    const int local = int(blockIdx.x) - p.tile_base[rb];
    const int bxs = local % p.rect_strips[rb], bys = local / p.rect_strips[rb];
    const int rx0 = p.rect[rb][0], rx1 = p.rect[rb][1];
    const int ry0 = p.rect[rb][2], ry1 = p.rect[rb][3];
    int x0 = rx0 + bxs * W;
    if (x0 > rx1 - W) x0 = rx1 - W > rx0 ? rx1 - W : rx0;
    int y_begin = ry0 + bys * p.chunk_rows;
    if (y_begin > ry1 - p.chunk_rows) y_begin = ry1 - p.chunk_rows > ry0 ? ry1 - p.chunk_rows : ry0;
    const int y_end = min(ry1, y_begin + p.chunk_rows);
    int seg0 = x0 - 8;  // first column of the row segments: 16-byte aligned
    seg0 = (seg0 >= 0 ? seg0 : seg0 - (ALIGN_COLS - 1)) / ALIGN_COLS * ALIGN_COLS;
    const TS* __restrict__ fsrc = static_cast<const TS*>(p.f_src);
    TS* __restrict__ fdst = static_cast<TS*>(p.f_dst);
    const CT* __restrict__ a_src = static_cast<const CT*>(p.a_src);
    CT* __restrict__ a_dst = static_cast<CT*>(p.a_dst);
    const TC* __restrict__ s_src = static_cast<const TC*>(p.s_src);
    TC* __restrict__ s_dst = static_cast<TC*>(p.s_dst);

    int64_t n_now = 0;  // the collision of this launch is at t_now = n_now dt
    if (MODE == 0) n_now = p.counter[p.parity] + 1;
    if (p.write_counter && blockIdx.x == 0 && t == 0)
        p.counter[p.parity ^ 1] = n_now;
    const double t_now = double(n_now) * p.dt;

    // ---- this thread's column
    const int gxr = x0 - 2 + t;  // raw column (an image beyond a periodic edge)
    const bool colA = g.perx ? (gxr >= -2 && gxr < nx + 2) : (gxr >= 0 && gxr < nx);
    const int gx = g.perx ? wrap_coord(gxr, nx) : gxr;
    const bool colB = colA && t >= 1 && t <= NT - 2;
    const bool colC = t >= 2 && t <= NT - 3 && gxr >= rx0 && gxr < rx1;
    const bool gxl = !g.perx && gx == 0, gxh = !g.perx && gx == nx - 1;
    const bool edge_x = gxl || gxh;
    const int tin1 = gxl ? min(t + 1, NT - 1) : max(t - 1, 0);
    const int tin2 = gxl ? min(t + 2, NT - 1) : max(t - 2, 0);
    const int tm = t > 0 ? t - 1 : t, tp = t < NT - 1 ? t + 1 : t;
    const int e_own = gxr - seg0;              // element of this column in a segment
    const int64_t col_off = int64_t(gxr) + kPadCols;  // raw column in the planes
    // periodic image of an output column (one at most for axes of >= 6 nodes)
    const bool short_x = g.perx && nx < 6, short_y = g.pery && ny < 6;
    const int img_x = (!g.perx || short_x) ? 0 : (gx < 3 ? nx : (gx >= nx - 3 ? -nx : 0));

    const int a0 = y_begin - 2;            // first row of stage A
    const int a_last = y_end + 1;          // last row of stage A
    const int npairs = (a_last - a0 + 2) / 2;
    auto row_loaded = [&](int a) { return a >= a0 && a <= a_last && (g.pery || (a >= 0 && a < ny)); };
    auto row_bytes = [&](int pair) {
        return uint32_t(ROW_BYTES) * (uint32_t(row_loaded(a0 + 2 * pair)) + uint32_t(row_loaded(a0 + 2 * pair + 1)));
    };
    // issue the bulk copies of a row pair into ring slot s (thread 0 only);
    // every address is checked for 16-byte alignment before anything is issued
    auto issue_pair = [&](int pair, int s) -> bool {
        unsigned char* base = ring + size_t(s) * PAIR_BYTES;
        const uint32_t bytes = row_bytes(pair);
        if (bytes == 0) return true;
        uintptr_t acc = reinterpret_cast<uintptr_t>(base);
        const TS* src0 = fsrc + g.at(seg0, 0);
        acc |= reinterpret_cast<uintptr_t>(src0) | uintptr_t(pitch * int64_t(sizeof(TS))) |
               uintptr_t(plane * int64_t(sizeof(TS)));
        if (acc & 15) return false;
        mbar_expect_tx(&bars[s], bytes);
        for (int h = 0; h < 2; ++h) {
            const int a = a0 + 2 * pair + h;
            if (!row_loaded(a)) continue;
            TS* dst = reinterpret_cast<TS*>(base + h * ROW_BYTES);
#pragma unroll
            for (int i = 0; i < 9; ++i)
                bulk_load(dst + i * SEG, src0 + i * plane + int64_t(a - ey(i)) * pitch, SEG * sizeof(TS), &bars[s]);
        }
        return true;
    };

    if (t == 0) {
        s_abort = 0;
        if (MODE == 0) {
            for (int s = 0; s < R; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
        }
    }
    if (t < 4) edge_now<TC, UT>(s_edge[t], p.bc[t], t_now, p.rho0 / p.c);
    __syncthreads();
    const EdgeNow<TC, UT>& ebx = s_edge[gxl ? 0 : 1];
    const int D = R - 3;  // pairs of lookahead
    uint32_t phase = 0, issued = 0;
    if (MODE == 0 && t == 0) {
        for (int pr = 0; pr < D && pr < npairs && !s_abort; ++pr) {
            if (issue_pair(pr, pr)) issued |= (row_bytes(pr) ? 1u : 0u) << pr;
            else s_abort = 2;
        }
    }
    // carries of the first pair of stage A, prefetched into registers
    UT anext[2][2];
    TC snext[2][2] = {{TC(0), TC(0)}, {TC(0), TC(0)}};
    auto load_a = [&](int pair) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int a = a0 + 2 * pair + h;
            if (MODE == 0 && colA && row_loaded(a)) {
                const int64_t o = int64_t(a + kPadRows) * pitch + col_off;
                anext[h][0] = UT::ld_global(a_src, o, plane);
                anext[h][1] = UT::ld_global(a_src + UP * plane, o, plane);
            }
        }
    };
    auto load_s = [&](int pair) {  // source carry of stage C's rows of `pair`
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kr = a0 + 2 * pair + h;
            if (MODE == 0 && colC && kr >= y_begin && kr < y_end) {
                const int64_t o = int64_t(kr + kPadRows) * pitch + col_off;
                snext[h][0] = s_src[o];
                snext[h][1] = s_src[o + plane];
            }
        }
    };
    load_a(0);

    bool bad = false;
    int sa = 0;  // su / sq pair slot of stage A's rows
    int ra = 0;  // ring pair slot of stage A's rows
    const int niter = npairs + 2;
    for (int q = 0; q < niter; ++q) {
        const int sb = sa == 0 ? 2 : sa - 1;  // pair slot of stage B's rows (a-2, a-1)
        const int sc = sa == 2 ? 0 : sa + 1;  // pair slot of stage C's rows (a-4, a-3)
        const int rc = ra >= 2 ? ra - 2 : ra - 2 + R;  // ring slot of stage C's rows
        const int a = a0 + 2 * q;
        // stage C's source carries (rows of pair q - 2, prefetched last iteration)
        TC scur[2][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            scur[h][0] = snext[h][0];
            scur[h][1] = snext[h][1];
        }

        // ---------------- stage A: rows a, a+1
        if (q < npairs) {
            if (MODE == 0 && row_bytes(q)) {
                if (!s_abort && !mbar_wait(&bars[ra], (phase >> ra) & 1u)) s_abort = 1;
                phase ^= 1u << ra;
                issued &= ~(1u << ra);
            }
            UT acur[2][2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                acur[h][0] = anext[h][0];
                acur[h][1] = anext[h][1];
            }
            if (q + 1 < npairs) load_a(q + 1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ar = a + h;
                UT* urow = su + ((sa * 2 + h) * 2) * NT;
                if (MODE == 0) {
                    if (colA && row_loaded(ar)) {
                        const TS* pf = reinterpret_cast<const TS*>(ring + size_t(ra) * PAIR_BYTES + h * ROW_BYTES) + e_own;
                        TC fA[9];
#pragma unroll
                        for (int i = 1; i < 9; ++i) fA[i] = Codec<TS, TC>::ld(pf[i * SEG - ex(i)], i, p);
                        const TC m0 = (fA[1] - fA[3]) + (fA[5] - fA[6]) + (fA[8] - fA[7]);
                        const TC m1 = (fA[2] - fA[4]) + (fA[5] - fA[8]) + (fA[6] - fA[7]);
                        urow[t] = acur[h][0].add(k.ku * m0);
                        urow[NT + t] = acur[h][1].add(k.ku * m1);
                    }
                } else if (colA && ar <= a_last) {
                    int gy = ar;
                    bool ok = true;
                    if (gy < 0 || gy >= ny) {
                        if (g.pery) gy = wrap_coord(gy, ny);
                        else ok = false;
                    }
                    if (ok) {
                        const int64_t hh = (int64_t(gy) * nx + gx) * 2;
                        urow[t] = UT::from_double(p.u0 ? p.u0[hh] : 0.0);
                        urow[NT + t] = UT::from_double(p.u0 ? p.u0[hh + 1] : 0.0);
                    }
                }
            }
        }
        __syncthreads();
        if (s_abort) break;  // uniform: written before the barrier
        // refill: the ring slot of pair q + D last served stage C of pair q - 3
        if (MODE == 0 && t == 0 && q + D < npairs) {
            const int rn = ra + D < R ? ra + D : ra + D - R;
            fence_proxy_async();
            if (issue_pair(q + D, rn)) issued |= (row_bytes(q + D) ? 1u : 0u) << rn;
            else s_abort = 2;
        }
        load_s(q - 1);  // stage C's rows of the next iteration (pair q - 1)

        // ---------------- stage B: rows a-2, a-1 (window rows w0..w5 = a-4..a+1)
        if (colB) {
            const UT* wrow[6] = {su + ((sc * 2 + 0) * 2) * NT, su + ((sc * 2 + 1) * 2) * NT,
                                 su + ((sb * 2 + 0) * 2) * NT, su + ((sb * 2 + 1) * 2) * NT,
                                 su + ((sa * 2 + 0) * 2) * NT, su + ((sa * 2 + 1) * 2) * NT};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = a - 2 + h;
                int gy = m;
                bool ok = m >= y_begin - 1 && m <= y_end;
                if (gy < 0 || gy >= ny) {
                    if (g.pery) gy = wrap_coord(gy, ny);
                    else ok = false;
                }
                if (!ok) continue;
                const bool gyl = !g.pery && gy == 0, gyh = !g.pery && gy == ny - 1;
                const EdgeNow<TC, UT>& eby = s_edge[gyl ? 2 : 3];
                const int w = 2 + h;  // window index of row m
                TC hh[2][2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const UT* r0 = wrow[w] + c * NT;
                    const UT u0 = r0[t];
                    hh[c][0] = du_axis<TC, UT>(r0[tm], u0, r0[tp], r0[tin1], r0[tin2], gxl, gxh, ebx, c) *
                               k.inv_2dx;
                    const UT* rm = wrow[w - 1] + c * NT;
                    const UT* rp = wrow[w + 1] + c * NT;
                    const UT* r1 = (gyl ? wrow[w + 1] : wrow[w - 1]) + c * NT;
                    const UT* r2 = (gyl ? wrow[w + 2] : wrow[w - 2]) + c * NT;
                    hh[c][1] = du_axis<TC, UT>(rm[t], u0, rp[t], r1[t], r2[t], gyl, gyh, eby, c) * k.inv_2dx;
                }
                TC q11, q12, q21, q22;
                const TC J = stress_remainder<TC>(hh[0][0], hh[0][1], hh[1][0], hh[1][1], k.lam, k.mu, q11, q12,
                                                  q21, q22);
                bad |= !(J > TC(0)) || !(fabs(q11) + fabs(q12) + fabs(q21) + fabs(q22) < TC(1e30));
                TC* qrow = sq + ((sb * 2 + h) * 4) * NT;
                qrow[t] = q11;
                qrow[NT + t] = q12;
                qrow[2 * NT + t] = q21;
                qrow[3 * NT + t] = q22;
                if (MODE == 1) {
                    const TC tr = hh[0][0] + hh[1][1];
                    TC* irow = sinit + ((sb * 2 + h) * 4) * NT;
                    irow[t] = -k.rho0 * tr;
                    irow[NT + t] = -k.mu * (TC(2) * hh[0][0] + tr) * k.inv_c2;
                    irow[2 * NT + t] = -k.mu * (hh[0][1] + hh[1][0]) * k.inv_c2;
                    irow[3 * NT + t] = -k.mu * (TC(2) * hh[1][1] + tr) * k.inv_c2;
                }
            }
        }
        __syncthreads();

        // ---------------- stage C: rows a-4, a-3 (Q window rows a-6..a-1)
        if (colC) {
            const TC* qw[6] = {sq + ((sa * 2 + 0) * 4) * NT, sq + ((sa * 2 + 1) * 4) * NT,
                               sq + ((sc * 2 + 0) * 4) * NT, sq + ((sc * 2 + 1) * 4) * NT,
                               sq + ((sb * 2 + 0) * 4) * NT, sq + ((sb * 2 + 1) * 4) * NT};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kr = a - 4 + h;
                if (kr < y_begin || kr >= y_end) continue;
                const int gy = kr;
                const bool gyl = !g.pery && gy == 0, gyh = !g.pery && gy == ny - 1;
                const int w = 2 + h;  // window index of row kr

                // s = (dt / c) 1S, 1S = rho0 b + Div(P + Pbar)   (Eq. source1)
                TC dQ[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const TC* r0 = qw[w] + c * NT;
                    if ((c & 1) == 0)  // Q_a1: derivative along x
                        dQ[c] = dq_axis<TC>(r0[tm], r0[t], r0[tp], r0[tin1], r0[tin2], gxl, gxh);
                    else {  // Q_a2: derivative along y
                        const TC* r1 = (gyl ? qw[w + 1] : qw[w - 1]) + c * NT;
                        const TC* r2 = (gyl ? qw[w + 2] : qw[w - 2]) + c * NT;
                        dQ[c] = dq_axis<TC>(qw[w - 1][c * NT + t], r0[t], qw[w + 1][c * NT + t], r1[t], r2[t], gyl,
                                            gyh);
                    }
                }
                const TC sn0 = k.sb0 + k.sq_scale * (dQ[0] + dQ[1]);
                const TC sn1 = k.sb1 + k.sq_scale * (dQ[2] + dQ[3]);

                const UT* urow = su + ((sc * 2 + h) * 2) * NT;
                UT ux = urow[t], uy = urow[NT + t];
                TC r, j0, j1, pxx, pxy, pyy;
                TC du0 = TC(0), du1 = TC(0);  // predictor correction of u*
                TC f[9];
                if (MODE == 0) {
                    const TS* pf =
                        reinterpret_cast<const TS*>(ring + size_t(rc) * PAIR_BYTES + h * ROW_BYTES) + e_own;
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = Codec<TS, TC>::ld(pf[i * SEG - ex(i)], i, p);
                    r = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
                    const TC m0 = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
                    const TC m1 = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
                    const TC dg = (f[5] + f[6]) + (f[7] + f[8]);
                    pxx = (f[1] + f[3]) + dg;
                    pyy = (f[2] + f[4]) + dg;
                    pxy = (f[5] - f[6]) + (f[7] - f[8]);
                    const TC so0 = scur[h][0], so1 = scur[h][1];
                    if (p.scheme == 1) {
                        j0 = m0 + TC(0.5) * sn0;
                        j1 = m1 + TC(0.5) * sn1;
                        du0 = k.ku * (TC(0.5) * (sn0 - so0));
                        du1 = k.ku * (TC(0.5) * (sn1 - so1));
                    } else {
                        j0 = m0 + TC(0.5) * so0;
                        j1 = m1 + TC(0.5) * so1;
                    }
                } else {
                    // initialisation of Algorithm 1: r = -rho0 Div u0,
                    // j = rho0 v0, Pbar = Pbar(Grad u0) (from stage B), f = f^eq
                    const TC* irow = sinit + ((sc * 2 + h) * 4) * NT;
                    r = irow[t];
                    pxx = irow[NT + t];
                    pxy = irow[2 * NT + t];
                    pyy = irow[3 * NT + t];
                    const int64_t hh = (int64_t(gy) * nx + gx) * 2;
                    j0 = k.rho0_over_c * TC(p.v0 ? p.v0[hh] : 0.0);
                    j1 = k.rho0_over_c * TC(p.v0 ? p.v0[hh + 1] : 0.0);
                }

                // equilibrium (Sec. 5), He forcing (Eq. source), BGK collision
                // (Eq. col), by opposite pairs: f^col_i = (1 - omega) f_i
                //   + w_i (omega E_i + 3 e_i.(omega jh + (1 - omega/2) s)),
                // E_i the even part of f^eq_i / w_i (equal for i and opposite)
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
                const TC ax = w1 * (k.omega * Ex), ay = w1 * (k.omega * Ey);
                const TC ap = w5 * (k.omega * Ep), am = w5 * (k.omega * Em);
                const TC bx = w1 * b0, by = w1 * b1;
                const TC bp = w5 * (b0 + b1), bm = w5 * (b1 - b0);
                TC fc[9];
                fc[0] = k.one_m_omega * f[0] + w0 * (k.omega * E0);
                fc[1] = k.one_m_omega * f[1] + (ax + bx);
                fc[3] = k.one_m_omega * f[3] + (ax - bx);
                fc[2] = k.one_m_omega * f[2] + (ay + by);
                fc[4] = k.one_m_omega * f[4] + (ay - by);
                fc[5] = k.one_m_omega * f[5] + (ap + bp);
                fc[7] = k.one_m_omega * f[7] + (ap - bp);
                fc[6] = k.one_m_omega * f[6] + (am + bm);
                fc[8] = k.one_m_omega * f[8] + (am - bm);

                // stores with the periodic images of seam nodes
                const int64_t o = int64_t(gy + kPadRows) * pitch + col_off;
                const int64_t img_y =
                    (!g.pery || short_y) ? 0 : (gy < 3 ? int64_t(ny) * pitch : (gy >= ny - 3 ? -int64_t(ny) * pitch : 0));
                const bool slow = short_x || short_y;
                auto put = [&](auto* base, auto v) {
                    if (slow) {
                        store_img(base, g, gx, gy, v);
                        return;
                    }
                    base[o] = v;
                    if (img_x) base[o + img_x] = v;
                    if (img_y) base[o + img_y] = v;
                    if (img_x && img_y) base[o + img_y + img_x] = v;
                };
#pragma unroll
                for (int i = 0; i < 9; ++i) put(fdst + i * plane, Codec<TS, TC>::st(fc[i], i, p));

                // links that leave the body through a bounded edge: boundary
                // rules of Sec. 6 into the first ghost row/column
                if (edge_x || gyl || gyh) {
                    const TC* qrow = qw[w];
                    const TC q11 = qrow[t], q12 = qrow[NT + t], q21 = qrow[2 * NT + t], q22 = qrow[3 * NT + t];
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        const int dx = gx + ex(i), dy = gy + ey(i);
                        const bool bx2 = !g.perx && (dx < 0 || dx >= nx);
                        const bool by2 = !g.pery && (dy < 0 || dy >= ny);
                        if (!bx2 && !by2) continue;
                        const int oi = opp(i);
                        const EdgeNow<TC, UT>* ea = bx2 ? &s_edge[dx < 0 ? 0 : 1] : nullptr;
                        const EdgeNow<TC, UT>* eb = by2 ? &s_edge[dy < 0 ? 2 : 3] : nullptr;
                        const bool da = ea && ea->kind == kDirichlet, db = eb && eb->kind == kDirichlet;
                        TC val;
                        if (da || db) {
                            // Eq. (bbcon) with jh* = rho0 v* / c (averaged over
                            // the Dirichlet edges of a corner link)
                            TC a0c, a1c;
                            if (da && db) {
                                a0c = TC(0.5) * (ea->jh[0] + eb->jh[0]);
                                a1c = TC(0.5) * (ea->jh[1] + eb->jh[1]);
                            } else {
                                const EdgeNow<TC, UT>* e = da ? ea : eb;
                                a0c = e->jh[0];
                                a1c = e->jh[1];
                            }
                            val = fc[i] - TC(2) * wgt<TC>(i) * eq_odd<TC>(i, a0c, a1c);
                        } else {
                            // Eq. (abbcon) with Pbar* of Sec. 6 in the wall-normal
                            // frame; a corner link: N = (N1 + N2)/sqrt(2),
                            // T* = (T1 + T2)/sqrt(2)
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
                            const TC N0 = TC(sx) * inv_len, N1 = TC(sy) * inv_len;
                            const TC g0 = -T0 * inv_len + q11 * N0 + q12 * N1;
                            const TC g1 = -T1 * inv_len + q21 * N0 + q22 * N1;
                            const TC t0 = -N1, t1 = N0;
                            const TC pnn = (N0 * g0 + N1 * g1) * k.inv_c2;
                            const TC pnt = (t0 * g0 + t1 * g1) * k.inv_c2;
                            const TC ptt = t0 * t0 * pxx + TC(2) * t0 * t1 * pxy + t1 * t1 * pyy;
                            const TC sxx = pnn * N0 * N0 + TC(2) * pnt * N0 * t0 + ptt * t0 * t0;
                            const TC syy = pnn * N1 * N1 + TC(2) * pnt * N1 * t1 + ptt * t1 * t1;
                            const TC sxy = pnn * N0 * N1 + pnt * (N0 * t1 + t0 * N1) + ptt * t0 * t1;
                            val = -fc[i] + TC(2) * wgt<TC>(i) * eq_even<TC>(i, r, sxx, sxy, syy);
                        }
                        store_img(fdst + oi * plane, g, dx, dy, Codec<TS, TC>::st(val, oi, p));
                    }
                }

                // carries for the next step: A' = u + ku (jh + s/2), u = u* + du
                const UT A0 = ux.add(du0 + k.ku * (j0 + TC(0.5) * sn0)).renorm();
                const UT A1 = uy.add(du1 + k.ku * (j1 + TC(0.5) * sn1)).renorm();
#pragma unroll
                for (int c = 0; c < UP; ++c) {
                    put(a_dst + c * plane, A0.part(c));
                    put(a_dst + (UP + c) * plane, A1.part(c));
                }
                put(s_dst, sn0);
                put(s_dst + plane, sn1);
                if (p.fields != nullptr) {
                    const int64_t fo = int64_t(gy) * nx + gx;
                    const int64_t np = int64_t(nx) * ny;
                    p.fields[fo] = ux.add(du0).to_double();
                    p.fields[np + fo] = uy.add(du1).to_double();
                    p.fields[2 * np + fo] = double(j0 * k.c_over_rho0);
                    p.fields[3 * np + fo] = double(j1 * k.c_over_rho0);
                    p.fields[4 * np + fo] = double(r);
                    if (!(fabs(double(j0)) + fabs(double(j1)) < 1e300)) bad = true;
                }
            }
        }
        sa = sa == 2 ? 0 : sa + 1;
        ra = ra + 1 == R ? 0 : ra + 1;
    }
    if (bad) atomicOr(p.flag, 1);
    if (MODE == 0 && s_abort && t == 0) {
        // a wait gave up or an address was misaligned: report, then let the
        // copies already in flight land before the CTA exits
        atomicOr(p.flag, s_abort == 2 ? 8 : 4);
        for (int s = 0; s < R; ++s)
            if (issued & (1u << s)) (void)mbar_wait(&bars[s], (phase >> s) & 1u);
    }
}

// ---------------------------------------------------------------- launchers

template <class TS, class TC, class UT, int NT>
size_t smem_bytes(int ring_slots, int mode) {
    const size_t pair = size_t(2) * 9 * (NT + kSegExtra) * sizeof(TS);
    return step_smem_fixed<UT, TC, NT>(mode) + (mode == 1 ? 0 : pair * ring_slots);
}

template <class TS, class TC, class UT, int NT, int MODE>
cudaError_t launch_one(const StepParams& p, cudaStream_t s) {
    auto kern = strip_step_kernel<TS, TC, UT, NT, MODE>;
    const size_t sm = smem_bytes<TS, TC, UT, NT>(p.ring_slots, MODE);
    static size_t configured = 0;  // largest dynamic shared memory set so far
    if (sm > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        configured = sm;
    }
    kern<<<dim3(p.tile_base[p.nrect > 0 ? p.nrect : 1]), NT, sm, s>>>(p);
    return cudaGetLastError();
}

// `fields` selects at run time whether the launch also writes u, v, r (the
// same instantiation runs either way, so results are bit-identical).
// `fields` selects at run time whether the launch also writes u, v, r (the
// same instantiation runs either way, so results are bit-identical).
// Initialisation: 128-thread CTAs over the whole body; edge bands: one-warp
// CTAs (a band is 2 or 3 nodes thick, so a strip of 28 output columns wastes
// little and many CTAs hide the row-pipeline latency).
template <class TS, class TC, class UT>
struct Variant {
    static constexpr int kInitNT = 128, kBandNT = 32;
    static cudaError_t run(const StepParams& p0, cudaStream_t s, int mode, bool fields) {
        StepParams p = p0;
        if (!fields) p.fields = nullptr;
        return mode == 1 ? launch_one<TS, TC, UT, kInitNT, 1>(p, s) : launch_one<TS, TC, UT, kBandNT, 0>(p, s);
    }
};

using V64 = Variant<double, double, UPlain<double>>;
using V32 = Variant<float, float, UPlain<float>>;
using V32c = Variant<float, float, UComp>;
using V16 = Variant<__half, float, UComp>;
using Vb16 = Variant<__nv_bfloat16, float, UComp>;

// Strip widths (output columns) of the general kernel: initialisation, bands;
// and of the interior kernel.
void strip_widths(int* init_w, int* band_w, int* interior_w) {
    *init_w = 128 - 4;
    *band_w = 32 - 4;
    *interior_w = 128 - 4;
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

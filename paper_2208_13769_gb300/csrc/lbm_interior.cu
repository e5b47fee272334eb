// lbm_interior.cu -- the fused step for the interior of the body.
//
// One launch advances the body from t_n to t_n+1 (Algorithm 1 of arXiv
// 2208.13769, with the paper's footnote predictor for u).  1S at a node needs
// P + Pbar on its 4 neighbours, which need u on a 2-node halo, which needs the
// streamed populations there.
//
// Every node at least 2 nodes from a bounded edge (3 from a periodic seam)
// needs none of the boundary machinery: no ghost rule in Grad u or Div Q, no
// bounced population, no periodic image.  This kernel advances exactly those
// nodes; the edge kernel of lbm_edge.cu advances the thin bands along the
// edges in the same step (both read the same source buffers and write
// disjoint nodes).
//
// Each CTA owns a strip of W <= 124 columns (strips never overlap; the first
// and last strip of a body may be narrower) and a chunk of rows, one thread
// per column plus a 2-column halo on each side, and walks the rows as a
// three-stage pipeline with a lag of one row per stage (written here for a
// walk down the chunk; chunks of odd index walk up it, the same with the
// row order mirrored):
//   stage A, row a     : pull-stream, first moment, predicted u*   (W + 4 cols)
//   stage B, row a - 1 : H = Grad u*, Q = P(F) + Pbar(H)           (W + 2 cols)
//   stage C, row a - 2 : 1S = rho0 b + Div Q, corrected j and u, equilibrium,
//                        BGK collision with He forcing, store       (W cols)
// The 9 population segments of each row arrive in a ring of shared-memory
// slots by bulk asynchronous copies (cp.async.bulk, one mbarrier per slot)
// issued D rows ahead of stage A; the two carries are prefetched one row
// ahead into registers.  u* and Q live in 3-row rolling buffers.
//
// Lattice units inside the kernels: m = sum_i e_i f_i, Pf = sum_i e_i e_i f_i,
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

#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_kernels.h"
#include "lbm_pipeline.cuh"

namespace lbm {

namespace {

// Shared memory of the interior tile: a 128-byte header (the ring's
// mbarriers, at most 8), the u* rows [3][2][NT] and the Q rows [3][4][NT],
// then the ring.
constexpr int kSmemHeader = 128;
template <class UT, class TC, int NT>
__host__ __device__ constexpr size_t interior_smem_fixed() {
    return (kSmemHeader + sizeof(UT) * 6 * NT + sizeof(TC) * 12 * NT + 127) / 128 * 128;
}

// Elements of one bulk-copied row segment: a strip of W <= NT - 4 output
// columns reads columns x0 - 3 .. x0 + W + 2 from a 16-byte aligned start
// (up to 16 / sizeof(TS) - 1 columns before x0 - 3), in a whole number of
// 16-byte units.
template <class TS, int NT>
__host__ __device__ constexpr int seg_elems() {
    return sizeof(TS) == 2 ? NT + 16 : NT + 8;
}

template <class TS, int NT>
__host__ __device__ constexpr size_t interior_row_bytes() {
    return size_t(9) * seg_elems<TS, NT>() * sizeof(TS);
}

}  // namespace

// One tile (column strip bx, row chunk by of the rectangle tg) of one body,
// the only tile of its CTA.  Returns false if a wait gave up or a copy was
// refused (reported in p.flag).  UNROLL3: the row loop unrolled by 3 (the
// row buffers' indices fixed at compile time, the kept populations changing
// roles instead of moving: fewer instructions, more registers; faster for
// the formats whose registers allow it).  KEEP: stage C takes the populations of
// its row from registers that stage A filled two rows earlier (18 more
// registers, 9 fewer shared-memory loads per node) instead of the ring, and
// the ring keeps every slot in flight.  XJ: the extrapolated scheme, whose
// carries are E = u(t) + F (the u* of stage A, in the u-carry planes),
// D = ku jh(t) and F = ku (3 jh(t) - jh(t - dt)) (in the source planes);
// else u* is A + ku m and the source planes hold the last source.
template <class TS, class TC, class UT, int NT, bool KEEP, bool XJ, bool UNROLL3, bool REV>
__device__ __forceinline__ bool interior_tile(const StepParams& p, const TileGeom& tg, int bx, int by,
                                              double* fields) {
    const int W = tg.strip_w;
    constexpr int SEG = seg_elems<TS, NT>();
    constexpr int ROW_BYTES = int(interior_row_bytes<TS, NT>());
    static_assert(ROW_BYTES % 16 == 0, "row size");
    constexpr int ALIGN_COLS = 16 / int(sizeof(TS));

    extern __shared__ __align__(128) unsigned char smem[];
    const int R = p.ring_slots;  // row slots: lookahead + 3
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    UT* su = reinterpret_cast<UT*>(smem + kSmemHeader);                          // [3][2][NT]
    TC* sq = reinterpret_cast<TC*>(smem + kSmemHeader + sizeof(UT) * 6 * NT);   // [3][4][NT]
    unsigned char* ring = smem + interior_smem_fixed<UT, TC, NT>();
    // a wait gave up: set in stage A, read after the row's first barrier, so
    // every thread takes the same decision
    __shared__ int s_abort;

    LatConsts<TC> k;
    k.load(p);
    const int64_t pitch = p.pitch, plane = p.plane;
    const int t = threadIdx.x;
    const int rx0 = tg.rect[0], rx1 = tg.rect[1], ry0 = tg.rect[2], ry1 = tg.rect[3];
    // strip bx of the strip grid, clipped to the rectangle
    const int x0 = tg.strip_x0 + bx * W;
    const int x_lo = max(rx0, x0), x_hi = min(rx1, x0 + W);
    const int chunk_rows = tg.chunk_rows;
    if (x_lo >= x_hi || by * chunk_rows >= ry1 - ry0) return true;
    int y_begin = ry0 + by * chunk_rows;
    if (y_begin > ry1 - chunk_rows) y_begin = ry1 - chunk_rows > ry0 ? ry1 - chunk_rows : ry0;
    const int y_end = min(ry1, y_begin + chunk_rows);
    // first column of the row segments: 16-byte aligned, inside the plane
    int seg0 = x0 - 3;
    seg0 = (seg0 >= 0 ? seg0 : seg0 - (ALIGN_COLS - 1)) / ALIGN_COLS * ALIGN_COLS;
    if (seg0 < -kPadCols) seg0 = -kPadCols;
    // elements of each segment this tile copies: through column x_hi + 2 (the
    // last one stage A pulls from), in whole 16-byte units (a strip narrower
    // than the widest copies less)
    const int seg_n = min(SEG, (x_hi + 3 - seg0 + ALIGN_COLS - 1) / ALIGN_COLS * ALIGN_COLS);

    const TS* __restrict__ fsrc = static_cast<const TS*>(p.f_src);
    TS* __restrict__ fdst = static_cast<TS*>(p.f_dst);
    // the u-carry's planes, per component
    const void* __restrict__ a_src = p.a_src;
    void* __restrict__ a_dst = p.a_dst;
    const typename UT::CView as0 = UT::cview(a_src, 0, plane), as1 = UT::cview(a_src, 1, plane);
    const typename UT::View ad0 = UT::view(a_dst, 0, plane), ad1 = UT::view(a_dst, 1, plane);
    const TC* __restrict__ s_src = static_cast<const TC*>(p.s_src);
    TC* __restrict__ s_dst = static_cast<TC*>(p.s_dst);

    const int gx = x0 - 2 + t;  // this thread's column
    const bool colA = gx >= x_lo - 2 && gx < x_hi + 2;
    const bool colB = gx >= x_lo - 1 && gx < x_hi + 1;
    const bool colC = gx >= x_lo && gx < x_hi;
    const int tm = t > 0 ? t - 1 : t, tp = t < NT - 1 ? t + 1 : t;
    const int e_own = gx - seg0;
    const int64_t col_off = int64_t(gx) + kPadCols;

    // the row walk: down the chunk, or up it (REV), so that two chunks
    // sharing a boundary read its halo rows at the same time (both at their
    // start or both at their end) and the second read hits L2; stage A's row
    // a = a0 + sg q, stage B at a - sg, stage C at a - 2 sg
    constexpr bool rev = REV;
    constexpr int sg = REV ? -1 : 1;
    const int a0 = rev ? y_end + 1 : y_begin - 2;
    const int niter = (y_end - y_begin) + 4;
    const TS* src_seg = fsrc + int64_t(kPadRows) * pitch + seg0 + kPadCols;  // row 0 of plane 0

    // bulk copies of row a into ring slot s (thread 0); the 16-byte alignment
    // of every address is checked before anything is issued.  A refused row
    // is reported in p.flag (bit 8) and never arrives, so the wait for it
    // gives up and the tile stops at the next barrier
    auto issue_row = [&](int a, int s) -> bool {
        unsigned char* base = ring + size_t(s) * ROW_BYTES;
        const uintptr_t acc = reinterpret_cast<uintptr_t>(base) | reinterpret_cast<uintptr_t>(src_seg) |
                              uintptr_t(pitch * int64_t(sizeof(TS))) | uintptr_t(plane * int64_t(sizeof(TS))) |
                              uintptr_t(seg_n * int(sizeof(TS)));
        if (acc & 15) {
            atomicOr(p.flag, 8);
            return false;
        }
        mbar_expect_tx(&bars[s], uint32_t(9 * seg_n * int(sizeof(TS))));
        TS* dst = reinterpret_cast<TS*>(base);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            bulk_load(dst + i * SEG, src_seg + i * plane + int64_t(a - ey(i)) * pitch, uint32_t(seg_n * sizeof(TS)),
                      &bars[s]);
        return true;
    };

    if (t == 0) {
        s_abort = 0;
        for (int s = 0; s < R; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // rows of lookahead: with KEEP a row's ring slot is free once stage A has
    // read it (stage C takes the row's populations from registers), so every
    // slot holds a row in flight; otherwise it also serves stage C two rows
    // later
    const int D = KEEP ? R : R - 3;
    uint32_t phase = 0, issued = 0;
    if (t == 0) {
        fence_proxy_async();  // the CTA's earlier shared-memory accesses precede the copies into the ring
    }
    if (t == 0)
        for (int j = 0; j < D && j < niter; ++j) {
            if (issue_row(a0 + sg * j, j)) issued |= 1u << j;
        }

    // 32-bit element offsets inside a plane (a plane holds fewer than 2^31
    // elements, checked at context creation) and per-plane base pointers,
    // which are the same for every thread of the CTA
    const int32_t pitch32 = int32_t(pitch);
    int32_t off_a = (a0 + kPadRows) * pitch32 + int32_t(col_off);  // row a of stage A, this column
    const int32_t dpitch = rev ? -pitch32 : pitch32;                   // to the walk's next row
    TS* fd[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fd[i] = fdst + int64_t(i) * plane;
    const TC* ss1 = s_src + plane;
    TC* sd1 = s_dst + plane;
    // the extrapolated scheme's F (planes 2, 3)
    const TC* sf0 = s_src + 2 * plane;
    const TC* sf1 = s_src + 3 * plane;

    // carries prefetched one row ahead
    typename UT::Raw an0, an1;  // as stored: decoded where stage A uses them
    TC sn_old0 = TC(0), sn_old1 = TC(0), f_old0 = TC(0), f_old1 = TC(0);
    if (colA) {
        an0 = UT::load_raw(as0, off_a, plane);
        an1 = UT::load_raw(as1, off_a, plane);
    }

    bool bad = false;
    int ra = 0;
    // the populations of this column as stage A pulled them (KEEP): stage C
    // of row a - 2 takes them from here, not the ring
    TC F0[9], F1[9], F2[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) F0[i] = F1[i] = F2[i] = TC(0);
    // One row of the pipeline.  sa = q mod 3 selects the u* and Q row buffers
    // (a compile-time constant when the loop is unrolled by 3); gcur receives
    // stage A's populations of row a, fp2 holds those of row a - 2.  Returns
    // false when the tile gives up.
    auto row = [&](int q, auto sa, TC* gcur, const TC* fp2) -> bool {
        const int sA = sa;                    // slot of row a
        const int sB = sA == 0 ? 2 : sA - 1;  // slot of row a - 1
        const int sC = sA == 2 ? 0 : sA + 1;  // slot of row a - 2 (and Q of row a - 3 in sq[sA])
        const int rc = ra >= 2 ? ra - 2 : ra - 2 + R;
        const TC so0 = sn_old0, so1 = sn_old1;  // source carry (XJ: D) of stage C's row
        const TC fo0 = f_old0, fo1 = f_old1;    // XJ: F of stage C's row

        // ---------------- stage A: row a
        if (!s_abort && !mbar_wait(&bars[ra], (phase >> ra) & 1u)) s_abort = 1;
        phase ^= 1u << ra;
        issued &= ~(1u << ra);
        if (colA) {
            const TS* pf = reinterpret_cast<const TS*>(ring + size_t(ra) * ROW_BYTES) + e_own;
            TC g[9];
#pragma unroll
            for (int i = 1; i < 9; ++i) g[i] = Codec<TS, TC>::ld(pf[i * SEG - ex(i)], i, p);
            if (KEEP) {
                gcur[0] = Codec<TS, TC>::ld(pf[0], 0, p);
#pragma unroll
                for (int i = 1; i < 9; ++i) gcur[i] = g[i];
            }
            if (XJ) {  // u* = u(t) + ku (3 jh(t) - jh(t - dt)) = E
                su[(sA * 2) * NT + t] = UT::decode(an0, p);
                su[(sA * 2 + 1) * NT + t] = UT::decode(an1, p);
            } else {
                const TC m0 = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
                const TC m1 = (g[2] - g[4]) + (g[5] - g[8]) + (g[6] - g[7]);
                su[(sA * 2) * NT + t] = UT::decode(an0, p).add(k.ku * m0);
                su[(sA * 2 + 1) * NT + t] = UT::decode(an1, p).add(k.ku * m1);
            }
            if (q + 1 < niter) {
                an0 = UT::load_raw(as0, off_a + dpitch, plane);
                an1 = UT::load_raw(as1, off_a + dpitch, plane);
            }
        }
        __syncthreads();
        if (s_abort) return false;
        if (t == 0 && q + D < niter) {
            // KEEP: the slot row a just left; else the slot of row a - 3, done
            const int rn = KEEP ? ra : (ra + D < R ? ra + D : ra + D - R);
            fence_proxy_async();
            if (issue_row(a0 + sg * (q + D), rn)) issued |= 1u << rn;
        }
        // source carry of the next iteration's stage C row (a - 1)
        if (colC && q >= 3 && q + 1 < niter) {
            const int32_t o = off_a - dpitch;  // row a - sg
            sn_old0 = s_src[o];
            sn_old1 = ss1[o];
            if (XJ) {
                f_old0 = sf0[o];
                f_old1 = sf1[o];
            }
        }

        // ---------------- stage B: row a - sg
        if (colB && q >= 2) {
            const UT* r0 = su + (sB * 2) * NT;
            // the rows below and above (a - 2 sg and a in the walk)
            const UT* rm = su + ((rev ? sA : sC) * 2) * NT;
            const UT* rp = su + ((rev ? sC : sA) * 2) * NT;
            const TC h11 = r0[tp].minus(r0[tm]) * k.inv_2dx;
            const TC h21 = r0[NT + tp].minus(r0[NT + tm]) * k.inv_2dx;
            const TC h12 = rp[t].minus(rm[t]) * k.inv_2dx;
            const TC h22 = rp[NT + t].minus(rm[NT + t]) * k.inv_2dx;
            TC q11, q12, q21, q22;
            const TC J = stress_remainder<TC>(h11, h12, h21, h22, k.lam, k.mu, q11, q12, q21, q22);
            bad |= !(J > TC(0));  // also catches a non-finite displacement gradient
            TC* qr = sq + (sB * 4) * NT;
            qr[t] = q11;
            qr[NT + t] = q12;
            qr[2 * NT + t] = q21;
            qr[3 * NT + t] = q22;
        }
        __syncthreads();

        // ---------------- stage C: row a - 2 sg
        if (colC && q >= 4) {
            const int gy = a0 + sg * (q - 2);
            const TC* qc = sq + (sC * 4) * NT;                 // Q of row a - 2 sg
            const TC* qm = sq + ((rev ? sB : sA) * 4) * NT;    // Q of the row below it
            const TC* qp = sq + ((rev ? sA : sB) * 4) * NT;    // Q of the row above it
            // s = (dt / c) 1S, 1S = rho0 b + Div(P + Pbar)   (Eq. source1)
            const TC sn0 = k.sb0 + k.sq_scale * ((qc[tp] - qc[tm]) + (qp[NT + t] - qm[NT + t]));
            const TC sn1 = k.sb1 + k.sq_scale * ((qc[2 * NT + tp] - qc[2 * NT + tm]) + (qp[3 * NT + t] - qm[3 * NT + t]));

            const TS* pf = reinterpret_cast<const TS*>(ring + size_t(rc) * ROW_BYTES) + e_own;
            TC f[9];
            if (KEEP) {
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = fp2[i];
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = Codec<TS, TC>::ld(pf[i * SEG - ex(i)], i, p);
            }
            const TC r = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
            const TC m0 = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
            const TC m1 = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
            const TC dg = (f[5] + f[6]) + (f[7] + f[8]);
            const TC pxx = (f[1] + f[3]) + dg;
            const TC pyy = (f[2] + f[4]) + dg;
            const TC pxy = (f[5] - f[6]) + (f[7] - f[8]);
            TC j0, j1, du0 = TC(0), du1 = TC(0);
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

            // equilibrium, He forcing and BGK collision by opposite pairs
            const TC tr15 = TC(1.5) * (pxx + pyy);
            const TC E0 = TC(2) * r - tr15;
            const TC Ex = TC(0.5) * r + TC(4.5) * pxx - tr15;
            const TC Ey = TC(0.5) * r + TC(4.5) * pyy - tr15;
            const TC Ed = -r + TC(4.5) * (pxx + pyy) - tr15;
            const TC Ep = Ed + TC(9) * pxy, Em = Ed - TC(9) * pxy;
            const TC w0 = wgt<TC>(0), w1 = wgt<TC>(1), w5 = wgt<TC>(5);
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
            const int32_t o = off_a - 2 * dpitch;  // row a - 2 sg = gy
#pragma unroll
            for (int i = 0; i < 9; ++i) fd[i][o] = Codec<TS, TC>::st(fc[i], i, p);

            // carries: A' = u + ku (jh + s/2), u = u* + du;  s' = s
            // (XJ: E' = u + ku (3 jh - jh(t)) = E - F + 4 D', D' = ku jh,
            // F' = 3 D' - D)
            const UT ux = su[(sC * 2) * NT + t], uy = su[(sC * 2 + 1) * NT + t];
            const TC ka0 = XJ ? k.ku * j0 : k.ku * (j0 + TC(0.5) * sn0);
            const TC ka1 = XJ ? k.ku * j1 : k.ku * (j1 + TC(0.5) * sn1);
            const UT A0 = XJ ? ux.add(TC(4) * ka0 - fo0).renorm() : ux.add(du0 + ka0).renorm();
            const UT A1 = XJ ? uy.add(TC(4) * ka1 - fo1).renorm() : uy.add(du1 + ka1).renorm();
            auto put = [o](auto* base, auto v) { base[o] = v; };
            UT::store(A0, A1, ad0, ad1, plane, p, put);
            if (XJ) {
                s_dst[o] = ka0;
                sd1[o] = ka1;
                s_dst[o + 2 * plane] = TC(3) * ka0 - so0;
                s_dst[o + 3 * plane] = TC(3) * ka1 - so1;
            } else {
                s_dst[o] = sn0;
                sd1[o] = sn1;
            }
            if (fields != nullptr) {
                const int64_t fo = int64_t(gy) * p.nx + gx;
                const int64_t np = int64_t(p.nx) * p.ny;
                fields[fo] = ux.add(du0).to_double();
                fields[np + fo] = uy.add(du1).to_double();
                fields[2 * np + fo] = double(j0 * k.c_over_rho0);
                fields[3 * np + fo] = double(j1 * k.c_over_rho0);
                fields[4 * np + fo] = double(r);
                if (!(isfinite(j0) && isfinite(j1))) bad = true;  // in the arithmetic type: no FP64 work
            }
        }
        ra = ra + 1 == R ? 0 : ra + 1;
        off_a += dpitch;
        return true;
    };
    if (UNROLL3) {
        // the kept populations change roles instead of moving: row q in
        // F[q mod 3], row q - 2 in F[(q + 1) mod 3]
        for (int q = 0; q < niter;) {
            if (!row(q, std::integral_constant<int, 0>(), F0, F1) || ++q >= niter) break;
            if (!row(q, std::integral_constant<int, 1>(), F1, F2) || ++q >= niter) break;
            if (!row(q, std::integral_constant<int, 2>(), F2, F0) || ++q >= niter) break;
        }
    } else {
        // F1 and F2 keep rows a - 1 and a - 2, rotated after each row
        int sa = 0;
        for (int q = 0; q < niter; ++q) {
            TC gcur[9];
            if (!row(q, sa, gcur, F2)) break;
            if (KEEP) {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    F2[i] = F1[i];
                    F1[i] = gcur[i];
                }
            }
            sa = sa == 2 ? 0 : sa + 1;
        }
    }
    if (bad) atomicOr(p.flag, 1);
    if (s_abort) {
        if (t == 0) {
            atomicOr(p.flag, 4);
            for (int s = 0; s < R; ++s)
                if (issued & (1u << s)) (void)mbar_wait(&bars[s], (phase >> s) & 1u);
        }
        return false;
    }
    return true;
}

// One CTA per tile over the launch's rectangles (one 1-D grid; a body
// without a hole has one rectangle).
// Whether the chunks of a single body alternate their row walk (the two
// directions as two compiled paths of the tile).  In one wave the chunks
// above and below a boundary then read its halo rows together: FP32 with
// the compensated carry reads 61.0 DRAM bytes per node instead of 63.9 and
// runs 2.4 % faster.  Not for the unrolled row loop, whose two copies made
// the plain-carry FP32 and 16-bit kernels 9 to 10 % slower.
template <bool UNROLL3>
__host__ __device__ constexpr bool alternate_walk() {
    return !UNROLL3;
}

template <class TS, class TC, class UT, int NT, int MINB, bool XJ, bool UNROLL3>
__global__ void __launch_bounds__(NT, MINB)
    interior_step_kernel(const __grid_constant__ StepParams p, const __grid_constant__ InteriorRects R) {
    constexpr bool ALT = alternate_walk<UNROLL3>();
    const int b = int(blockIdx.x);
    const int q = (b >= R.first[1]) + (b >= R.first[2]) + (b >= R.first[3]);
    TileGeom tg;
    int tx, f;
    // the rectangle by constant indices (no indexed reads of the parameters)
    if (q == 0) {
        tg = R.g[0];
        tx = R.tiles_x[0];
        f = R.first[0];
    } else if (q == 1) {
        tg = R.g[1];
        tx = R.tiles_x[1];
        f = R.first[1];
    } else if (q == 2) {
        tg = R.g[2];
        tx = R.tiles_x[2];
        f = R.first[2];
    } else {
        tg = R.g[3];
        tx = R.tiles_x[3];
        f = R.first[3];
    }
    const int local = b - f;
    // chunks of odd index walk up (see interior_tile)
    const int bx = local % tx, by = local / tx;
    if (ALT && (by & 1))
        interior_tile<TS, TC, UT, NT, true, XJ, UNROLL3, true>(p, tg, bx, by, p.fields);
    else
        interior_tile<TS, TC, UT, NT, true, XJ, UNROLL3, false>(p, tg, bx, by, p.fields);
}

// The interiors of a batch of bodies for one time step: one CTA per interior
// tile (member rectangle, strip, chunk) of a list ordered longest first, the
// tile's parameters (the member's, with the rectangle and its strip grid)
// read from the device table into shared memory.  The tile is the
// single-body kernel's, so every node of a member takes the same arithmetic
// as when the member is stepped alone.
template <class TS, class TC, class UT, int NT, int MINB, bool UNROLL3>
__global__ void __launch_bounds__(NT, MINB) batch_interior_kernel(const __grid_constant__ BatchInteriorLaunch L) {
    __shared__ __align__(16) StepParams sp;
    const BatchItem it = L.items[blockIdx.x];
    {
        const int4* src = reinterpret_cast<const int4*>(L.params + it.inst);
        int4* dst = reinterpret_cast<int4*>(&sp);
        for (int q = int(threadIdx.x); q < int(sizeof(StepParams) / 16); q += NT) dst[q] = src[q];
    }
    __syncthreads();
    const TileGeom tg = {{sp.rect[0], sp.rect[1], sp.rect[2], sp.rect[3]}, sp.strip_x0, sp.strip_w, sp.chunk_rows};
    // chunks of odd index walk up their rows, as in the single-body kernel:
    // the list holds a member's chunks row by row, so the chunks on either
    // side of a boundary run at about the same time and read its halo rows
    // together (not the unrolled row loop, whose second copy would cost more
    // than the L2 hits give)
    if (!UNROLL3 && (it.b & 1))
        interior_tile<TS, TC, UT, NT, true, false, UNROLL3, true>(sp, tg, it.a, it.b, L.fields ? sp.fields : nullptr);
    else
        interior_tile<TS, TC, UT, NT, true, false, UNROLL3, false>(sp, tg, it.a, it.b, L.fields ? sp.fields : nullptr);
}

template <class TS, class TC, class UT, int NT>
size_t interior_smem_bytes(int ring_slots) {
    return interior_smem_fixed<UT, TC, NT>() + interior_row_bytes<TS, NT>() * size_t(ring_slots);
}

template <class TS, class TC, class UT, int NT, int MINB, bool UNROLL3, bool XJ>
cudaError_t launch_interior_x(const StepParams& p, const InteriorRects& R, cudaStream_t s) {
    auto kern = interior_step_kernel<TS, TC, UT, NT, MINB, XJ, UNROLL3>;
    const size_t sm = interior_smem_bytes<TS, TC, UT, NT>(p.ring_slots);
    static size_t configured = 0;
    if (sm > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        configured = sm;
    }
    if (R.total <= 0) return cudaSuccess;
    kern<<<R.total, NT, sm, s>>>(p, R);
    return cudaGetLastError();
}

// (the extrapolated scheme's variant keeps the rotating loop: its extra
// carries leave no registers for the unrolled one)
template <class TS, class TC, class UT, int NT, int MINB, bool UNROLL3>
cudaError_t launch_interior_t(const StepParams& p, const InteriorRects& R, cudaStream_t s) {
    return p.scheme == 2 ? launch_interior_x<TS, TC, UT, NT, MINB, false, true>(p, R, s)
                         : launch_interior_x<TS, TC, UT, NT, MINB, UNROLL3, false>(p, R, s);
}

template <class TS, class TC, class UT, int NT, int MINB, bool UNROLL3>
cudaError_t launch_batch_interior_t(const BatchInteriorLaunch& L, int ring_slots, cudaStream_t s, int* resident) {
    auto kern = batch_interior_kernel<TS, TC, UT, NT, MINB, UNROLL3>;
    const size_t sm = interior_smem_bytes<TS, TC, UT, NT>(ring_slots);
    static size_t configured = 0;
    if (sm > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        configured = sm;
    }
    if (resident) {  // CTAs per SM of this kernel with this ring
        *resident = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, kern, NT, sm);
        if (e != cudaSuccess) return e;
    }
    if (L.nitems <= 0) return cudaSuccess;
    kern<<<L.nitems, NT, sm, s>>>(L);
    return cudaGetLastError();
}

// The row loops of the single-body interior kernel (launch_interior); the
// register caps hold six CTAs per SM (the parameters come from shared
// memory here, not the launch's constant bank, which takes more registers
// unless capped: 96 to 104).
cudaError_t launch_batch_interior(int fmt, const BatchInteriorLaunch& L, int ring_slots, cudaStream_t s,
                                  int* resident) {
    constexpr int NT = kInteriorThreads;
    switch (fmt) {
        case kFmtF64:
            return launch_batch_interior_t<double, double, UPlain<double>, NT, 2, false>(L, ring_slots, s, resident);
        case kFmtF32:
            return launch_batch_interior_t<float, float, UPlain<float>, NT, 6, true>(L, ring_slots, s, resident);
        case kFmtF32C:
            return launch_batch_interior_t<float, float, UComp, NT, 6, false>(L, ring_slots, s, resident);
        case kFmtF32H:
            return launch_batch_interior_t<float, float, UCompH, NT, 6, false>(L, ring_slots, s, resident);
        case kFmtF16:
            return launch_batch_interior_t<__half, float, UComp, NT, 6, true>(L, ring_slots, s, resident);
        case kFmtBF16:
            return launch_batch_interior_t<__nv_bfloat16, float, UComp, NT, 6, true>(L, ring_slots, s, resident);
    }
    return cudaErrorInvalidValue;
}

void interior_strips(int fmt, int rx0, int rx1, int aligned, int* strip_x0, int* strip_w, int* nstrips) {
    int W = 124, xg = rx0;  // 128 threads: the strip and its 2-column halo on each side
    if (aligned == 1 || aligned == 2) {
        // the fewest strips of equal width on a grid of 32-byte sectors
        // (aligned 1: 8 columns of a 4- or 8-byte plane, 16 of a 2-byte
        // plane), so that no two CTAs store into one sector even when they
        // run far apart in time, or of 16-byte units (aligned 2: 2, 4 or 8
        // columns, wider strips of 16-bit storage at the price of a shared
        // sector at each strip boundary); column x sits at x + kPadCols of a
        // plane row and rows start 256-byte aligned
        const bool half = fmt == kFmtF16 || fmt == kFmtBF16;
        const int es = fmt == kFmtF64 ? 8 : (half ? 2 : 4);
        const int sec = aligned == 1 ? (half ? 16 : 8) : 16 / es;
        const int wmax = 124 / sec * sec;
        const int g0 = ((-kPadCols) % sec + sec) % sec - sec;  // g0 + kPadCols is a multiple of sec
        auto fdiv = [](int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
        xg = g0 + fdiv(rx0 - g0, sec) * sec;
        const int span = rx1 - xg, n = (span + wmax - 1) / wmax;
        W = ((span + n - 1) / n + sec - 1) / sec * sec;
    }
    *strip_x0 = xg;
    *strip_w = W;
    *nstrips = (rx1 - xg + W - 1) / W;  // the first and last strips may be partial
}

template <class TS, class TC, class UT, int NT, int MINB, bool UNROLL3>
int interior_occupancy_t(int ring_slots) {
    auto kern = interior_step_kernel<TS, TC, UT, NT, MINB, false, UNROLL3>;
    const size_t sm = interior_smem_bytes<TS, TC, UT, NT>(ring_slots);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NT, sm) != cudaSuccess) return 0;
    return n;
}

// Per format: the minimum CTAs per SM (the register cap) and the row loop's
// form, as measured on the 4096 x 2048 body: FP16 / BF16 gain 4.5 % from the
// unrolled loop at 80 registers, plain-carry FP32 3 % at 72 registers (7
// CTAs per SM); the compensated carry has no registers to spare and runs the
// rotating loop (the unrolled one was 3 % slower at 80 registers).
int interior_occupancy(int fmt, int ring_slots) {
    switch (fmt) {
        case kFmtF64: return interior_occupancy_t<double, double, UPlain<double>, 128, 2, false>(ring_slots);
        case kFmtF32: return interior_occupancy_t<float, float, UPlain<float>, 128, 7, true>(ring_slots);
        case kFmtF32C: return interior_occupancy_t<float, float, UComp, 128, 4, false>(ring_slots);
        case kFmtF32H: return interior_occupancy_t<float, float, UCompH, 128, 4, false>(ring_slots);
        case kFmtF16: return interior_occupancy_t<__half, float, UComp, 128, 4, true>(ring_slots);
        default: return interior_occupancy_t<__nv_bfloat16, float, UComp, 128, 4, true>(ring_slots);
    }
}

size_t interior_smem(int fmt, int ring_slots) {
    switch (fmt) {
        case kFmtF64: return interior_smem_bytes<double, double, UPlain<double>, 128>(ring_slots);
        case kFmtF32: return interior_smem_bytes<float, float, UPlain<float>, 128>(ring_slots);
        case kFmtF32C: return interior_smem_bytes<float, float, UComp, 128>(ring_slots);
        case kFmtF32H: return interior_smem_bytes<float, float, UCompH, 128>(ring_slots);
        case kFmtF16: return interior_smem_bytes<__half, float, UComp, 128>(ring_slots);
        default: return interior_smem_bytes<__nv_bfloat16, float, UComp, 128>(ring_slots);
    }
}

cudaError_t launch_interior(int fmt, const StepParams& p0, const InteriorRects& R, cudaStream_t s, bool fields) {
    StepParams p = p0;
    if (!fields) p.fields = nullptr;
    switch (fmt) {
        case kFmtF64: return launch_interior_t<double, double, UPlain<double>, 128, 2, false>(p, R, s);
        case kFmtF32: return launch_interior_t<float, float, UPlain<float>, 128, 7, true>(p, R, s);
        case kFmtF32C: return launch_interior_t<float, float, UComp, 128, 4, false>(p, R, s);
        case kFmtF32H: return launch_interior_t<float, float, UCompH, 128, 4, false>(p, R, s);
        case kFmtF16: return launch_interior_t<__half, float, UComp, 128, 4, true>(p, R, s);
        case kFmtBF16: return launch_interior_t<__nv_bfloat16, float, UComp, 128, 4, true>(p, R, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm

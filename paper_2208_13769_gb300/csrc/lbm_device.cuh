// lbm_device.cuh -- device-side pieces of the fused Lagrangian LBM step.
//
// D2Q9 lattice (Sec. 3), equilibrium and source populations (Sec. 5),
// neo-Hooke P(F) (Sec. 7), Poisson stress Pbar(H) (Eq. Plin), the storage
// codecs of the populations and the displacement-carry number types.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_params.h"

namespace lbm {

// ---------------------------------------------------------------- lattice
// Directions: 0 rest; 1..4 axis links (+x, +y, -x, -y); 5..8 diagonals
// (+x+y, -x+y, -x-y, +x-y).  Weights 4/9, 1/9, 1/36.
__host__ __device__ constexpr int ex(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
template <class T>
__host__ __device__ constexpr T wgt(int i) {
    return i == 0 ? T(4) / T(9) : (i <= 4 ? T(1) / T(9) : T(1) / T(36));
}
// w x for a lattice weight w = wgt<T>(i).  1/9 and 1/36 are not binary
// fractions: FP32(1/9) = (1 + 2^-27) / 9, and FP32(4/9), FP32(1/36) are 4 and
// 1/4 times it, so a plain FP32 product scales every equilibrium population
// by 1 + 2^-27.  The collision would then add omega 2^-27 of the mass and
// momentum at every node and step, always with the same sign, and the FP32
// path would drift from the exact solution linearly in time (on the
// 4096 x 2048 clamped body: 8.3e-9 of u per step, 4.1e-5 after 5000 steps).
// The product with the weight's representation error, -w 2^-27 (exact),
// goes into one FMA with the exact product w x, which leaves a single
// rounding of (w - w 2^-27) x, of no preferred sign: after 5000 steps of
// that body the FP32 error of u fell from 4.1e-5 to 3.5e-6, of P on a
// 192 x 96 clamped body from 9.2e-5 to 9.8e-6.  In FP64 the weights' error
// is about 2^-55 and the plain product is kept; so is it with 16-bit
// storage (TS), whose own rounding dominates (see Codec).
template <class TS, class T>
__device__ __forceinline__ T wmul(T w, T x) {
    if constexpr (std::is_same<TS, float>::value && std::is_same<T, float>::value)
        return __fmaf_rn(w, x, __fmul_rn(-w * 0x1p-27f, x));
    else
        return w * x;
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "axis opposites");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "diagonal opposites");

// Per-step constants in the arithmetic type T.
template <class T>
struct Consts {
    T c, inv_c, inv_cs2, omega, one_m_omega, force_pref, half_dt, k_u, rho0, inv_rho0, lam, mu,
        inv_2dx, b0, b1;
    __device__ void load(const StepParams& p) {
        c = T(p.c);
        inv_c = T(1.0 / p.c);
        inv_cs2 = T(1.0 / p.cs2);
        omega = T(p.omega);
        one_m_omega = T(1.0 - p.omega);
        force_pref = T(p.dt * (1.0 - 0.5 * p.omega));
        half_dt = T(0.5 * p.dt);
        k_u = T(p.dt / (2.0 * p.rho0));
        rho0 = T(p.rho0);
        inv_rho0 = T(1.0 / p.rho0);
        lam = T(p.lambda);
        mu = T(p.mu);
        inv_2dx = T(1.0 / (2.0 * p.dX));
        b0 = T(p.body[0]);
        b1 = T(p.body[1]);
    }
};

// Even part of the equilibrium for direction i, divided by w_i:
//   r + (Pbar - r Cs^2 I):(C_i C_i - Cs^2 I) / (2 Cs^4)
// expanded with c^2 = 3 Cs^2 into
//   r (2 - 3/2 |e_i|^2) + (3 e_i.Pbar.e_i - tr Pbar) / (2 Cs^2).
template <class T>
__device__ __forceinline__ T feq_even_over_w(int i, T r, T pxx, T pxy, T pyy, T inv_cs2) {
    const int e2 = ex(i) * ex(i) + ey(i) * ey(i);
    const T tr = pxx + pyy;
    T epe = T(ex(i) * ex(i)) * pxx + T(ey(i) * ey(i)) * pyy + T(2 * ex(i) * ey(i)) * pxy;
    T rterm = (e2 == 0) ? T(2) * r : (e2 == 1 ? T(0.5) * r : -r);
    return rterm + (T(3) * epe - tr) * (T(0.5) * inv_cs2);
}

// Odd part of f^eq / w_i: C_i . j / Cs^2 = 3 (e_i . j) / c.
template <class T>
__device__ __forceinline__ T feq_odd_over_w(int i, T j0, T j1, T inv_c) {
    return T(3) * (T(ex(i)) * j0 + T(ey(i)) * j1) * inv_c;
}

// ---------------------------------------------------------------- material
// Q = P(F) + Pbar(H): the neo-Hooke first Piola-Kirchhoff stress of Sec. 7,
// P = mu (F - F^-T) + lambda/2 (J^2 - 1) F^-T, plus the Poisson stress of
// Eq. (Plin), Pbar = -mu (H + H^T + tr H I) -- the nonlinear remainder that
// drives 1S.  Both stresses are O(mu |H|) while Q is O((lambda - mu) |H|) +
// O(mu |H|^2), so Q is expanded in H before it is evaluated: with
// d = J - 1 = tr H + D, D = H11 H22 - H12 H21,
//   J Q11 = mu (2 D - d (1 + 2 H11 + H22)) + lambda/2 d (2 + d) (1 + H22)
//   J Q22 = mu (2 D - d (1 + 2 H22 + H11)) + lambda/2 d (2 + d) (1 + H11)
//   J Q12 = -H21 d (mu + lambda/2 (2 + d)),  J Q21 = -H12 d (mu + lambda/2 (2 + d)).
// No term of order mu cancels, so the rounding error of Q is relative to
// mu |H| rather than to mu.  Returns J.
// 1 / J, J = det F near 1 for any admissible deformation.  FP32: the
// hardware's approximate reciprocal, one instruction on the critical path of
// stage B (its error, about an ulp, is far inside the FP32 path's
// tolerance); FP64: the correctly rounded reciprocal, for the FP64 path's
// parity with the oracle.
__device__ __forceinline__ float rcp_j(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_j(double x) { return __drcp_rn(x); }

template <class T>
__device__ __forceinline__ T stress_remainder(T h11, T h12, T h21, T h22, T lam, T mu, T& q11, T& q12,
                                              T& q21, T& q22) {
    const T D = h11 * h22 - h12 * h21;
    const T d = (h11 + h22) + D;
    const T J = T(1) + d;
    const T invJ = rcp_j(J);
    const T vol = T(0.5) * lam * d * (T(2) + d);
    q11 = (mu * (T(2) * D - d * (T(1) + T(2) * h11 + h22)) + vol * (T(1) + h22)) * invJ;
    q22 = (mu * (T(2) * D - d * (T(1) + T(2) * h22 + h11)) + vol * (T(1) + h11)) * invJ;
    const T g = -d * (mu + T(0.5) * lam * (T(2) + d)) * invJ;
    q12 = g * h21;
    q21 = g * h12;
    return J;
}

// ---------------------------------------------------------------- storage
// Population codecs: stored value <-> arithmetic value.
template <class S, class T>
struct Codec;
template <>
struct Codec<double, double> {
    __device__ __forceinline__ static double ld(double s, int, const StepParams&) { return s; }
    __device__ __forceinline__ static double st(double v, int, const StepParams&) { return v; }
};
template <>
struct Codec<float, float> {
    __device__ __forceinline__ static float ld(float s, int, const StepParams&) { return s; }
    __device__ __forceinline__ static float st(float v, int, const StepParams&) { return v; }
};
// 16-bit storage keeps h_i = f_i / (w_i 2^-s); the scale pair per direction
// (w_i 2^-s and its inverse) is precomputed on the host.  The scaling
// products are rounded on their own (never fused into a neighbouring add), so
// a decoded population has one value wherever and whenever it is decoded.
// (w_i 2^-s rounded to FP32 is 1 + 2^-27 times too large, as in wmul; at the
// storage's own rounding, 2^-11 per step, that bias does not show: with it
// compensated, in the decode and in the collision, the FP16 displacement
// error of the 4096 x 2048 clamped body after 5000 steps was 1.1e-4 against
// 6.3e-5 without, so 16-bit storage keeps the plain products.)
template <>
struct Codec<__half, float> {
    __device__ __forceinline__ static float ld(__half s, int i, const StepParams& p) {
        return __fmul_rn(__half2float(s), p.dec_scale[i]);
    }
    __device__ __forceinline__ static __half st(float v, int i, const StepParams& p) {
        return __float2half_rn(__fmul_rn(v, p.enc_scale[i]));
    }
};
template <>
struct Codec<__nv_bfloat16, float> {
    __device__ __forceinline__ static float ld(__nv_bfloat16 s, int i, const StepParams& p) {
        return __fmul_rn(__bfloat162float(s), p.dec_scale[i]);
    }
    __device__ __forceinline__ static __nv_bfloat16 st(float v, int i, const StepParams& p) {
        return __float2bfloat16_rn(__fmul_rn(v, p.enc_scale[i]));
    }
};

// ---------------------------------------------------------------- u-carry
// Displacement number types.  Each provides: loading one component of a node
// from the carry buffer and storing it back (the buffer's layout is the
// type's own, below), construction from an FP64 value, adding an increment
// (in the arithmetic type), renormalisation before storing, differences (in
// the arithmetic type), the difference to an FP64 value, and conversion to
// double.  A component's planes are reached through a view (pointers taken
// once per kernel); store() of both components hands each stored word to
// put(plane, value), which writes it at the node (and its periodic images,
// in the edge kernel).

// Layout of a carry buffer, for copies that move its words without
// interpreting them (the seam images).
enum CarryLayout : int {
    kCarryOne = 0,    // one word of the arithmetic type per component: planes x, y
    kCarryPair = 1,   // two FP32 words per component: planes x.hi, x.lo, y.hi, y.lo
    kCarryPair16 = 2  // FP32 high word, 16-bit low word: x.hi, x.lo16, y.hi, y.lo16 (1.5 planes each)
};

template <class T>
struct UPlain {  // u kept in T itself (FP64 or FP32)
    static constexpr int layout = kCarryOne;
    T v;
    // a component's plane
    template <class P>
    struct ViewT {
        P* w;
    };
    using View = ViewT<T>;
    using CView = ViewT<const T>;
    __device__ __forceinline__ static View view(void* a, int comp, int64_t plane) {
        return View{static_cast<T*>(a) + comp * plane};
    }
    __device__ __forceinline__ static CView cview(const void* a, int comp, int64_t plane) {
        return CView{static_cast<const T*>(a) + comp * plane};
    }
    // the stored words as loaded (decode() turns them into the value; a
    // prefetch keeps them raw so that nothing waits for the load early)
    using Raw = UPlain;
    __device__ __forceinline__ static Raw load_raw(const CView& c, int64_t o, int64_t) { return UPlain{c.w[o]}; }
    __device__ __forceinline__ static UPlain decode(const Raw& r, const StepParams&) { return r; }
    __device__ __forceinline__ static UPlain load(const CView& c, int64_t o, int64_t plane, const StepParams& p) {
        return decode(load_raw(c, o, plane), p);
    }
    template <class Put>
    __device__ __forceinline__ static void store(const UPlain& x, const UPlain& y, const View& cx, const View& cy,
                                                 int64_t, const StepParams&, Put&& put) {
        put(cx.w, x.v);
        put(cy.w, y.v);
    }
    __device__ __forceinline__ static UPlain from_double(double d) { return UPlain{T(d)}; }
    __device__ __forceinline__ UPlain add(T d) const { return UPlain{v + d}; }
    __device__ __forceinline__ UPlain renorm() const { return *this; }
    __device__ __forceinline__ T minus(const UPlain& o) const { return v - o.v; }
    __device__ __forceinline__ T minus_d(double d) const { return T(double(v) - d); }
    __device__ __forceinline__ double to_double() const { return double(v); }
};

// Unevaluated sum hi + lo of two floats ("double-float", about 48
// significant bits).  Increments go into lo (lo stays small, so its rounding
// is far below ulp(hi)); renorm() folds lo back with Knuth's two-sum before
// the value is stored, leaving |lo| <= ulp(hi) / 2.
// LO16 = false: lo stored as a float (16 bytes per node for both components).
// LO16 = true: lo stored as FP16 of lo 2^k, k = StepParams::lo_log2 chosen per
// body so that |lo| 2^k stays below 2^15 while |u| < 2^(40 - k); u keeps
// about 35 significant bits in 12 bytes per node.  A larger |u| saturates the
// low word (FP32 precision, no overflow).
template <bool LO16>
struct UPair {
    static constexpr int layout = LO16 ? kCarryPair16 : kCarryPair;
    float hi, lo;
    // a component's high-word plane; its low words follow in the next
    // plane's worth of memory (plane floats, or the first half of it)
    using Lo = typename std::conditional<LO16, __half, float>::type;
    struct View {
        float* hi;
        Lo* lo;
    };
    struct CView {
        const float* hi;
    };
    // first float of component comp: after 2 planes of floats per component,
    // or after 1.5 (a multiple of 32 floats: plane is a multiple of 64)
    __device__ __forceinline__ static int64_t comp_offset(int comp, int64_t plane) {
        return LO16 ? comp * (plane + plane / 2) : comp * 2 * plane;
    }
    __device__ __forceinline__ static View view(void* a, int comp, int64_t plane) {
        float* h = static_cast<float*>(a) + comp_offset(comp, plane);
        return View{h, reinterpret_cast<Lo*>(h + plane)};
    }
    __device__ __forceinline__ static CView cview(const void* a, int comp, int64_t plane) {
        return CView{static_cast<const float*>(a) + comp_offset(comp, plane)};
    }
    struct Raw {
        float hi;
        Lo lo;
    };
    __device__ __forceinline__ static Raw load_raw(const CView& c, int64_t o, int64_t plane) {
        return Raw{c.hi[o], reinterpret_cast<const Lo*>(c.hi + plane)[o]};
    }
    __device__ __forceinline__ static UPair decode(const Raw& r, const StepParams& p) {
        if constexpr (LO16)
            return UPair{r.hi, __fmul_rn(__half2float(r.lo), p.lo_scale[1])};
        else
            return UPair{r.hi, r.lo};
    }
    __device__ __forceinline__ static UPair load(const CView& c, int64_t o, int64_t plane, const StepParams& p) {
        return decode(load_raw(c, o, plane), p);
    }
    __device__ __forceinline__ Lo lo_word(const StepParams& p) const {
        if constexpr (LO16) {
            // round to nearest, finite values beyond the FP16 range clamped
            // to +-65504 (cvt's satfinite)
            unsigned short r;
            asm("cvt.rn.satfinite.f16.f32 %0, %1;" : "=h"(r) : "f"(__fmul_rn(lo, p.lo_scale[0])));
            return __ushort_as_half(r);
        } else {
            return lo;
        }
    }
    // both components (the high words first: fewer registers live in the
    // interior kernel than component by component)
    template <class Put>
    __device__ __forceinline__ static void store(const UPair& x, const UPair& y, const View& cx, const View& cy,
                                                 int64_t, const StepParams& p, Put&& put) {
        put(cx.hi, x.hi);
        put(cy.hi, y.hi);
        put(cx.lo, x.lo_word(p));
        put(cy.lo, y.lo_word(p));
    }
    __device__ __forceinline__ static UPair from_double(double d) {
        const float h = __double2float_rn(d);
        return UPair{h, __double2float_rn(d - double(h))};
    }
    __device__ __forceinline__ UPair add(float d) const { return UPair{hi, __fadd_rn(lo, d)}; }
    __device__ __forceinline__ UPair renorm() const {
        const float s = __fadd_rn(hi, lo);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(lo, bb));
        return UPair{s, e};
    }
    __device__ __forceinline__ float minus(const UPair& o) const {
        return __fadd_rn(__fsub_rn(hi, o.hi), __fsub_rn(lo, o.lo));
    }
    __device__ __forceinline__ float minus_d(double d) const {
        return __double2float_rn((double(hi) - d) + double(lo));
    }
    __device__ __forceinline__ double to_double() const { return double(hi) + double(lo); }
};
using UComp = UPair<false>;
using UCompH = UPair<true>;

}  // namespace lbm

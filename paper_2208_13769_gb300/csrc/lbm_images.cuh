// lbm_images.cuh -- the device copy of one seam-image tile (lbm_images.h),
// shared by the image kernel and the edge kernel's image CTAs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"
#include "lbm_images.h"
#include "lbm_params.h"

namespace lbm {

template <int BYTES>
struct RawBits;
template <>
struct RawBits<2> {
    using T = uint16_t;
};
template <>
struct RawBits<4> {
    using T = uint32_t;
};
template <>
struct RawBits<8> {
    using T = uint64_t;
};

__device__ __forceinline__ int image_wrap(int g, int n) {
    const int w = g % n;
    return w < 0 ? w + n : w;
}

// Thread k of a CTA copies image position k of tile tl: the node (x mod nx,
// y mod ny) in every plane of the instance's destination state.  ES: bytes
// of a stored population; EC: bytes of an element of the arithmetic type;
// CL: the u-carry's layout (CarryLayout in lbm_device.cuh).  Every load
// first, then every store: one memory round trip per thread (a copy loop
// whose store may alias the next load would wait for each).
template <int ES, int EC, int CL>
__device__ __forceinline__ void image_copy(const StepParams* __restrict__ params, const ImageTile& tl, int k) {
    using TS = typename RawBits<ES>::T;
    using TC = typename RawBits<EC>::T;
    const int w = tl.x1 - tl.x0;
    if (w <= 0 || k >= w * (tl.y1 - tl.y0)) return;
    const StepParams& p = params[tl.inst];
    const int xi = tl.x0 + k % w, yi = tl.y0 + k / w;
    const int xs = image_wrap(xi, p.nx), ys = image_wrap(yi, p.ny);
    const int64_t pitch = p.pitch, plane = p.plane;
    const int64_t di = int64_t(yi + kPadRows) * pitch + xi + kPadCols;
    const int64_t si = int64_t(ys + kPadRows) * pitch + xs + kPadCols;
    // u-carry words (the layouts of UPlain / UPair): NA words of TC at
    // offsets ao[c] (in TC elements), and for 16-bit low words NL more of 16
    // bits, each in the half plane after its component's high word
    constexpr int NA = CL == kCarryPair ? 4 : 2;
    constexpr int NL = CL == kCarryPair16 ? 2 : 0;
    const int64_t cstep = CL == kCarryPair16 ? plane + plane / 2 : (CL == kCarryPair ? 2 * plane : plane);
    TS* f = static_cast<TS*>(p.f_dst);
    TC* a = static_cast<TC*>(p.a_dst);
    auto ao = [&](int c) { return CL == kCarryPair ? c * plane : c * cstep; };
    auto al = [&](int c) { return reinterpret_cast<uint16_t*>(a + c * cstep + plane); };
    TC* s = static_cast<TC*>(p.s_dst);
    const bool xj = p.scheme == 2;  // the extrapolated scheme carries two more planes
    TS vf[9];
    TC va[NA], vs[4];
    uint16_t vl[NL > 0 ? NL : 1];
#pragma unroll
    for (int i = 0; i < 9; ++i) vf[i] = f[i * plane + si];
#pragma unroll
    for (int c = 0; c < NA; ++c) va[c] = a[ao(c) + si];
#pragma unroll
    for (int c = 0; c < NL; ++c) vl[c] = al(c)[si];
#pragma unroll
    for (int c = 0; c < 4; ++c) vs[c] = (c < 2 || xj) ? s[c * plane + si] : TC(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i * plane + di] = vf[i];
#pragma unroll
    for (int c = 0; c < NA; ++c) a[ao(c) + di] = va[c];
#pragma unroll
    for (int c = 0; c < NL; ++c) al(c)[di] = vl[c];
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (c < 2 || xj) s[c * plane + di] = vs[c];
}

}  // namespace lbm

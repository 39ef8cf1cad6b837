// collide_f32.cuh -- storage conversions of the reduced-precision forms and
// the FP32 BGK collision on deviations (see step_f32.cu); shared by the
// two-copy and ghost-buffer steps.
#pragma once

#include "tile.cuh"

namespace lbm {

template <class L, class S>
struct F32Io;

template <class L>
struct F32Io<L, StoreF32> {
    template <int I>
    __device__ static __forceinline__ float dev(unsigned int r, const StepArgs&) {
        return __uint_as_float(r) - (float)Link<L, I>::w;
    }
    template <int I>
    __device__ static __forceinline__ unsigned int raw(float g, const StepArgs&) {
        return __float_as_uint((float)Link<L, I>::w + g);
    }
};

template <class L>
struct F32Io<L, StoreF32S> {
    template <int I>
    __device__ static __forceinline__ float dev(unsigned int r, const StepArgs&) {
        return __uint_as_float(r);
    }
    template <int I>
    __device__ static __forceinline__ unsigned int raw(float g, const StepArgs&) {
        return __float_as_uint(g);
    }
};

template <class L>
struct F32Io<L, StoreF16S> {
    template <int I>
    __device__ static __forceinline__ float dev(unsigned short r, const StepArgs& a) {
        return __half2float(__ushort_as_half(r)) * a.f16_inv_scale_f;
    }
    template <int I>
    __device__ static __forceinline__ unsigned short raw(float g, const StepArgs& a) {
        return __half_as_ushort(__float2half_rn(g * a.f16_scale_f));
    }
};

// g*_i = g_i - w (g_i - (f^eq_i - w_i)) + S_i, written per pair of opposite
// links (i, opp(i)) as g*_i = (1 - w) g_i + E + O and g*_opp = (1 - w) g_opp +
// E - O, with y = c_i.u and, per weight class c,
//   E = w w_c (rho - 1 - 1.5 rho |u|^2) - 3 (1 - w/2) w_c u.F
//       + y (4.5 w w_c rho y + 9 (1 - w/2) w_i c_i.F)          (symmetric)
//   O = 3 w w_c rho y + 3 (1 - w/2) w_i c_i.F                  (antisymmetric)
// (rho -> 1 in the rho factors for the incompressible model, Eq. 4).
template <class L, int MODEL>
__device__ __forceinline__ void collide_f32(float (&g)[L::Q], const F32Consts& k, const float* F) {
    float dr = 0.f, jx = 0.5f * F[0], jy = 0.5f * F[1], jz = 0.5f * F[2];
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        dr += g[i];
        if constexpr (K::cx > 0) jx += g[i];
        if constexpr (K::cx < 0) jx -= g[i];
        if constexpr (K::cy > 0) jy += g[i];
        if constexpr (K::cy < 0) jy -= g[i];
        if constexpr (K::cz > 0) jz += g[i];
        if constexpr (K::cz < 0) jz -= g[i];
    });
    constexpr bool QC = MODEL == LBM_QUASI_COMPRESSIBLE;
    const float rho = 1.f + dr;
    float ux = jx, uy = jy, uz = jz;
    if constexpr (QC) {
        const float inv = 1.f / rho;
        ux *= inv;
        uy *= inv;
        uz *= inv;
    }
    const float usq = ux * ux + uy * uy + uz * uz;
    const float uF = ux * F[0] + uy * F[1] + uz * F[2];
    const float rq = QC ? rho : 1.f;
    const float base = dr - 1.5f * rq * usq;
    float Ec = 0.f, Sc = 0.f, Oc = 0.f;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        constexpr int cl = K::cls;
        if constexpr (i == 0 || Link<L, i - (i > 0)>::cls != cl) {  // first link of a class
            Ec = k.ow[cl] * base - k.kw3[cl] * uF;
            Sc = 4.5f * k.ow[cl] * rq;
            Oc = 3.f * k.ow[cl] * rq;
        }
        if constexpr (i == 0) {
            g[0] = __fmaf_rn(k.keep, g[0], Ec);
        } else if constexpr (i < K::opp) {
            constexpr int j = K::opp;
            const float y = K::cx * ux + K::cy * uy + K::cz * uz;
            const float E = __fmaf_rn(y, __fmaf_rn(Sc, y, k.be[i]), Ec);
            const float O = __fmaf_rn(Oc, y, k.so[i]);
            g[i] = __fmaf_rn(k.keep, g[i], E + O);
            g[j] = __fmaf_rn(k.keep, g[j], E - O);
        }
    });
}

}  // namespace lbm

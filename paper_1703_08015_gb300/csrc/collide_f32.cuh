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

template <class L, int MODEL>
__device__ __forceinline__ void collide_f32(float (&g)[L::Q], float omega, const float* F) {
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
    const float rho = 1.f + dr;
    float ux = jx, uy = jy, uz = jz;
    if constexpr (MODEL == LBM_QUASI_COMPRESSIBLE) {
        const float inv = 1.f / rho;
        ux *= inv;
        uy *= inv;
        uz *= inv;
    }
    const float usq = ux * ux + uy * uy + uz * uz;
    const float uF = ux * F[0] + uy * F[1] + uz * F[2];
    const float kf = 1.f - 0.5f * omega;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        constexpr float w = (float)K::w;
        const float cu = K::cx * ux + K::cy * uy + K::cz * uz;
        const float cF = K::cx * F[0] + K::cy * F[1] + K::cz * F[2];
        const float poly = 3.f * cu + 4.5f * cu * cu - 1.5f * usq;
        const float geq = w * (dr + (MODEL == LBM_QUASI_COMPRESSIBLE ? rho * poly : poly));
        const float Sf = kf * w * (3.f * (cF - uF) + 9.f * cu * cF);
        g[i] = g[i] - omega * (g[i] - geq) + Sf;
    });
}

}  // namespace lbm

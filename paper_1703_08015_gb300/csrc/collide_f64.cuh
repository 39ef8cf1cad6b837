// collide_f64.cuh -- the BGK collision of one node in native FP64.
//
//   rho = sum_i f_i,  j = sum_i c_i f_i,  u = (j + F/2) / rho   (Eq. 5; Eq. 6: u = j + F/2)
//   f^eq_i = w_i rho (1 + 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u)    (Eq. 3; Eq. 4: w_i (rho + ...))
//   f*_i = f_i - (f_i - f^eq_i) / tau + S_i                     (Eq. 7 with Eq. 2)
//   S_i = (1 - 1/(2 tau)) w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)] (Guo forcing, not in the paper)
#pragma once

#include "lattice.cuh"
#include "lbm.h"

namespace lbm {

template <class L>
__device__ __forceinline__ void moments_f64(const double (&f)[L::Q], double& rho, double& jx, double& jy,
                                            double& jz) {
    rho = 0.0;
    jx = jy = jz = 0.0;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        rho += f[i];
        if constexpr (K::cx > 0) jx += f[i];
        if constexpr (K::cx < 0) jx -= f[i];
        if constexpr (K::cy > 0) jy += f[i];
        if constexpr (K::cy < 0) jy -= f[i];
        if constexpr (K::cz > 0) jz += f[i];
        if constexpr (K::cz < 0) jz -= f[i];
    });
}

template <class L, int MODEL>
__device__ __forceinline__ void velocity_f64(double rho, double jx, double jy, double jz, const double* F,
                                             double& ux, double& uy, double& uz) {
    ux = jx + 0.5 * F[0];
    uy = jy + 0.5 * F[1];
    uz = jz + 0.5 * F[2];
    if constexpr (MODEL == LBM_QUASI_COMPRESSIBLE) {
        const double inv = 1.0 / rho;
        ux *= inv;
        uy *= inv;
        uz *= inv;
    }
}

template <class L, int MODEL>
__device__ __forceinline__ void collide_f64(double (&f)[L::Q], double omega, const double* F) {
    double rho, jx, jy, jz, ux, uy, uz;
    moments_f64<L>(f, rho, jx, jy, jz);
    velocity_f64<L, MODEL>(rho, jx, jy, jz, F, ux, uy, uz);
    const double usq = ux * ux + uy * uy + uz * uz;
    const double uF = ux * F[0] + uy * F[1] + uz * F[2];
    const double kf = 1.0 - 0.5 * omega;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        const double cu = K::cx * ux + K::cy * uy + K::cz * uz;
        const double cF = K::cx * F[0] + K::cy * F[1] + K::cz * F[2];
        const double poly = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq;
        const double feq = MODEL == LBM_QUASI_COMPRESSIBLE ? K::w * rho * (1.0 + poly) : K::w * (rho + poly);
        const double S = kf * K::w * (3.0 * (cF - uF) + 9.0 * cu * cF);
        f[i] = f[i] - omega * (f[i] - feq) + S;
    });
}

}  // namespace lbm

// step_fixed.cu -- the FP64 tiled step computed without FP64 instructions.
//
// GB300 executes FP64 at a small fraction of its integer and FP32 rate, so
// this kernel evaluates the FP64 BGK update (Eq. 2, 3, 5, 7 with Guo forcing)
// in 64-bit fixed point with resolution 2^-60 and rounds once, to nearest
// even, when it writes the FP64 result.
//
// Inputs.  The PDFs stay close to their weights w_i.  When f_i lies in the
// same binade as w_i (same sign and exponent), f_i - w_i is the difference of
// the two significands, so g_i = (f_i - w_i) * 2^60 is an exact integer
// obtained by subtracting bit patterns.
//
// Collision.  With rho = 1 + sum g_i, J = sum c_i g_i + F/2 (= rho u) and
// Y_i = c_i.J, the update of Eq. 7 with Eq. 2, Eq. 3 and Guo forcing reads
//   f*_i - w_i = (1-w) g_i + w w_i (rho-1) + 3 w w_i Y_i + 3 (1-w/2) w_i c_i.F
//              + (w_i/rho) [ Y_i (4.5 w Y_i + 9 (1-w/2) c_i.F) - 1.5 w J.J - 3 (1-w/2) J.F ]
// (w = 1/tau; the incompressible model of Eq. 4/6 drops the 1/rho).  Sums are
// exact; every product is a 64x64-bit high multiply against a constant scaled
// by 2^59..2^62, truncated at 2^-60 or finer.
//
// Fallback.  A node whose inputs or outputs leave the binade of their weight,
// whose |J| >= 1/16 or whose |rho - 1| >= 1/32 (or that holds NaN/Inf) is
// recomputed with native FP64 instructions, so every node gets the FP64
// update; only the rounding differs between the two paths.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "collide_ff.cuh"

namespace lbm {

// Unbiased binary exponent of a positive constant (compile time).
constexpr int fp_exponent(double w) {
    int e = 0;
    while (w < 1.0) {
        w *= 2.0;
        e--;
    }
    while (w >= 2.0) {
        w *= 0.5;
        e++;
    }
    return e;
}

template <class L, int I>
struct FixLink {
    using K = Link<L, I>;
    // g = (bits(f) - bits(w)) << SHIFT is (f - w) in units of 2^-60
    static constexpr int SHIFT = fp_exponent(K::w) + 8;
    static_assert(SHIFT >= 0 && SHIFT <= 8, "weights must lie in [2^-8, 1)");
    static constexpr int REP = I < K::opp ? I : K::opp;  // representative of the +-c pair
    static constexpr int SIGN = I < K::opp ? 1 : -1;
};

// a * K / 2^L, floor, for |a| < 2^(L-1) and K a constant scaled by 2^L.
template <int L>
__device__ __forceinline__ long long qmul(long long a, long long K) {
    return __mul64hi(a << (64 - L), K);
}

// x / 2^S rounded to nearest, ties to even.
template <int S>
__device__ __forceinline__ long long rne_shift(long long x) {
    if constexpr (S == 0) {
        return x;
    } else {
        const long long q = x >> S;
        const long long r = x & ((1ll << S) - 1);
        const long long half = 1ll << (S - 1);
        return q + (long long)((r > half) | ((r == half) & (q & 1)));
    }
}

__device__ __forceinline__ bool small(long long x, int log2bound) {
    // |x| < 2^log2bound
    return (unsigned long long)(x + (1ll << log2bound)) < (2ull << log2bound);
}

template <class L, int C>
constexpr int first_of_class() {
    int i = 0;
    while (i < L::Q && L::cls_[i] != C) i++;
    return i;
}

// The fixed-point update of one node.  `out` points at the node's slot of
// link 0 in the destination tile (links are `stride` apart); each +-c pair is
// stored as soon as it is computed.  Returns false when the node must be
// recomputed in FP64 (its stores are then overwritten by the caller).
template <class L, int MODEL>
__device__ __forceinline__ bool collide_fixed(const unsigned long long (&b)[L::Q], const FixedConsts& k,
                                              unsigned long long* out, int stride) {
    constexpr int Q = L::Q;
    long long g[Q];
    bool ok = true;
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const unsigned long long wb = (unsigned long long)k.w_bits[Link<L, i>::cls];
        ok &= ((b[i] ^ wb) >> 52) == 0;
        g[i] = (long long)(b[i] - wb) << FixLink<L, i>::SHIFT;
    });
    long long dr = k.dws, jx = k.half_f[0], jy = k.half_f[1], jz = k.half_f[2];
    static_for<0, Q>([&](auto I) {
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
    ok &= small(dr, 55) & small(jx, 56) & small(jy, 56) & small(jz, 56);
    if (!ok) return false;

    // 1 / rho = 1 + e: start from 1 - d + d^2, two Newton steps (error < 2^-60 for |d| < 2^-5)
    long long e = 0;
    if constexpr (MODEL == LBM_QUASI_COMPRESSIBLE) {
        e = -dr + qmul<60>(dr, dr);
#pragma unroll
        for (int it = 0; it < 2; it++) {
            const long long t = dr + e + qmul<60>(dr, e);  // rho (1 + e) - 1
            e = e - t - qmul<60>(e, t);
        }
    }
    const long long jj = qmul<60>(jx, jx) + qmul<60>(jy, jy) + (L::D == 3 ? qmul<60>(jz, jz) : 0);
    const long long gamma = qmul<61>(jj, k.g1) + qmul<60>(jx, k.kf[0]) + qmul<60>(jy, k.kf[1]) +
                            (L::D == 3 ? qmul<60>(jz, k.kf[2]) : 0);
    auto emit = [&](auto I, long long gs) {
        constexpr int i = decltype(I)::value;
        const unsigned long long wb = (unsigned long long)k.w_bits[Link<L, i>::cls];
        const unsigned long long o = wb + (unsigned long long)rne_shift<FixLink<L, i>::SHIFT>(gs);
        ok &= ((o ^ wb) >> 52) == 0;
        out[i * stride] = o;
    };
    long long R = 0, V = 0, PX = 0, PY = 0, PZ = 0;  // scalars of the current weight class
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using F = FixLink<L, i>;
        using K = Link<L, i>;
        if constexpr (F::REP == i) {
            constexpr int c = K::cls;
            if constexpr (i == first_of_class<L, c>()) {
                R = qmul<62>(dr, k.k_rho[c]);
                V = MODEL == LBM_QUASI_COMPRESSIBLE ? k.w60[c] + qmul<62>(e, k.kw[c]) : k.w60[c];
                if constexpr (c > 0) {
                    PX = qmul<61>(jx, k.k_j[c]);
                    PY = qmul<61>(jy, k.k_j[c]);
                    if constexpr (L::D == 3) PZ = qmul<61>(jz, k.k_j[c]);
                }
            }
            if constexpr (i == 0) {
                emit(I, qmul<62>(g[0], k.k_keep) + R + qmul<60>(-gamma, V));
            } else {
                constexpr int j = K::opp;
                const long long Y = K::cx * jx + K::cy * jy + K::cz * jz;
                const long long A = qmul<59>(Y, k.alpha) + k.beta[i];
                const long long T = qmul<60>(Y, A);
                const long long E = R + qmul<60>(T - gamma, V);
                const long long O = K::cx * PX + K::cy * PY + K::cz * PZ + k.so[i];
                emit(I, qmul<62>(g[i], k.k_keep) + E + O);
                emit(std::integral_constant<int, j>{}, qmul<62>(g[j], k.k_keep) + E - O);
            }
        }
    });
    return ok;
}

template <class L, int A, int MODEL, int MINB>
__global__ void __launch_bounds__(work_threads<L, A>(), MINB) k_step_fixed(const StepArgs a) {
    using TL = Tile<L, A>;
    using T = unsigned long long;
    __shared__ NeighShared<TL, work_tiles()> sh;
    WorkNode wn;
    if (!stage_work<TL, work_tiles(), work_threads<L, A>()>(sh, a, wn)) return;
    const NodePos<A> p = node_pos<TL>(wn.node);
    T b[L::Q];
    const int rank = gather<L, A, work_tiles(), T>(sh, a.src, wn.lt, wn.node, p, b);
    const int stride = sh.loc[wn.lt][TL::CENTER].y;
    T* out = own_slot<TL, work_tiles(), T>(sh, a.dst, wn.lt, rank);
    if (!collide_fixed<L, MODEL>(b, a.fx, out, stride)) {
        // out of range: the same update in native FP64 (a call, so that its
        // registers do not weigh on the fixed-point path)
        update_fp64<L, A, MODEL, work_tiles()>(sh, a, wn, p, out, stride);
    }
}

template <class L, int A, int MODEL, int MINB>
cudaError_t launch_step_fixed(const StepArgs& a, cudaStream_t s) {
    if (a.n_work_blocks == 0) return cudaSuccess;
    k_step_fixed<L, A, MODEL, MINB><<<a.n_work_blocks, work_threads<L, A>(), 0, s>>>(a);
    return cudaGetLastError();
}

// ---- host: constants -------------------------------------------------------
static long long fix(double v, int L) { return std::llround(std::ldexp(v, L)); }

template <class L>
static void fixed_consts_for(const lbm_params* p, FixedConsts* k) {
    const double omega = 1.0 / p->tau;
    const double kf = 1.0 - 0.5 * omega;
    double F[3] = {p->force[0], p->force[1], L::D == 3 ? p->force[2] : 0.0};
    for (int c = 0; c < 3; c++) {
        const double w = L::wc_[c];
        std::memcpy(&k->w_bits[c], &w, sizeof w);
        k->w60[c] = fix(w, 60);  // exact: every weight is a multiple of 2^-60
        k->kw[c] = fix(w, 62);
        k->k_rho[c] = fix(omega * w, 62);
        k->k_j[c] = fix(3.0 * omega * w, 61);
    }
    k->k_keep = fix(1.0 - omega, 62);
    k->alpha = fix(4.5 * omega, 59);
    k->g1 = fix(1.5 * omega, 61);
    for (int a = 0; a < 3; a++) {
        k->kf[a] = fix(3.0 * kf * F[a], 60);
        k->half_f[a] = fix(0.5 * F[a], 60);
    }
    long long ws = 0;
    for (int i = 0; i < L::Q; i++) {
        const double cF = L::cx_[i] * F[0] + L::cy_[i] * F[1] + L::cz_[i] * F[2];
        const double w = L::wc_[L::cls_[i]];
        k->beta[i] = fix(9.0 * kf * cF, 60);
        k->so[i] = fix(3.0 * kf * w * cF, 60);
        ws += fix(w, 60);
    }
    k->dws = ws - (1ll << 60);
}

void fixed_consts(const lbm_params* p, FixedConsts* k) {
    *k = FixedConsts{};
    if (p->lattice == LBM_D2Q9)
        fixed_consts_for<D2Q9>(p, k);
    else if (p->lattice == LBM_D3Q19)
        fixed_consts_for<D3Q19>(p, k);
}

template <class L, int A>
static StepLaunch pick(int model) {
    constexpr int MINB = fp64_step_min_blocks<L, A>();
    return model == LBM_QUASI_COMPRESSIBLE ? &launch_step_fixed<L, A, LBM_QUASI_COMPRESSIBLE, MINB>
                                           : &launch_step_fixed<L, A, LBM_INCOMPRESSIBLE, MINB>;
}

StepLaunch select_step_fixed(int lattice, int a, int model) {
    if (lattice == LBM_D2Q9) {
        if (a == 8) return pick<D2Q9, 8>(model);
        if (a == 16) return pick<D2Q9, 16>(model);
        if (a == 32) return pick<D2Q9, 32>(model);
    } else if (lattice == LBM_D3Q19) {
        if (a == 4) return pick<D3Q19, 4>(model);
        if (a == 8) return pick<D3Q19, 8>(model);
    }
    return nullptr;
}

}  // namespace lbm

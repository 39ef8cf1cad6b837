// collide_ff.cuh -- the FP64 BGK update with float-float arithmetic (see
// step_ff.cu for the scheme); shared by the two-copy and ghost-buffer steps.
#pragma once

#include "collide_f64.cuh"
#include "tile.cuh"

namespace lbm {

struct ff {
    float h, l;
};

// s + e = a + b exactly, for |a| >= |b| (or a = 0).
__device__ __forceinline__ ff fast2(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return ff{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// Sums are renormalised (after cancellation the low part could otherwise
// grow to the size of the high part, and a following product would evaluate
// it in single precision); products return (p, e) with |e| within a few ulps
// of p, which every consumer accepts, saving a two-sum per product.
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    const ff s = two_sum(x.h, y.h);
    return fast2(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}

// x + y without the final renormalisation, for sums that only feed further
// sums (ff_sum3): the error is the same as ff_add's, but the low part may
// exceed half an ulp of the high part after cancellation, which a following
// product would evaluate in single precision.
__device__ __forceinline__ ff ff_add_lazy(ff x, ff y) {
    const ff s = two_sum(x.h, y.h);
    return ff{s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l))};
}

__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.h, -x.l}; }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return ff{p, e};
}

__device__ __forceinline__ ff ff_sqr(ff x) {
    const float p = __fmul_rn(x.h, x.h);
    float e = __fmaf_rn(x.h, x.h, -p);
    e = __fmaf_rn(__fmul_rn(2.f, x.h), x.l, e);
    return ff{p, e};
}

__device__ __forceinline__ ff ff_c(const float2 k) { return ff{k.x, k.y}; }

constexpr float pow2f(int e) {
    float v = 1.f;
    while (e > 0) {
        v *= 2.f;
        e--;
    }
    while (e < 0) {
        v *= 0.5f;
        e++;
    }
    return v;
}

constexpr int fp_exp(double w) {
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
struct FFLink {
    using K = Link<L, I>;
    static constexpr int E = fp_exp(K::w);  // binade of w_i: ulp(w_i) = 2^(E - 52)
    static constexpr int SHIFT = E + 8;     // d << SHIFT is g in units of 2^-60
};

__device__ __forceinline__ bool small_ll(long long x, int log2bound) {
    return (unsigned long long)(x + (1ll << log2bound)) < (2ull << log2bound);
}

// -2^47 <= x < 2^47, from the high word alone.
__device__ __forceinline__ bool within_2p47(long long x) {
    return (unsigned)((int)(x >> 32) + (1 << 15)) < (1u << 16);
}

// Distance from w to the nearer edge of its binade [2^e, 2^(e+1)), in ulps of w.
constexpr double ulps_to_binade_edge(double w) {
    const int e = fp_exp(w);
    const double lo = e >= 0 ? pow2f(e) : 1.0 / (double)pow2f(-e), ulp = lo / 4503599627370496.0;  // 2^52
    const double d = (w - lo) < (2.0 * lo - w) ? (w - lo) : (2.0 * lo - w);
    return d / ulp;
}

// A value x * 2^-60 (|x| < 2^57) as float-float, exactly up to the last piece.
__device__ __forceinline__ ff q60_to_ff(long long x) {
    const float f2 = __fmul_rn(__int2float_rn((int)(x >> 48)), pow2f(-12));
    const float f1 = __fmul_rn(__int2float_rn((int)((x >> 24) & 0xFFFFFF)), pow2f(-36));
    const float f0 = __fmul_rn(__int2float_rn((int)(x & 0xFFFFFF)), pow2f(-60));
    const ff s = fast2(f2, f1);
    return fast2(s.h, __fadd_rn(s.l, f0));
}

// a + b + c with the rounding errors of both high-part sums kept in the low
// part (not renormalised: ulp_round takes any low part below 2^30).
__device__ __forceinline__ ff ff_sum3(ff a, ff b, ff c) {
    const ff s = two_sum(a.h, b.h);
    const ff t = two_sum(s.h, c.h);
    return ff{t.h, __fadd_rn(__fadd_rn(__fadd_rn(a.l, b.l), __fadd_rn(c.l, s.l)), t.l)};
}

// FP64 bit pattern of w + r ulp(w) with r the integer within one unit of
// x = x.h + x.l (units of ulp(w)): x.h splits exactly into hi 2^24 + rem, and
// rem and x.l are rounded to integers separately.  (A single FP32 -> int64
// conversion of x.h is slower here: those conversions issue at a fraction of
// the 32-bit rate.)
//
// The result stays in the binade of w (same sign and exponent bits): |r| <
// 2^47 + 2^30 + 1 ulps, and every lattice weight lies at least 2^48 ulps from
// the edges of its binade (checked at compile time in collide_ff).
__device__ __forceinline__ unsigned long long ulp_round(ff x, unsigned long long wb, bool& ok) {
    ok &= fabsf(x.h) < pow2f(47) && fabsf(x.l) < pow2f(30);
    const int hi = __float2int_rz(__fmul_rn(x.h, pow2f(-24)));            // |hi| < 2^23
    const float rem = __fmaf_rn(__int2float_rn(hi), -pow2f(24), x.h);     // exact, |rem| < 2^24
    const int lo = __float2int_rn(rem) + __float2int_rn(x.l);
    return wb + (unsigned long long)(((long long)hi << 24) + (long long)lo);
}

template <class L, int C>
constexpr int ff_first_of_class() {
    int i = 0;
    while (i < L::Q && L::cls_[i] != C) i++;
    return i;
}

// The node's update in native FP64 (the range fallback of the float-float and
// fixed-point steps): the words are gathered again, collided and stored.  Not
// inlined: as a call its registers stay off the step's hot path (inline, the
// FP64 update held enough registers to spill the whole D3Q19 step).
template <class L, int A, int MODEL, int KMAX>
__device__ __noinline__ void update_fp64(const NeighShared<Tile<L, A>, KMAX>& sh, const StepArgs& a,
                                            const WorkNode& wn, const NodePos<A>& p, unsigned long long* out,
                                            int stride) {
    unsigned long long b[L::Q];
    gather<L, A, KMAX, unsigned long long>(sh, a.src, wn.lt, wn.node, p, b);
    double f[L::Q];
    static_for<0, L::Q>([&](auto I) { f[decltype(I)::value] = __longlong_as_double((long long)b[decltype(I)::value]); });
    collide_f64<L, MODEL>(f, a.omega, a.force);
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        out[i * stride] = (unsigned long long)__double_as_longlong(f[i]);
    });
}

template <class L, int MODEL>
__device__ __forceinline__ bool collide_ff(const unsigned long long (&b)[L::Q], const FixedConsts& k,
                                           const FFConsts& c, unsigned long long* out, int stride) {
    constexpr int Q = L::Q;
    static_assert(ulps_to_binade_edge(L::wc_[0]) >= 281474976710656.0 &&
                      ulps_to_binade_edge(L::wc_[1]) >= 281474976710656.0 &&
                      ulps_to_binade_edge(L::wc_[2]) >= 281474976710656.0,
                  "a weight within 2^48 ulps of its binade edge: ulp_round would need its binade check");
    long long d[Q];
    bool ok = true;
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        d[i] = (long long)(b[i] - (unsigned long long)k.w_bits[Link<L, i>::cls]);
        ok &= within_2p47(d[i]);  // also rejects another binade, sign, NaN/Inf
    });
    // exact sums per class (units of ulp(w_c)), then one shift per class to 2^-60
    long long sr[3] = {0, 0, 0}, sx[3] = {0, 0, 0}, sy[3] = {0, 0, 0}, sz[3] = {0, 0, 0};
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        constexpr int cl = K::cls;
        sr[cl] += d[i];
        if constexpr (K::cx > 0) sx[cl] += d[i];
        if constexpr (K::cx < 0) sx[cl] -= d[i];
        if constexpr (K::cy > 0) sy[cl] += d[i];
        if constexpr (K::cy < 0) sy[cl] -= d[i];
        if constexpr (K::cz > 0) sz[cl] += d[i];
        if constexpr (K::cz < 0) sz[cl] -= d[i];
    });
    constexpr int S0 = FFLink<L, ff_first_of_class<L, 0>()>::SHIFT, S1 = FFLink<L, ff_first_of_class<L, 1>()>::SHIFT,
                  S2 = FFLink<L, ff_first_of_class<L, 2>()>::SHIFT;
    const long long dr = k.dws + (sr[0] << S0) + (sr[1] << S1) + (sr[2] << S2);
    const long long jx = k.half_f[0] + (sx[1] << S1) + (sx[2] << S2);
    const long long jy = k.half_f[1] + (sy[1] << S1) + (sy[2] << S2);
    const long long jz = k.half_f[2] + (sz[1] << S1) + (sz[2] << S2);
    ok &= small_ll(dr, 55) & small_ll(jx, 56) & small_ll(jy, 56) & small_ll(jz, 56);
    if (!ok) return false;

    const ff DR = q60_to_ff(dr), JX = q60_to_ff(jx), JY = q60_to_ff(jy);
    const ff JZ = L::D == 3 ? q60_to_ff(jz) : ff{0.f, 0.f};
    ff RINV{1.f, 0.f};  // 1 / rho
    if constexpr (MODEL == LBM_QUASI_COMPRESSIBLE) {
        ff rho = fast2(1.f, DR.h);
        rho = fast2(rho.h, __fadd_rn(rho.l, DR.l));
        const float r0 = __frcp_rn(rho.h);
        // r = r0 + r0 (1 - rho r0), with 1 - rho r0 formed exactly enough
        const float p = __fmul_rn(rho.h, r0);
        const float pe = __fmaf_rn(rho.h, r0, -p);
        const float er = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p), pe), __fmul_rn(rho.l, r0));
        RINV = fast2(r0, __fmul_rn(r0, er));
    }
    // gamma = 1.5 w |p|^2 + 3 (1 - w/2) p.F, p = j + F/2
    // (sums that feed a product are renormalised, the others are lazy)
    const ff jj = ff_add(ff_add_lazy(ff_sqr(JX), ff_sqr(JY)), ff_sqr(JZ));
    const ff gamma = ff_add(ff_mul(jj, ff_c(c.g1)),
                            ff_add_lazy(ff_add_lazy(ff_mul(JX, ff_c(c.kf[0])), ff_mul(JY, ff_c(c.kf[1]))),
                                        ff_mul(JZ, ff_c(c.kf[2]))));
    // per class, in units of ulp(w_c): V = w_c / rho, C = w w_c drho - gamma V,
    // formed at the first link of the class (links come class by class)
    ff V{0.f, 0.f}, C{0.f, 0.f};
    const ff KEEP = ff_c(c.keep);
    // (1 - w) g_i in ulps: g_i = d_i ulp(w_i), d_i split into exact 24-bit halves
    auto kept = [&](auto I) {
        constexpr int i = decltype(I)::value;
        const ff g{__fmul_rn(__int2float_rn((int)(d[i] >> 24)), pow2f(24)), __int2float_rn((int)(d[i] & 0xFFFFFF))};
        return ff_mul(g, KEEP);
    };
    auto store = [&](auto I, ff x) {
        constexpr int i = decltype(I)::value;
        out[i * stride] = ulp_round(x, (unsigned long long)k.w_bits[Link<L, i>::cls], ok);
    };
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        if constexpr (i == ff_first_of_class<L, K::cls>()) {
            V = MODEL == LBM_QUASI_COMPRESSIBLE ? ff_mul(RINV, ff_c(c.w[K::cls])) : ff_c(c.w[K::cls]);
            C = ff_add_lazy(ff_mul(DR, ff_c(c.rho[K::cls])), ff_neg(ff_mul(gamma, V)));
        }
        if constexpr (i == 0) {
            const ff x = ff_add_lazy(kept(I), C);
            store(I, x);
        } else if constexpr (i < K::opp) {
            constexpr int j = K::opp;
            constexpr int cl = K::cls;
            // y = c_i . p
            ff Y{0.f, 0.f};
            bool first = true;
            auto acc = [&](int sgn, const ff& JA) {
                const ff t = sgn > 0 ? JA : ff_neg(JA);
                Y = first ? t : ff_add(Y, t);
                first = false;
            };
            if constexpr (K::cx != 0) acc(K::cx, JX);
            if constexpr (K::cy != 0) acc(K::cy, JY);
            if constexpr (K::cz != 0) acc(K::cz, JZ);
            // symmetric part E = C + y (4.5 w y + 9 (1 - w/2) c_i.F) V, antisymmetric part
            // O = 3 w w_c y + 3 (1 - w/2) w_c c_i.F (all in ulps of w_c)
            const ff T = ff_mul(Y, ff_add(ff_mul(Y, ff_c(c.alpha)), ff_c(c.beta[i])));
            const ff E = ff_add_lazy(C, ff_mul(T, V));
            const ff O = ff_add_lazy(ff_mul(Y, ff_c(c.j[cl])), ff_c(c.so[i]));
            store(I, ff_sum3(kept(I), E, O));
            store(std::integral_constant<int, j>{}, ff_sum3(kept(std::integral_constant<int, j>{}), E, ff_neg(O)));
        }
    });
    return ok;
}

}  // namespace lbm

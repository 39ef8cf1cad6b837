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

// x + y renormalised (the low part within half an ulp of the high part);
// products return (p, e) with |e| within a few ulps of p, which every
// consumer accepts, saving a two-sum per product.
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    const ff s = two_sum(x.h, y.h);
    return fast2(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}

// x + y without the final renormalisation.  The value is as accurate as
// ff_add's, but after cancellation the low part may exceed half an ulp of the
// high part: it stays within about 1.5 ulps of the larger operand's high
// part.  A product then evaluates that low part in single precision, an
// error of about 2^-47 times the operands' magnitudes, the same order as a
// float-float product's own rounding; every sum of the collision that feeds
// a product or a further sum is taken this way (the results are rounded to
// FP64 in units of ulp(w), where such errors are a small fraction of a unit).
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
// part (not renormalised: ulp_round takes any low part below 1.5 2^24).
__device__ __forceinline__ ff ff_sum3(ff a, ff b, ff c) {
    const ff s = two_sum(a.h, b.h);
    const ff t = two_sum(s.h, c.h);
    return ff{t.h, __fadd_rn(__fadd_rn(__fadd_rn(a.l, b.l), __fadd_rn(c.l, s.l)), t.l)};
}

// FP64 bit pattern of w + r ulp(w) with r within one unit of x = x.h + x.l
// (units of ulp(w)).  x.h is split at 2^24 by rounding it to the nearest
// multiple of 2^24 with one addition: t = x.h + 1.5 2^47 lies in [2^47, 2^48)
// for |x.h| < 2^46, where the floats are the multiples of 2^24, so
// bits(t) - bits(1.5 2^47) counts them and the remainder rem = x.h - (t -
// 1.5 2^47) is exact (|rem| <= 2^23).  With |x.l| < 1.5 2^24 (the low part of
// keep d_i alone reaches 2^24 near equilibrium: d_i's low piece is not
// centred), |rem + x.l| < 2^25: below 2^24 its float sum and the conversion to
// an integer are each within 1/2, at or above 2^24 the sum is already an
// integer within 1; so r = (t - 1.5 2^47) + RN_int(rem + x.l) is within one
// unit of x.  (A truncating split would take three FP32 <-> int conversions
// per value, which issue at a fraction of the FP32 rate; one conversion of the
// summed remainder instead of one per part measured 1 % faster.)
//
// The result stays in the binade of w (same sign and exponent bits): |r| <
// 2^46 + 2^26 ulps, and every lattice weight lies at least 2^48 ulps from
// the edges of its binade (checked at compile time in collide_ff).
constexpr float kLowBound = 25165824.0f;  // 1.5 * 2^24
constexpr float kSplit24 = 211106232532992.0f;  // 1.5 * 2^47: floats in [2^47, 2^48) are multiples of 2^24
__device__ __forceinline__ unsigned long long ulp_assemble(unsigned long long wb, float t, int lo) {
    const long long k = (long long)wb - ((long long)__float_as_int(kSplit24) << 24);
    return (unsigned long long)(k + ((long long)(unsigned)__float_as_int(t) << 24) + (long long)lo);
}

__device__ __forceinline__ unsigned long long ulp_round(ff x, unsigned long long wb, bool& ok) {
    ok &= fabsf(x.h) < pow2f(46) && fabsf(x.l) < kLowBound;
    const float t = __fadd_rn(x.h, kSplit24);
    const float rem = __fsub_rn(x.h, __fsub_rn(t, kSplit24));  // exact, |rem| <= 2^23
    return ulp_assemble(wb, t, __float2int_rn(__fadd_rn(rem, x.l)));  // |rem + x.l| < 2^25
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

// update_fp64 for the steps that stage neighbour records (gather_rec).
template <class L, int A, int MODEL, int KMAX>
__device__ __noinline__ void update_fp64_rec(const RecShared<Tile<L, A>, KMAX>& sh, const StepArgs& a,
                                             const WorkNode& wn, const NodePos<A>& p) {
    unsigned long long b[L::Q];
    int stride;
    unsigned long long* out = gather_rec<L, A, KMAX, unsigned long long>(sh, a.src, a.dst, wn.lt, wn.node, p, b, stride);
    double f[L::Q];
    static_for<0, L::Q>([&](auto I) { f[decltype(I)::value] = __longlong_as_double((long long)b[decltype(I)::value]); });
    collide_f64<L, MODEL>(f, a.omega, a.force);
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        out[i * stride] = (unsigned long long)__double_as_longlong(f[i]);
    });
}

// ---- two float-float numbers at once (f32x2) ------------------------------------
// sm_100-family GPUs issue two FP32 additions, multiplications or fused
// multiply-adds in one instruction (add/sub/mul/fma .f32x2).  The collision
// below evaluates its float-float arithmetic two lanes at a time: two pairs
// of opposite links, or the two links of one pair.  Every lane performs the
// operations of the scalar helpers above, in the same order, so the results
// are the same bits.
struct ff2 {
    float2 h, l;
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 a, b, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "sub.rn.f32x2 r, a, b;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

__device__ __forceinline__ ff2 pack2(ff a, ff b) { return ff2{make_float2(a.h, b.h), make_float2(a.l, b.l)}; }
__device__ __forceinline__ ff lane0(ff2 x) { return ff{x.h.x, x.l.x}; }
__device__ __forceinline__ ff lane1(ff2 x) { return ff{x.h.y, x.l.y}; }
__device__ __forceinline__ ff2 ff2_neg(ff2 x) { return ff2{neg2(x.h), neg2(x.l)}; }

__device__ __forceinline__ ff2 fast2_2(float2 a, float2 b) {
    const float2 s = add2(a, b);
    return ff2{s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ ff2 two_sum_2(float2 a, float2 b) {
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    return ff2{s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}

__device__ __forceinline__ ff2 ff_add_lazy_2(ff2 x, ff2 y) {
    const ff2 s = two_sum_2(x.h, y.h);
    return ff2{s.h, add2(s.l, add2(x.l, y.l))};
}

__device__ __forceinline__ ff2 ff_mul_2(ff2 x, ff2 y) {
    const float2 p = mul2(x.h, y.h);
    float2 e = fma2(x.h, y.h, neg2(p));
    e = fma2(x.h, y.l, e);
    e = fma2(x.l, y.h, e);
    return ff2{p, e};
}

__device__ __forceinline__ ff2 ff_sqr_2(ff2 x) {
    const float2 p = mul2(x.h, x.h);
    float2 e = fma2(x.h, x.h, neg2(p));
    e = fma2(mul2(bc2(2.f), x.h), x.l, e);
    return ff2{p, e};
}

__device__ __forceinline__ ff2 ff_sum3_2(ff2 a, ff2 b, ff2 c) {
    const ff2 s = two_sum_2(a.h, b.h);
    const ff2 t = two_sum_2(s.h, c.h);
    return ff2{t.h, add2(add2(add2(a.l, b.l), add2(c.l, s.l)), t.l)};
}

__device__ __forceinline__ ff2 ff2_c(const float2 ka, const float2 kb) {
    return ff2{make_float2(ka.x, kb.x), make_float2(ka.y, kb.y)};
}
__device__ __forceinline__ ff2 ff2_bc(const ff k) { return ff2{bc2(k.h), bc2(k.l)}; }
__device__ __forceinline__ ff2 ff2_k(const FF2C& k) { return ff2{k.h, k.l}; }

// q60_to_ff of two values.
__device__ __forceinline__ ff2 q60_to_ff_2(long long a, long long b) {
    const float2 f2 = mul2(make_float2(__int2float_rn((int)(a >> 48)), __int2float_rn((int)(b >> 48))),
                           bc2(pow2f(-12)));
    const float2 f1 = mul2(make_float2(__int2float_rn((int)((a >> 24) & 0xFFFFFF)),
                                       __int2float_rn((int)((b >> 24) & 0xFFFFFF))),
                           bc2(pow2f(-36)));
    const float2 f0 = mul2(make_float2(__int2float_rn((int)(a & 0xFFFFFF)), __int2float_rn((int)(b & 0xFFFFFF))),
                           bc2(pow2f(-60)));
    const ff2 s = fast2_2(f2, f1);
    return fast2_2(s.h, add2(s.l, f0));
}

// d_i (ulps of w_i) of two links as exact float-float pieces (see kept in the
// scalar form: two 24-bit halves).
__device__ __forceinline__ ff2 d_to_ff_2(long long a, long long b) {
    const float2 h = mul2(make_float2(__int2float_rn((int)(a >> 24)), __int2float_rn((int)(b >> 24))),
                          bc2(pow2f(24)));
    return ff2{h, make_float2(__int2float_rn((int)(a & 0xFFFFFF)), __int2float_rn((int)(b & 0xFFFFFF)))};
}

// ulp_round of two results (bit patterns of two links of weight bits wa, wb).
__device__ __forceinline__ void ulp_round_2(ff2 x, unsigned long long wa, unsigned long long wb, bool& ok,
                                            unsigned long long& oa, unsigned long long& ob) {
    ok &= fabsf(x.h.x) < pow2f(46) && fabsf(x.l.x) < kLowBound && fabsf(x.h.y) < pow2f(46) &&
          fabsf(x.l.y) < kLowBound;
    const float2 t = add2(x.h, bc2(kSplit24));
    const float2 rem = sub2(x.h, sub2(t, bc2(kSplit24)));  // exact, |rem| <= 2^23
    const float2 lo = add2(rem, x.l);                        // see ulp_round
    oa = ulp_assemble(wa, t.x, __float2int_rn(lo.x));
    ob = ulp_assemble(wb, t.y, __float2int_rn(lo.y));
}

// The pair of opposite links that starts at link I (I < opp(I)).
template <class L, int I>
struct FFPair {
    using K = Link<L, I>;
    static constexpr int i = I, j = K::opp, cls = K::cls;
    static constexpr int n_comp = (K::cx != 0) + (K::cy != 0) + (K::cz != 0);
    // k-th nonzero component of c_i: axis (0..2) and sign
    static constexpr int axis(int k) {
        int a = 0, n = 0;
        const int c[3] = {K::cx, K::cy, K::cz};
        for (a = 0; a < 3; a++)
            if (c[a] != 0 && n++ == k) return a;
        return -1;
    }
    static constexpr int sign(int k) {
        const int c[3] = {K::cx, K::cy, K::cz};
        return c[axis(k)];
    }
};

// The first links of the pairs of opposite links, in link order, grouped two
// by two when both pairs have the same number of nonzero components (and so
// the same sequence of operations); a pair left alone packs its two links.
// FAX >= 0: the body force lies along axis FAX (or is zero), so the pairs
// with c_i . F = 0 carry no forcing terms (beta_i = so_i = 0); they are
// grouped together (nob[g]) and skip those terms.  A group that keeps its
// forcing terms holds the same pairs as in the general grouping (FAX = -1),
// whose per-group constants it reads; the lone pair reads per-link ones.
template <class L, int FAX = -1>
struct FFGroups;
template <int FAX>
struct FFGroups<D2Q9, FAX> {
    static_assert(FAX == -1, "D2Q9 takes the general grouping");
    static constexpr int n = 2;
    static constexpr int a[2] = {1, 5}, b[2] = {2, 6};
    static constexpr bool nob[2] = {false, false};
    static constexpr int lone = -1;
};
template <>
struct FFGroups<D3Q19, -1> {
    static constexpr int n = 4;
    static constexpr int a[4] = {1, 7, 11, 15}, b[4] = {3, 9, 13, 17};
    static constexpr bool nob[4] = {false, false, false, false};
    static constexpr int lone = 5;
};
template <>
struct FFGroups<D3Q19, 0> {  // F along x: (3,4)+(5,6) and (15,16)+(17,18) unforced
    static constexpr int n = 4;
    static constexpr int a[4] = {3, 7, 11, 15}, b[4] = {5, 9, 13, 17};
    static constexpr bool nob[4] = {true, false, false, true};
    static constexpr int lone = 1;
};
template <>
struct FFGroups<D3Q19, 1> {  // F along y: (1,2)+(5,6) and (11,12)+(13,14) unforced
    static constexpr int n = 4;
    static constexpr int a[4] = {1, 7, 11, 15}, b[4] = {5, 9, 13, 17};
    static constexpr bool nob[4] = {true, false, true, false};
    static constexpr int lone = 3;
};
template <>
struct FFGroups<D3Q19, 2> {  // F along z: (1,2)+(3,4) and (7,8)+(9,10) unforced
    static constexpr int n = 4;
    static constexpr int a[4] = {1, 7, 11, 15}, b[4] = {3, 9, 13, 17};
    static constexpr bool nob[4] = {true, true, false, false};
    static constexpr int lone = 5;
};

// Component of link I along axis X (0 for X < 0).
template <class L, int I, int X>
constexpr int link_comp() {
    return X == 0 ? Link<L, I>::cx : (X == 1 ? Link<L, I>::cy : (X == 2 ? Link<L, I>::cz : 0));
}

template <class L, int MODEL, int FAX = -1>
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
    // exact sums per class (units of ulp(w_c)), then one shift per class to
    // 2^-60; each pair of opposite links enters through its sum and difference
    long long sr[3] = {d[0], 0, 0}, sx[3] = {0, 0, 0}, sy[3] = {0, 0, 0}, sz[3] = {0, 0, 0};
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        if constexpr (i < K::opp) {
            constexpr int cl = K::cls;
            const long long sp = d[i] + d[K::opp], dp = d[i] - d[K::opp];
            sr[cl] += sp;
            if constexpr (K::cx > 0) sx[cl] += dp;
            if constexpr (K::cx < 0) sx[cl] -= dp;
            if constexpr (K::cy > 0) sy[cl] += dp;
            if constexpr (K::cy < 0) sy[cl] -= dp;
            if constexpr (K::cz > 0) sz[cl] += dp;
            if constexpr (K::cz < 0) sz[cl] -= dp;
        }
    });
    constexpr int S0 = FFLink<L, ff_first_of_class<L, 0>()>::SHIFT, S1 = FFLink<L, ff_first_of_class<L, 1>()>::SHIFT,
                  S2 = FFLink<L, ff_first_of_class<L, 2>()>::SHIFT;
    const long long dr = k.dws + (sr[0] << S0) + (sr[1] << S1) + (sr[2] << S2);
    const long long jx = k.half_f[0] + (sx[1] << S1) + (sx[2] << S2);
    const long long jy = k.half_f[1] + (sy[1] << S1) + (sy[2] << S2);
    const long long jz = k.half_f[2] + (sz[1] << S1) + (sz[2] << S2);
    ok &= small_ll(dr, 55) & small_ll(jx, 56) & small_ll(jy, 56) & small_ll(jz, 56);
    if (!ok) return false;

    // (j_x, j_y) side by side: the first group's c_i . p of its two pairs
    const ff2 JXY = q60_to_ff_2(jx, jy);
    const ff JX = lane0(JXY), JY = lane1(JXY);
    ff DR, JZ;
    if constexpr (L::D == 3) {
        const ff2 t = q60_to_ff_2(dr, jz);
        DR = lane0(t);
        JZ = lane1(t);
    } else {
        DR = q60_to_ff(dr);
        JZ = ff{0.f, 0.f};
    }
    const ff J[3] = {JX, JY, JZ};
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
    // gamma = 1.5 w |p|^2 + 3 (1 - w/2) p.F, p = j + F/2 (lazy sums, see
    // ff_add_lazy)
    ff gamma;
    {
        const ff2 sq = ff_sqr_2(JXY);
        const ff2 kfx = ff_mul_2(JXY, ff2_k(c.kf01));
        const ff jj = ff_add_lazy(ff_add_lazy(lane0(sq), lane1(sq)), ff_sqr(JZ));
        gamma = ff_add_lazy(ff_mul(jj, ff_c(c.g1)), ff_add_lazy(ff_add_lazy(lane0(kfx), lane1(kfx)), ff_mul(JZ, ff_c(c.kf[2]))));
    }
    // per class, in units of ulp(w_c): V = w_c / rho, C = w w_c drho - gamma V;
    // classes 1 and 2 in both lanes (each group of pairs is single-class), each
    // formed right before the links of its class
    const ff2 KEEP = ff2_k(c.keep2);
    const ff2 ALPHA = ff2_k(c.alpha2);
    // the rest link: (1 - w) g_0 + C_0
    {
        const ff V0 = MODEL == LBM_QUASI_COMPRESSIBLE ? ff_mul(RINV, ff_c(c.w[0])) : ff_c(c.w[0]);
        const ff C0 = ff_add_lazy(ff_mul(DR, ff_c(c.rho[0])), ff_neg(ff_mul(gamma, V0)));
        const ff g{__fmul_rn(__int2float_rn((int)(d[0] >> 24)), pow2f(24)), __int2float_rn((int)(d[0] & 0xFFFFFF))};
        const ff x = ff_add_lazy(ff_mul(g, ff_c(c.keep)), C0);
        out[0] = ulp_round(x, (unsigned long long)k.w_bits[0], ok);
    }
    auto class_consts = [&](const FF2C& wcc, const FF2C& rcc, ff2& VV, ff2& CC) {
        VV = MODEL == LBM_QUASI_COMPRESSIBLE ? ff_mul_2(ff2_bc(RINV), ff2_k(wcc)) : ff2_k(wcc);
        CC = ff_add_lazy_2(ff_mul_2(ff2_bc(DR), ff2_k(rcc)), ff2_neg(ff_mul_2(ff2_bc(gamma), VV)));
    };
    // two pairs of opposite links at once: lanes (pair A, pair B)
    using GR = FFGroups<L, FAX>;
    auto group = [&](auto G, const ff2& VV, const ff2& CC) {
        constexpr int g = decltype(G)::value;
        using PA = FFPair<L, GR::a[g]>;
        using PB = FFPair<L, GR::b[g]>;
        static_assert(PA::n_comp == PB::n_comp, "grouped pairs take the same operations");
        static_assert(PA::cls == PB::cls && PA::cls > 0, "a group takes one class of links");
        static_assert(GR::nob[g] ? (link_comp<L, GR::a[g], FAX>() == 0 && link_comp<L, GR::b[g], FAX>() == 0)
                                 : (GR::a[g] == FFGroups<L>::a[g] && GR::b[g] == FFGroups<L>::b[g]),
                      "an unforced group has c.F = 0; a forced one reads the general group's constants");
        // y = c_i . p
        auto comp = [&](auto Kc) {
            constexpr int kk = decltype(Kc)::value;
            const ff a = J[PA::axis(kk)], bb = J[PB::axis(kk)];
            return pack2(PA::sign(kk) > 0 ? a : ff_neg(a), PB::sign(kk) > 0 ? bb : ff_neg(bb));
        };
        ff2 Y = comp(std::integral_constant<int, 0>{});
        static_for<1, PA::n_comp>([&](auto Kc) { Y = ff_add_lazy_2(Y, comp(Kc)); });
        // without forcing terms the sums with beta = so = 0 are left out: adding
        // a zero float-float lazily returns its operand, so the bits are the
        // general grouping's
        ff2 T, O;
        if constexpr (GR::nob[g]) {
            T = ff_mul_2(Y, ff_mul_2(Y, ALPHA));
            O = ff_mul_2(Y, ff2_k(c.j2[g]));
        } else {
            T = ff_mul_2(Y, ff_add_lazy_2(ff_mul_2(Y, ALPHA), ff2_k(c.beta2[g])));
            O = ff_add_lazy_2(ff_mul_2(Y, ff2_k(c.j2[g])), ff2_k(c.so2[g]));
        }
        const ff2 E = ff_add_lazy_2(CC, ff_mul_2(T, VV));
        const ff2 xi = ff_sum3_2(ff_mul_2(d_to_ff_2(d[PA::i], d[PB::i]), KEEP), E, O);
        unsigned long long r0, r1;
        ulp_round_2(xi, (unsigned long long)k.w_bits[PA::cls], (unsigned long long)k.w_bits[PB::cls], ok, r0, r1);
        out[PA::i * stride] = r0;
        out[PB::i * stride] = r1;
        const ff2 xj = ff_sum3_2(ff_mul_2(d_to_ff_2(d[PA::j], d[PB::j]), KEEP), E, ff2_neg(O));
        ulp_round_2(xj, (unsigned long long)k.w_bits[PA::cls], (unsigned long long)k.w_bits[PB::cls], ok, r0, r1);
        out[PA::j * stride] = r0;
        out[PB::j * stride] = r1;
    };
    // a pair left alone: lanes (link i, link opp(i))
    auto lone = [&](auto LN, const ff2& VV, const ff2& CC) {
        using P = FFPair<L, decltype(LN)::value>;
        ff Y{0.f, 0.f};
        static_for<0, P::n_comp>([&](auto Kc) {
            constexpr int kk = decltype(Kc)::value;
            const ff t = P::sign(kk) > 0 ? J[P::axis(kk)] : ff_neg(J[P::axis(kk)]);
            Y = kk == 0 ? t : ff_add_lazy(Y, t);
        });
        const ff T = ff_mul(Y, ff_add_lazy(ff_mul(Y, ff_c(c.alpha)), ff_c(c.beta[P::i])));
        const ff E = ff_add_lazy(lane0(CC), ff_mul(T, lane0(VV)));
        const ff O = ff_add_lazy(ff_mul(Y, ff_c(c.j[P::cls])), ff_c(c.so[P::i]));
        const ff2 x = ff_sum3_2(ff_mul_2(d_to_ff_2(d[P::i], d[P::j]), KEEP), ff2_bc(E), pack2(O, ff_neg(O)));
        unsigned long long r0, r1;
        ulp_round_2(x, (unsigned long long)k.w_bits[P::cls], (unsigned long long)k.w_bits[P::cls], ok, r0, r1);
        out[P::i * stride] = r0;
        out[P::j * stride] = r1;
    };
    static_assert(GR::lone < 0 || Link<L, (GR::lone > 0 ? GR::lone : 1)>::cls == 1, "the lone pair is of class 1");
    {  // class 1: the first group and the lone pair
        ff2 VV, CC;
        class_consts(c.w11, c.rho11, VV, CC);
        // (the order only moves register pressure: with a force axis the lone
        // pair first spilled less and measured 2 % faster, in general last)
        if constexpr (FAX >= 0 && GR::lone > 0) lone(std::integral_constant<int, GR::lone>{}, VV, CC);
        group(std::integral_constant<int, 0>{}, VV, CC);
        if constexpr (FAX < 0 && GR::lone > 0) lone(std::integral_constant<int, GR::lone>{}, VV, CC);
    }
    {  // class 2: the other groups
        ff2 VV, CC;
        class_consts(c.w22, c.rho22, VV, CC);
        static_for<1, GR::n>([&](auto G) { group(G, VV, CC); });
    }
    return ok;
}

}  // namespace lbm

// nodes.cu -- kernels that visit every node of every non-empty tile once:
// equilibrium start, moments with FP64 reductions, and dense export/import
// of the PDFs.  None of them is on the per-step path.
#include <cmath>

#include "collide_ff.cuh"

namespace lbm {

constexpr int kStats = 8;  // mass, momentum x/y/z, |u|^2, |u - u_saved|^2, fluid count, spare
constexpr int kMomentGroups = 8;  // tile groups per block of the moments kernel

template <class L, int A>
__device__ __forceinline__ bool dense_index(const NodeArgs& a, int tile, const NodePos<A>& p, size_t& n) {
    const int x = __ldg(a.coords + 3 * tile) * A + p.lx;
    const int y = __ldg(a.coords + 3 * tile + 1) * A + p.ly;
    const int z = __ldg(a.coords + 3 * tile + 2) * A + p.lz;
    if (x >= a.nx || y >= a.ny || z >= a.nz) return false;
    n = (size_t)x + (size_t)a.nx * ((size_t)y + (size_t)a.ny * z);
    return true;
}

template <class TL>
__device__ __forceinline__ bool own_fluid(const uint64_t* __restrict__ tmask, int tile, int node) {
    return (__ldg(tmask + (size_t)tile * TL::W + (node >> 6)) >> (node & 63)) & 1ull;
}

// ---- equilibrium start ---------------------------------------------------------
template <class L, int A, int MODEL, class S>
__global__ void k_init(const NodeArgs a) {
    using TL = Tile<L, A>;
    using T = typename S::T;
    if ((int)blockIdx.x >= a.n_tiles) return;
    const int tile = a.tile_begin + blockIdx.x;
    const int node = threadIdx.x;
    const NodePos<A> p = node_pos<TL>(node);
    size_t n = 0;
    if (!own_fluid<TL>(a.tmask, tile, node) || !dense_index<L, A>(a, tile, p, n)) return;
    const int stride = a.tile_stride[tile];
    T* out = static_cast<T*>(const_cast<void*>(a.pdf)) + a.tile_off[tile] +
             fluid_rank<TL::W>(a.tmask + (size_t)tile * TL::W, node);
    if (!a.rho_in && !a.u_in) {  // the rest start: f^eq_i = w_i rho0 (Eq. 3 and Eq. 4 alike)
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            out[i * stride] = S::template from_f64<L, i>(Link<L, i>::w * a.rho0, a.f16_scale);
        });
        return;
    }
    const double rho = a.rho_in ? a.rho_in[n] : a.rho0;
    const size_t N = (size_t)a.nx * a.ny * a.nz;
    const double ux = a.u_in ? a.u_in[n] : 0.0;
    const double uy = a.u_in ? a.u_in[N + n] : 0.0;
    const double uz = a.u_in && L::D == 3 ? a.u_in[2 * N + n] : 0.0;
    const double usq = ux * ux + uy * uy + uz * uz;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        const double cu = K::cx * ux + K::cy * uy + K::cz * uz;
        const double poly = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq;
        const double feq = MODEL == LBM_QUASI_COMPRESSIBLE ? K::w * rho * (1.0 + poly) : K::w * (rho + poly);
        out[i * stride] = S::template from_f64<L, i>(feq, a.f16_scale);
    });
}

// ---- moments and reductions ---------------------------------------------------------
// The moments (Eq. 5; Eq. 6 for the incompressible model) of every fluid node
// are formed without FP64 instructions, which GB300 issues at a small
// fraction of its FP32 rate: FP64 words in the exact range of the float-float
// step give rho - 1 and j as exact integer sums (units of 2^-60), every other
// form sums its deviations f_i - w_i in float-float; u = (j + F/2) / rho
// follows in float-float.  A node whose FP64 words fall outside that range
// (or are not finite) takes the FP64 formulas.  Each thread accumulates its
// nodes of kMomentGroups tile groups in float-float, and the block sums its
// threads in a fixed order; the per-block partials are FP64.

__device__ __forceinline__ ff ff_of(double v) {
    const float h = __double2float_rn(v);
    return ff{h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double dbl_of(ff x) { return (double)x.h + (double)x.l; }

// x + y for a float y, low part not renormalised (callers renormalise once).
__device__ __forceinline__ ff ff_acc(ff x, float y) {
    const ff s = two_sum(x.h, y);
    return ff{s.h, __fadd_rn(x.l, s.l)};
}
__device__ __forceinline__ ff ff_norm(ff x) { return fast2(x.h, x.l); }

template <class L>
constexpr long long q60_weight_excess() {  // sum_i w_i in units of 2^-60, minus 2^60 (exact)
    long long s = 0;
    for (int i = 0; i < L::Q; i++) s += (long long)(L::wc_[L::cls_[i]] * 1152921504606846976.0);
    return s - (1ll << 60);
}

// rho - 1 and j (before the force) from FP64 words; false when a word is
// outside the exact range (the caller then takes the FP64 formulas).
template <class L>
__device__ __forceinline__ bool moments_words(const unsigned long long (&b)[L::Q], ff& dr, ff& jx, ff& jy, ff& jz) {
    long long sr[3] = {0, 0, 0}, sx[3] = {0, 0, 0}, sy[3] = {0, 0, 0}, sz[3] = {0, 0, 0};
    bool ok = true;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        constexpr int cl = K::cls;
        const long long d = (long long)(b[i] - (unsigned long long)__double_as_longlong(K::w));
        ok &= within_2p47(d);
        sr[cl] += d;
        if constexpr (K::cx > 0) sx[cl] += d;
        if constexpr (K::cx < 0) sx[cl] -= d;
        if constexpr (K::cy > 0) sy[cl] += d;
        if constexpr (K::cy < 0) sy[cl] -= d;
        if constexpr (K::cz > 0) sz[cl] += d;
        if constexpr (K::cz < 0) sz[cl] -= d;
    });
    constexpr int S0 = FFLink<L, ff_first_of_class<L, 0>()>::SHIFT, S1 = FFLink<L, ff_first_of_class<L, 1>()>::SHIFT,
                  S2 = FFLink<L, ff_first_of_class<L, 2>()>::SHIFT;
    const long long r = q60_weight_excess<L>() + (sr[0] << S0) + (sr[1] << S1) + (sr[2] << S2);
    const long long x = (sx[1] << S1) + (sx[2] << S2), y = (sy[1] << S1) + (sy[2] << S2);
    const long long z = (sz[1] << S1) + (sz[2] << S2);
    ok &= small_ll(r, 56) & small_ll(x, 56) & small_ll(y, 56) & small_ll(z, 56);
    dr = q60_to_ff(r);
    jx = q60_to_ff(x);
    jy = q60_to_ff(y);
    jz = L::D == 3 ? q60_to_ff(z) : ff{0.f, 0.f};
    return ok;
}

// The same from FP32 / FP16 words: float-float sums of the deviations (FP32
// values: of f_i itself, less sum_i w_i = 1 at the end).
template <class L, class S>
__device__ __forceinline__ void moments_words(const typename S::T (&raw)[L::Q], const NodeArgs& a, ff& dr, ff& jx,
                                              ff& jy, ff& jz) {
    ff r{0.f, 0.f}, x{0.f, 0.f}, y{0.f, 0.f}, z{0.f, 0.f};
    const float inv_scale = (float)a.f16_inv_scale;  // a power of two
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using K = Link<L, i>;
        float g;
        if constexpr (S::id == LBM_STORE_F16S)
            g = __half2float(__ushort_as_half(raw[i])) * inv_scale;
        else
            g = __uint_as_float(raw[i]);
        r = ff_acc(r, g);
        if constexpr (K::cx > 0) x = ff_acc(x, g);
        if constexpr (K::cx < 0) x = ff_acc(x, -g);
        if constexpr (K::cy > 0) y = ff_acc(y, g);
        if constexpr (K::cy < 0) y = ff_acc(y, -g);
        if constexpr (K::cz > 0) z = ff_acc(z, g);
        if constexpr (K::cz < 0) z = ff_acc(z, -g);
    });
    r = ff_norm(r);
    if constexpr (S::id == LBM_STORE_F32) r = ff_add(r, ff{-1.f, 0.f});
    dr = r;
    jx = ff_norm(x);
    jy = ff_norm(y);
    jz = ff_norm(z);
}

template <class L, int A, int TPB, int MODEL, class S>
__global__ void __launch_bounds__(TPB* Tile<L, A>::NT, TPB* Tile<L, A>::NT > 256 ? 1 : (S::id == LBM_STORE_F64 ? 2 : 3))
    k_moments(const NodeArgs a) {
    using TL = Tile<L, A>;
    using T = typename S::T;
    constexpr int NTH = TPB * TL::NT;
    constexpr int PER_TILE = TL::NN * TL::W;
    static_assert(TPB * PER_TILE <= NTH, "one neighbourhood entry per thread at most");
    __shared__ NeighShared<TL, TPB> sh[2];
    __shared__ double red[NTH / 32][kStats];
    const int lt = threadIdx.x / TL::NT;
    const int node = threadIdx.x - lt * TL::NT;
    const int tile_end = a.tile_begin + a.n_tiles;
    const int n_groups = (a.n_tiles + TPB - 1) / TPB;
    const NodePos<A> p = node_pos<TL>(node);
    const bool want_fields = a.rho_out || a.u_out;
    const size_t N = (size_t)a.nx * a.ny * a.nz;  // fields only for a single-sample launch
    const ff half_f[3] = {ff_of(0.5 * a.force[0]), ff_of(0.5 * a.force[1]), ff_of(L::D == 3 ? 0.5 * a.force[2] : 0.0)};
    ff acc_dr{0.f, 0.f}, acc_m[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, acc_u2{0.f, 0.f}, acc_du2{0.f, 0.f};
    int count = 0;

    // The neighbourhood of the next tile group is staged while this one is
    // worked on (two buffers): this thread's entry e = (tile, slot, word) is
    // read as the neighbour index two groups ahead and as the neighbour's
    // record one group ahead, so no round trip to memory stands between two
    // groups.
    const int e = threadIdx.x;
    const bool has_entry = e < TPB * PER_TILE;
    const int e_lt = e / PER_TILE, e_rem = e - e_lt * PER_TILE;
    const int e_slot = e_rem / TL::W, e_w = e_rem - e_slot * TL::W;
    auto load_nb = [&](int g) {
        const int t = a.tile_begin + g * TPB + e_lt;
        return has_entry && t < tile_end ? __ldg(a.nbr + (size_t)t * TL::NN + e_slot) : -1;
    };
    auto load_rec = [&](int nb) {
        if (nb < 0) return make_ulonglong2(0ull, 0ull);
        if (e_w == 0) return __ldg(a.tinfo + nb);
        return make_ulonglong2(__ldg(a.tmask + (size_t)nb * TL::W + e_w), 0ull);
    };
    auto store = [&](NeighShared<TL, TPB>& s, const ulonglong2 r, long long origin) {
        if (e == 0) s.origin = origin;
        if (!has_entry) return;
        s.m[e_lt][e_slot][e_w] = r.x;
        if (e_w == 0)
            s.loc[e_lt][e_slot] = r.y ? make_int2((int)((long long)(r.y >> 24) - origin), (int)(r.y & 0xFFFFFFull))
                                      : make_int2(0, 0);
    };
    const int g0 = blockIdx.x * kMomentGroups;
    const int g_end = min(n_groups, g0 + kMomentGroups);
    if (g0 < g_end) store(sh[0], load_rec(load_nb(g0)), __ldg(a.tile_off + a.tile_begin + g0 * TPB));
    int nb_next = g0 + 1 < g_end ? load_nb(g0 + 1) : -1;
    __syncthreads();
    for (int g = g0; g < g_end; g++) {
        NeighShared<TL, TPB>& cur = sh[(g - g0) & 1];
        const bool more = g + 1 < g_end;
        ulonglong2 rec_next = make_ulonglong2(0ull, 0ull);
        long long origin_next = 0;
        if (more) {
            rec_next = load_rec(nb_next);
            origin_next = __ldg(a.tile_off + a.tile_begin + (g + 1) * TPB);
        }
        const int nb_after = g + 2 < g_end ? load_nb(g + 2) : -1;
        const int tile = a.tile_begin + g * TPB + lt;
        size_t n = 0;
        if (tile < tile_end && mask_bit(cur, lt, TL::CENTER, node) && (!want_fields || dense_index<L, A>(a, tile, p, n))) {
            T raw[L::Q];
            const int rank = gather<L, A, TPB, T>(cur, a.pdf, lt, node, p, raw);
            const long long slot = (cur.origin + cur.loc[lt][TL::CENTER].x) / L::Q + rank;
            float2 prev[3];
            float2* us = a.residual && a.u_saved ? a.u_saved + slot : nullptr;
            if (us) {
#pragma unroll
                for (int k = 0; k < 3; k++) prev[k] = us[k * a.n_slots];
            }
            ff dr, j[3], u[3];
            bool exact = true;
            if constexpr (S::id == LBM_STORE_F64)
                exact = moments_words<L>(raw, dr, j[0], j[1], j[2]);
            else
                moments_words<L, S>(raw, a, dr, j[0], j[1], j[2]);
            if (exact) {
#pragma unroll
                for (int k = 0; k < 3; k++) j[k] = ff_add(j[k], half_f[k]);  // j + F/2
                if constexpr (MODEL == LBM_QUASI_COMPRESSIBLE) {
                    // 1 / rho as in the float-float step
                    ff rho = fast2(1.f, dr.h);
                    rho = fast2(rho.h, __fadd_rn(rho.l, dr.l));
                    const float r0 = __frcp_rn(rho.h);
                    const float pr = __fmul_rn(rho.h, r0);
                    const float pe = __fmaf_rn(rho.h, r0, -pr);
                    const float er = __fsub_rn(__fsub_rn(__fsub_rn(1.f, pr), pe), __fmul_rn(rho.l, r0));
                    const ff rinv = fast2(r0, __fmul_rn(r0, er));
#pragma unroll
                    for (int k = 0; k < 3; k++) u[k] = ff_norm(ff_mul(j[k], rinv));
                } else {
#pragma unroll
                    for (int k = 0; k < 3; k++) u[k] = j[k];
                }
            } else {  // outside the exact range, or not finite: the FP64 formulas
                double f[L::Q];
                static_for<0, L::Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    f[i] = S::template to_f64<L, i>(raw[i], a.f16_inv_scale);
                });
                double rho, jx, jy, jz, ux, uy, uz;
                moments_f64<L>(f, rho, jx, jy, jz);
                velocity_f64<L, MODEL>(rho, jx, jy, jz, a.force, ux, uy, uz);
                dr = ff_of(rho - 1.0);
                j[0] = ff_of(jx + 0.5 * a.force[0]);
                j[1] = ff_of(jy + 0.5 * a.force[1]);
                j[2] = ff_of(jz + 0.5 * a.force[2]);
                u[0] = ff_of(ux);
                u[1] = ff_of(uy);
                u[2] = ff_of(uz);
            }
            if (a.rho_out) a.rho_out[n] = 1.0 + dbl_of(dr);
            if (a.u_out) {
                a.u_out[n] = dbl_of(u[0]);
                a.u_out[N + n] = dbl_of(u[1]);
                if (L::D == 3) a.u_out[2 * N + n] = dbl_of(u[2]);
            }
            acc_dr = ff_add(acc_dr, dr);
            // momentum rho u: j + F/2 (Eq. 5); rho (j + F/2) for the incompressible u (Eq. 6)
#pragma unroll
            for (int k = 0; k < 3; k++)
                acc_m[k] = ff_add(acc_m[k], MODEL == LBM_QUASI_COMPRESSIBLE ? j[k] : ff_mul(fast2(1.f, dr.h), j[k]));
            acc_u2 = ff_acc(acc_u2, __fmaf_rn(u[0].h, u[0].h, __fmaf_rn(u[1].h, u[1].h, __fmul_rn(u[2].h, u[2].h))));
            if (us) {
                float du2 = 0.f;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const float d = ff_add(u[k], ff{-prev[k].x, -prev[k].y}).h;
                    du2 = __fmaf_rn(d, d, du2);
                    us[k * a.n_slots] = make_float2(u[k].h, u[k].l);
                }
                acc_du2 = ff_acc(acc_du2, du2);
            }
            count++;
        }
        if (more) store(sh[(g + 1 - g0) & 1], rec_next, origin_next);
        nb_next = nb_after;
        __syncthreads();  // the next group's neighbourhood is staged; this one's buffer is free
    }
    // deterministic block sum: float-float butterfly within each warp, then warps in order
    ff v[6] = {acc_dr, acc_m[0], acc_m[1], acc_m[2], ff_norm(acc_u2), ff_norm(acc_du2)};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < 6; k++)
            v[k] = ff_add(v[k], ff{__shfl_xor_sync(0xffffffffu, v[k].h, off), __shfl_xor_sync(0xffffffffu, v[k].l, off)});
        count += __shfl_xor_sync(0xffffffffu, count, off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[warp][0] = (double)count + dbl_of(v[0]);  // mass: sum of 1 + (rho - 1)
#pragma unroll
        for (int k = 1; k < 6; k++) red[warp][k] = dbl_of(v[k]);
        red[warp][6] = (double)count;
        red[warp][7] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x < kStats) {
        double s = 0.0;
        for (int w = 0; w < NTH / 32; w++) s += red[w][threadIdx.x];
        a.partials[(size_t)blockIdx.x * kStats + threadIdx.x] = s;
    }
}

// One block sums the per-block partials in a fixed order.
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ partials, int nblocks,
                                               double* __restrict__ result) {
    __shared__ double sm[256][kStats];
    double acc[kStats];
#pragma unroll
    for (int k = 0; k < kStats; k++) acc[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256)
#pragma unroll
        for (int k = 0; k < kStats; k++) acc[k] += partials[(size_t)b * kStats + k];
#pragma unroll
    for (int k = 0; k < kStats; k++) sm[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < kStats; k++) sm[threadIdx.x][k] += sm[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x < kStats) result[threadIdx.x] = sm[0][threadIdx.x];
}

// ---- dense export / import ----------------------------------------------------------
template <class L, int A, class S>
__global__ void k_export(const NodeArgs a) {
    using TL = Tile<L, A>;
    using T = typename S::T;
    if ((int)blockIdx.x >= a.n_tiles) return;
    const int tile = a.tile_begin + blockIdx.x, node = threadIdx.x;
    if (!own_fluid<TL>(a.tmask, tile, node)) return;
    const NodePos<A> p = node_pos<TL>(node);
    size_t n;
    if (!dense_index<L, A>(a, tile, p, n)) return;
    const size_t N = (size_t)a.nx * a.ny * a.nz;
    const int stride = a.tile_stride[tile];
    const T* in = static_cast<const T*>(a.pdf) + a.tile_off[tile] +
                  fluid_rank<TL::W>(a.tmask + (size_t)tile * TL::W, node);
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        a.dense_pdf[i * N + n] = S::template to_f64<L, i>(in[i * stride], a.f16_inv_scale);
    });
}

template <class L, int A, class S>
__global__ void k_import(const NodeArgs a) {
    using TL = Tile<L, A>;
    using T = typename S::T;
    if ((int)blockIdx.x >= a.n_tiles) return;
    const int tile = a.tile_begin + blockIdx.x, node = threadIdx.x;
    if (!own_fluid<TL>(a.tmask, tile, node)) return;
    const NodePos<A> p = node_pos<TL>(node);
    size_t n;
    if (!dense_index<L, A>(a, tile, p, n)) return;
    const size_t N = (size_t)a.nx * a.ny * a.nz;
    const int stride = a.tile_stride[tile];
    T* out = static_cast<T*>(const_cast<void*>(a.pdf)) + a.tile_off[tile] +
             fluid_rank<TL::W>(a.tmask + (size_t)tile * TL::W, node);
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        out[i * stride] = S::template from_f64<L, i>(a.dense_pdf_in[i * N + n], a.f16_scale);
    });
}

// cur[k] = (cur[k] + prev[k]) / 2 over the raw words of one PDF copy.
__global__ void k_average_f64(double* __restrict__ cur, const double* __restrict__ prev, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        cur[k] = __dmul_rn(__dadd_rn(cur[k], prev[k]), 0.5);
}

__global__ void k_average_f32(float* __restrict__ cur, const float* __restrict__ prev, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        cur[k] = __fmul_rn(__fadd_rn(cur[k], prev[k]), 0.5f);
}

__global__ void k_average_f16(__half* __restrict__ cur, const __half* __restrict__ prev, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        cur[k] = __float2half_rn(0.5f * (__half2float(cur[k]) + __half2float(prev[k])));
}

__global__ void k_fill_nan(double* p, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        p[k] = __longlong_as_double(0x7ff8000000000000ll);
}

// ---- the step kernels' fluid-node list ---------------------------------------------------
// nodes[first(k) + r] = k * NT + node for the r-th fluid node of tile k (row
// order), first(k) = tile_off[k] / q (a tile's block holds q links of its nf
// fluid nodes): the list the host would build, written where the tables are.
template <class TL>
__global__ void k_node_list(const uint64_t* __restrict__ tmask, const long long* __restrict__ tile_off, int q,
                            uint32_t* __restrict__ nodes) {
    const int tile = blockIdx.x;
    const long long first = __ldg(tile_off + tile) / q;
    for (int node = threadIdx.x; node < TL::NT; node += blockDim.x) {
        if (!own_fluid<TL>(tmask, tile, node)) continue;
        const int r = fluid_rank<TL::W>(tmask + (size_t)tile * TL::W, node);
        nodes[first + r] = (uint32_t)tile * (uint32_t)TL::NT + (uint32_t)node;
    }
}

template <class L, int A>
cudaError_t launch_node_list(const uint64_t* tmask, const long long* tile_off, int n_tiles, uint32_t* nodes,
                             cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    constexpr int NT = Tile<L, A>::NT;
    k_node_list<Tile<L, A>><<<n_tiles, NT < 256 ? NT : 256, 0, s>>>(tmask, tile_off, L::Q, nodes);
    return cudaGetLastError();
}

NodeListLaunch select_node_list(int lattice, int a) {
    if (lattice == LBM_D2Q9) {
        if (a == 8) return &launch_node_list<D2Q9, 8>;
        if (a == 16) return &launch_node_list<D2Q9, 16>;
        if (a == 32) return &launch_node_list<D2Q9, 32>;
    } else if (lattice == LBM_D3Q19) {
        if (a == 4) return &launch_node_list<D3Q19, 4>;
        if (a == 8) return &launch_node_list<D3Q19, 8>;
    }
    return nullptr;
}

// ---- neighbour records on the device ------------------------------------------------
// nbr[k][slot] of compact tile k (coordinates coords[k]) for the 3^d slots
// (dx fastest, then dy, dz; offsets -1 .. +1): the compact index of the tile at
// coords + offset, wrapped on a periodic axis, -1 beyond a wall or where the
// tile was removed -- the host rule of build_tiling.
__global__ void k_build_nbr(const int32_t* __restrict__ coords, const int32_t* __restrict__ tile_map, int n_ftiles,
                            int d, int ntx, int nty, int ntz, int perx, int pery, int perz, int32_t* __restrict__ nbr) {
    const int nn = d == 3 ? 27 : 9;
    const long long total = (long long)n_ftiles * nn;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / nn), slot = (int)(e - (long long)k * nn);
        int q[3] = {coords[3 * k] + slot % 3 - 1, coords[3 * k + 1] + (slot / 3) % 3 - 1,
                    d == 3 ? coords[3 * k + 2] + slot / 9 - 1 : 0};
        const int nt[3] = {ntx, nty, ntz}, per[3] = {perx, pery, perz};
        bool ok = true;
        for (int ax = 0; ax < d; ax++) {
            if (q[ax] < 0 || q[ax] >= nt[ax]) {
                if (per[ax])
                    q[ax] = (q[ax] + nt[ax]) % nt[ax];
                else
                    ok = false;
            }
        }
        nbr[e] = ok ? tile_map[((long long)q[2] * nty + q[1]) * ntx + q[0]] : -1;
    }
}

// *far = 1 if a tile and one of its neighbours lie more than 2^30 values apart
__global__ void k_far_check(const int32_t* __restrict__ nbr, const long long* __restrict__ tile_off, int n_ftiles,
                            int nn, unsigned* far) {
    const long long total = (long long)n_ftiles * nn;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int nb = nbr[e];
        if (nb >= 0) {
            const long long dv = tile_off[nb] - tile_off[e / nn];
            if (dv > (1ll << 30) || dv < -(1ll << 30)) atomicOr(far, 1u);
        }
    }
}

cudaError_t launch_build_nbr(const int32_t* coords, const int32_t* tile_map, int n_ftiles, int d, int ntx, int nty,
                             int ntz, const int per[3], int32_t* nbr, cudaStream_t s) {
    const long long total = (long long)n_ftiles * (d == 3 ? 27 : 9);
    if (total == 0) return cudaSuccess;
    const long long blocks = (total + 255) / 256;
    k_build_nbr<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(coords, tile_map, n_ftiles, d, ntx, nty, ntz,
                                                                         per[0], per[1], per[2], nbr);
    return cudaGetLastError();
}

cudaError_t launch_far_check(const int32_t* nbr, const long long* tile_off, int n_ftiles, int nn, unsigned* far,
                             cudaStream_t s) {
    const long long total = (long long)n_ftiles * nn;
    if (total == 0) return cudaSuccess;
    const long long blocks = (total + 255) / 256;
    k_far_check<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(nbr, tile_off, n_ftiles, nn, far);
    return cudaGetLastError();
}

// ---- per-tile neighbour records (one-word tiles) -----------------------------------
__global__ void k_build_ntab(const int32_t* __restrict__ nbr, const uint64_t* __restrict__ tmask,
                             const long long* __restrict__ tile_off, const int32_t* __restrict__ tile_stride,
                             int n_tiles, int nn, NRec* __restrict__ ntab) {
    const long long total = (long long)n_tiles * nn;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(k / nn), nb = nbr[k];
        NRec r{0ull, 0, 0};
        if (nb >= 0) {
            r.m = tmask[nb];
            r.off = (int)(tile_off[nb] - tile_off[t]);
            r.stride = tile_stride[nb];
        }
        ntab[k] = r;
    }
}

cudaError_t launch_build_ntab(const int32_t* nbr, const uint64_t* tmask, const long long* tile_off,
                              const int32_t* tile_stride, int n_tiles, int nn, NRec* ntab, cudaStream_t s) {
    const long long total = (long long)n_tiles * nn;
    if (total == 0) return cudaSuccess;
    const long long blocks = (total + 255) / 256;
    k_build_ntab<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(nbr, tmask, tile_off, tile_stride, n_tiles,
                                                                            nn, ntab);
    return cudaGetLastError();
}

// ---- launchers ------------------------------------------------------------------------
template <class L, int A, int MODEL, class S>
cudaError_t launch_init(const NodeArgs& a, cudaStream_t s) {
    if (a.n_tiles == 0) return cudaSuccess;
    k_init<L, A, MODEL, S><<<a.n_tiles, Tile<L, A>::NT, 0, s>>>(a);
    return cudaGetLastError();
}

template <class L, int A, int MODEL, class S>
cudaError_t launch_moments(const NodeArgs& a, cudaStream_t s) {
    constexpr int TPB = tiles_per_block<L, A>();
    const int groups = (a.n_tiles + TPB - 1) / TPB;
    const int blocks = (groups + kMomentGroups - 1) / kMomentGroups;
    if (blocks == 0) return cudaSuccess;
    k_moments<L, A, TPB, MODEL, S><<<blocks, TPB * Tile<L, A>::NT, 0, s>>>(a);
    return cudaGetLastError();
}

template <class L, int A, class S>
cudaError_t launch_export(const NodeArgs& a, cudaStream_t s) {
    if (a.n_tiles == 0) return cudaSuccess;
    k_export<L, A, S><<<a.n_tiles, Tile<L, A>::NT, 0, s>>>(a);
    return cudaGetLastError();
}

template <class L, int A, class S>
cudaError_t launch_import(const NodeArgs& a, cudaStream_t s) {
    if (a.n_tiles == 0) return cudaSuccess;
    k_import<L, A, S><<<a.n_tiles, Tile<L, A>::NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fill_nan(double* p, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t blocks = (n + 255) / 256;
    k_fill_nan<<<(unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8), 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

cudaError_t launch_average(void* cur, const void* prev, size_t bytes, int storage, cudaStream_t s) {
    const size_t width = storage == LBM_STORE_F64 ? 8 : (storage == LBM_STORE_F16S ? 2 : 4);
    const size_t n = bytes / width;
    if (n == 0) return cudaSuccess;
    const size_t blocks = (n + 255) / 256;
    const unsigned grid = (unsigned)(blocks < 152 * 64 ? blocks : 152 * 64);
    if (width == 8)
        k_average_f64<<<grid, 256, 0, s>>>(static_cast<double*>(cur), static_cast<const double*>(prev), n);
    else if (width == 4)
        k_average_f32<<<grid, 256, 0, s>>>(static_cast<float*>(cur), static_cast<const float*>(prev), n);
    else
        k_average_f16<<<grid, 256, 0, s>>>(static_cast<__half*>(cur), static_cast<const __half*>(prev), n);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double* partials, int nblocks, double* result, cudaStream_t s) {
    k_reduce<<<1, 256, 0, s>>>(partials, nblocks, result);
    return cudaGetLastError();
}

int node_blocks(int lattice, int a, int n_tiles) {
    int nt = 1;
    const int d = lattice == LBM_D2Q9 ? 2 : 3;
    for (int k = 0; k < d; k++) nt *= a;
    const int tpb = nt >= 256 ? 1 : 256 / nt;
    const int groups = (n_tiles + tpb - 1) / tpb;
    return (groups + kMomentGroups - 1) / kMomentGroups;
}

// ---- selection ------------------------------------------------------------------------
#define LBM_FOR_GEOMETRY(MACRO)                      \
    if (lattice == LBM_D2Q9) {                       \
        if (a == 8) MACRO(D2Q9, 8)                   \
        if (a == 16) MACRO(D2Q9, 16)                 \
        if (a == 32) MACRO(D2Q9, 32)                 \
    } else if (lattice == LBM_D3Q19) {               \
        if (a == 4) MACRO(D3Q19, 4)                  \
        if (a == 8) MACRO(D3Q19, 8)                  \
    }

#define LBM_BY_STORAGE(F, ...)                                      \
    switch (storage) {                                             \
        case LBM_STORE_F64: return &F<__VA_ARGS__, StoreF64>;      \
        case LBM_STORE_F32: return &F<__VA_ARGS__, StoreF32>;      \
        case LBM_STORE_F16S: return &F<__VA_ARGS__, StoreF16S>;    \
        case LBM_STORE_F32S: return &F<__VA_ARGS__, StoreF32S>;    \
        default: return nullptr;                                   \
    }

NodeLaunch select_init(int lattice, int a, int model, int storage) {
#define M(L, A)                                                                       \
    {                                                                                 \
        if (model == LBM_QUASI_COMPRESSIBLE) LBM_BY_STORAGE(launch_init, L, A, 0)     \
        LBM_BY_STORAGE(launch_init, L, A, 1)                                          \
    }
    LBM_FOR_GEOMETRY(M)
#undef M
    return nullptr;
}

NodeLaunch select_moments(int lattice, int a, int model, int storage) {
#define M(L, A)                                                                        \
    {                                                                                  \
        if (model == LBM_QUASI_COMPRESSIBLE) LBM_BY_STORAGE(launch_moments, L, A, 0)   \
        LBM_BY_STORAGE(launch_moments, L, A, 1)                                        \
    }
    LBM_FOR_GEOMETRY(M)
#undef M
    return nullptr;
}

NodeLaunch select_export(int lattice, int a, int storage) {
#define M(L, A) LBM_BY_STORAGE(launch_export, L, A)
    LBM_FOR_GEOMETRY(M)
#undef M
    return nullptr;
}

NodeLaunch select_import(int lattice, int a, int storage) {
#define M(L, A) LBM_BY_STORAGE(launch_import, L, A)
    LBM_FOR_GEOMETRY(M)
#undef M
    return nullptr;
}

}  // namespace lbm

// step_ff.cu -- the FP64 tiled step with float-float arithmetic.
//
// Same update as step_fixed.cu (Eq. 7 with Eq. 2, Eq. 3/4, Eq. 5/6 and Guo
// forcing, written on deviations g_i = f_i - w_i), but every product is
// evaluated on pairs of FP32 numbers (hi + lo, ~48 significant bits) with
// fused multiply-adds, which GB300 issues at its full FP32 rate, instead of
// 64x64-bit integer multiplies.
//
//   * g_i comes from the FP64 bit patterns exactly: d_i = bits(f_i) - bits(w_i)
//     is an integer when f_i shares the binade of w_i, and two 24-bit halves of
//     d_i convert to FP32 exactly when |d_i| < 2^47;
//   * rho - 1 and j are exact 64-bit integer sums (units of 2^-60), converted
//     to float-float once per node;
//   * every quantity of link class c is formed directly in units of
//     ulp(w_c) (the scale is folded into the constants), and every f*_i is
//     rounded once to FP64: the integer count of ulps is taken within one unit
//     of the float-float result.
// Nodes outside that range (|f_i - w_i| beyond ~w_i/32, a result beyond
// ~w_i/64, |j| >= 1/16, |rho - 1| >= 1/32, NaN, negative values) are
// recomputed in native FP64.
#include <cmath>
#include <type_traits>

#include "collide_ff.cuh"

namespace lbm {

template <class L, int A, int MODEL, int MINB, int BT, int FAX>
__global__ void __launch_bounds__(BT, MINB) k_step_ff(const StepArgs a) {
    using TL = Tile<L, A>;
    using T = unsigned long long;
    if constexpr (TL::W == 1) {
        // the neighbourhood from the per-tile neighbour records
        __shared__ RecShared<TL, work_tiles()> sh;
        // the work block that runs pf_ahead blocks later: its source range is
        // requested from the L2 once this block's staging is done
        const int pfb = (int)blockIdx.x + a.pf_ahead;
        const bool pf = threadIdx.x == 0 && a.pf_ahead > 0 && pfb < a.n_work_blocks;
        WorkBlock pw{};
        if (pf) pw = a.blocks[pfb];
        WorkNode wn;
        const bool active = stage_work_rec<TL, work_tiles(), BT>(sh, a, wn);
        if (pf) prefetch_work_block<TL::NN>(a, pw);
        if (!active) return;
        const NodePos<A> p = node_pos<TL>(wn.node);
        T b[L::Q];
        int stride;
        T* out = gather_rec<L, A, work_tiles(), T>(sh, a.src, a.dst, wn.lt, wn.node, p, b, stride);
        // out of range: the same update in native FP64 (a call, so that its
        // registers do not weigh on the float-float path)
        if (!collide_ff<L, MODEL, FAX>(b, a.fx, a.ffc, out, stride))
            update_fp64_rec<L, A, MODEL, work_tiles()>(sh, a, wn, p);
    } else {
        __shared__ NeighShared<TL, work_tiles()> sh;
        WorkNode wn;
        if (!stage_work<TL, work_tiles(), BT>(sh, a, wn)) return;
        const NodePos<A> p = node_pos<TL>(wn.node);
        T b[L::Q];
        const int rank = gather<L, A, work_tiles(), T>(sh, a.src, wn.lt, wn.node, p, b);
        const int stride = sh.loc[wn.lt][TL::CENTER].y;
        T* out = own_slot<TL, work_tiles(), T>(sh, a.dst, wn.lt, rank);
        if (!collide_ff<L, MODEL, FAX>(b, a.fx, a.ffc, out, stride))
            update_fp64<L, A, MODEL, work_tiles()>(sh, a, wn, p, out, stride);
    }
}

template <class L, int A, int MODEL, int MINB, int BT, int FAX>
cudaError_t launch_step_ff(const StepArgs& a, cudaStream_t s) {
    if (a.n_work_blocks == 0) return cudaSuccess;
    k_step_ff<L, A, MODEL, MINB, BT, FAX><<<a.n_work_blocks, BT, 0, s>>>(a);
    return cudaGetLastError();
}

// ---- host: float-float constants ------------------------------------------------
static float2 split(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

static FF2C lanes(float2 a, float2 b) { return FF2C{make_float2(a.x, b.x), make_float2(a.y, b.y)}; }

template <class L>
static void ff_consts_for(const lbm_params* p, FFConsts* k) {
    const double omega = 1.0 / p->tau;
    const double kf = 1.0 - 0.5 * omega;
    const double F[3] = {p->force[0], p->force[1], L::D == 3 ? p->force[2] : 0.0};
    // class quantities in units of ulp(w_c) = 2^(E_c - 52) (exact power-of-two scales)
    double to_ulp[3];
    for (int c = 0; c < 3; c++) {
        int e = 0;
        std::frexp(L::wc_[c], &e);  // w_c = m 2^e, m in [1/2, 1): E_c = e - 1
        to_ulp[c] = std::ldexp(1.0, 52 - (e - 1));
    }
    for (int c = 0; c < 3; c++) {
        const double w = L::wc_[c];
        k->w[c] = split(w * to_ulp[c]);
        k->rho[c] = split(omega * w * to_ulp[c]);
        k->j[c] = split(3.0 * omega * w * to_ulp[c]);
    }
    k->keep = split(1.0 - omega);
    k->alpha = split(4.5 * omega);
    k->g1 = split(1.5 * omega);
    for (int a = 0; a < 3; a++) k->kf[a] = split(3.0 * kf * F[a]);
    for (int i = 0; i < L::Q; i++) {
        const double cF = L::cx_[i] * F[0] + L::cy_[i] * F[1] + L::cz_[i] * F[2];
        k->beta[i] = split(9.0 * kf * cF);
        k->so[i] = split(3.0 * kf * L::wc_[L::cls_[i]] * cF * to_ulp[L::cls_[i]]);
    }
    k->keep2 = lanes(k->keep, k->keep);
    k->alpha2 = lanes(k->alpha, k->alpha);
    k->w12 = lanes(k->w[1], k->w[2]);
    k->rho12 = lanes(k->rho[1], k->rho[2]);
    k->kf01 = lanes(k->kf[0], k->kf[1]);
    k->w11 = lanes(k->w[1], k->w[1]);
    k->w22 = lanes(k->w[2], k->w[2]);
    k->rho11 = lanes(k->rho[1], k->rho[1]);
    k->rho22 = lanes(k->rho[2], k->rho[2]);
    for (int g = 0; g < FFGroups<L>::n; g++) {
        const int a = FFGroups<L>::a[g], b = FFGroups<L>::b[g];
        k->beta2[g] = lanes(k->beta[a], k->beta[b]);
        k->j2[g] = lanes(k->j[L::cls_[a]], k->j[L::cls_[b]]);
        k->so2[g] = lanes(k->so[a], k->so[b]);
    }
}

void ff_consts(const lbm_params* p, FFConsts* k) {
    *k = FFConsts{};
    if (p->lattice == LBM_D2Q9)
        ff_consts_for<D2Q9>(p, k);
    else if (p->lattice == LBM_D3Q19)
        ff_consts_for<D3Q19>(p, k);
}

// Work blocks of 128 nodes run seven blocks per SM (the compiler holds them
// to 72 registers, 40-56 B of spill): 28 resident warps hide more of the gather
// latency than 24 at 80 registers (328 against 348 us per 256^3 step; 64
// registers and eight blocks spill 100 B, 345 us).
template <class L, int A, int BT, int FAX>
static StepLaunch pick_model(int model) {
    constexpr int MINB = BT == work_threads<L, A>() ? fp64_step_min_blocks<L, A>() : 7;
    return model == LBM_QUASI_COMPRESSIBLE ? &launch_step_ff<L, A, LBM_QUASI_COMPRESSIBLE, MINB, BT, FAX>
                                           : &launch_step_ff<L, A, LBM_INCOMPRESSIBLE, MINB, BT, FAX>;
}

// The default D3Q19 step (4^3 tiles, 128-node blocks) also comes with the
// groupings for a body force along one axis (FFGroups), which leave out the
// forcing terms of the four pairs with c_i . F = 0: the same bits in fewer
// instructions.
template <class L, int A, int BT>
static StepLaunch pick_bt(int model, int fax) {
    if constexpr (std::is_same<L, D3Q19>::value && A == 4 && BT == 128) {
        if (fax == 0) return pick_model<L, A, BT, 0>(model);
        if (fax == 1) return pick_model<L, A, BT, 1>(model);
        if (fax == 2) return pick_model<L, A, BT, 2>(model);
    }
    return pick_model<L, A, BT, -1>(model);
}

// block_nodes: 0 (the default work blocks) or 128 where they hold 256 nodes
// and a tile fits in 128 (a work block never splits a tile)
template <class L, int A>
static StepLaunch pick(int model, int block_nodes, int fax) {
    constexpr int BD = work_threads<L, A>();
    if constexpr (BD == 256 && Tile<L, A>::NT <= 128) {
        if (block_nodes == 128) return pick_bt<L, A, 128>(model, fax);
    }

    if (block_nodes != 0 && block_nodes != BD) return nullptr;
    return pick_bt<L, A, BD>(model, fax);
}

int ff_force_axis(int lattice, const double force[3]) {
    if (lattice != LBM_D3Q19) return -1;
    int nz = 0, ax = 0;
    for (int k = 0; k < 3; k++)
        if (force[k] != 0.0) {
            nz++;
            ax = k;
        }
    return nz <= 1 ? ax : -1;
}

StepLaunch select_step_ff(int lattice, int a, int model, int block_nodes, int fax) {
    if (lattice == LBM_D2Q9) {
        if (a == 8) return pick<D2Q9, 8>(model, block_nodes, -1);
        if (a == 16) return pick<D2Q9, 16>(model, block_nodes, -1);
        if (a == 32) return pick<D2Q9, 32>(model, block_nodes, -1);
    } else if (lattice == LBM_D3Q19) {
        if (a == 4) return pick<D3Q19, 4>(model, block_nodes, fax);
        if (a == 8) return pick<D3Q19, 8>(model, block_nodes, fax);
    }
    return nullptr;
}

}  // namespace lbm

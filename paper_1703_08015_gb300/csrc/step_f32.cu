// step_f32.cu -- reduced-precision storage forms of the tiled step (not in
// the paper): PDFs stored as FP32 values, as FP32 deviations f_i - w_i, or as
// FP16 deviations h_i = RN_fp16((f_i - w_i) * S) with a power-of-two scale S;
// the collision runs in FP32 in every case.  Storing deviations keeps the
// rounding relative to f_i - w_i, so slow hydrodynamic drifts are not lost
// in the rounding of f_i ~ w_i.
//
// The collision works on deviations g_i = f_i - w_i so that FP32 rounding acts
// on the small deviation, not on f_i itself:
//   rho - 1 = sum g_i,   j = sum c_i g_i + F/2,   u = j / rho  (Eq. 5; Eq. 6: u = j)
//   f^eq_i - w_i = w_i [ (rho - 1) + rho (3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u) ]   (Eq. 3)
//                = w_i [ (rho - 1) + 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u ]          (Eq. 4)
//   g*_i = g_i - (g_i - (f^eq_i - w_i)) / tau + S_i  (Eq. 7 with Eq. 2, Guo forcing S_i)
#include "collide_f32.cuh"

namespace lbm {

template <class L, int A, int MODEL, class S, int BT, bool PERSIST>
__global__ void __launch_bounds__(BT, (!PERSIST && BT <= 256) ? 1536 / BT : 1) k_step_f32(const StepArgs a) {
    using TL = Tile<L, A>;
    using T = typename S::T;
    using IO = F32Io<L, S>;
    __shared__ NeighShared<TL, work_tiles()> sh;
    // one work block per thread block, or (persistent) a grid-stride loop over them
    for (int wbi = blockIdx.x; wbi < a.n_work_blocks; wbi += PERSIST ? (int)gridDim.x : a.n_work_blocks) {
        // the work block that runs pf_ahead blocks later: its source range is
        // requested from the L2 once this block's staging is done
        const bool pf = !PERSIST && threadIdx.x == 0 && a.pf_ahead > 0 && wbi + a.pf_ahead < a.n_work_blocks;
        WorkBlock pw{};
        if (pf) pw = a.blocks[wbi + a.pf_ahead];
        WorkNode wn;
        const bool active = stage_work_at<TL, work_tiles(), BT>(sh, a, wbi, wn);
        if (pf) prefetch_work_block<TL::NN>(a, pw);
        if (active) {
            const NodePos<A> p = node_pos<TL>(wn.node);
            T raw[L::Q];
            const int rank = gather<L, A, work_tiles(), T>(sh, a.src, wn.lt, wn.node, p, raw);
            const int stride = sh.loc[wn.lt][TL::CENTER].y;
            float g[L::Q];
            static_for<0, L::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                g[i] = IO::template dev<i>(raw[i], a);
            });
            collide_f32<L, MODEL>(g, a.f32c, a.force_f);
            T* out = own_slot<TL, work_tiles(), T>(sh, a.dst, wn.lt, rank);
            static_for<0, L::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                out[i * stride] = IO::template raw<i>(g[i], a);
            });
        }
        if (PERSIST) __syncthreads();  // the staging arrays are refilled for the next work block
    }
}

template <class L, int A, int MODEL, class S, int BT, bool PERSIST>
cudaError_t launch_step_f32(const StepArgs& a, cudaStream_t s) {
    if (a.n_work_blocks == 0) return cudaSuccess;
    int grid = a.n_work_blocks;
    if (PERSIST) {
        static int resident = 0;  // blocks of this kernel the GPU holds at once
        if (!resident) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_f32<L, A, MODEL, S, BT, PERSIST>, BT, 0);
            resident = sms * (per_sm > 0 ? per_sm : 1);
        }
        grid = a.n_work_blocks < resident ? a.n_work_blocks : resident;
    }
    k_step_f32<L, A, MODEL, S, BT, PERSIST><<<grid, BT, 0, s>>>(a);
    return cudaGetLastError();
}

template <class L, int A, int MODEL, class S>
static StepLaunch pick_shape(int block_nodes, int persistent) {
    constexpr int BD = work_threads<L, A>();
    if constexpr (BD == 256 && Tile<L, A>::NT <= 128) {  // a work block never splits a tile
        if (block_nodes == 128)
            return persistent ? &launch_step_f32<L, A, MODEL, S, 128, true> : &launch_step_f32<L, A, MODEL, S, 128, false>;
    }
    if (block_nodes != 0 && block_nodes != BD) return nullptr;
    return persistent ? &launch_step_f32<L, A, MODEL, S, BD, true> : &launch_step_f32<L, A, MODEL, S, BD, false>;
}

template <class L, int A, class S>
static StepLaunch pick(int model, int block_nodes, int persistent) {
    return model == LBM_QUASI_COMPRESSIBLE ? pick_shape<L, A, LBM_QUASI_COMPRESSIBLE, S>(block_nodes, persistent)
                                           : pick_shape<L, A, LBM_INCOMPRESSIBLE, S>(block_nodes, persistent);
}

template <class L, int A>
static StepLaunch pick_storage(int model, int storage, int block_nodes, int persistent) {
    if (storage == LBM_STORE_F32) return pick<L, A, StoreF32>(model, block_nodes, persistent);
    if (storage == LBM_STORE_F16S) return pick<L, A, StoreF16S>(model, block_nodes, persistent);
    if (storage == LBM_STORE_F32S) return pick<L, A, StoreF32S>(model, block_nodes, persistent);
    return nullptr;
}

template <class L>
static void f32_consts_for(double omega, const double* force, F32Consts* k) {
    const double kf = 1.0 - 0.5 * omega;
    const double F[3] = {force[0], force[1], L::D == 3 ? force[2] : 0.0};
    k->keep = (float)(1.0 - omega);
    for (int c = 0; c < 3; c++) {
        k->ow[c] = (float)(omega * L::wc_[c]);
        k->kw3[c] = (float)(3.0 * kf * L::wc_[c]);
    }
    for (int i = 0; i < L::Q; i++) {
        const double cF = L::cx_[i] * F[0] + L::cy_[i] * F[1] + L::cz_[i] * F[2];
        const double w = L::wc_[L::cls_[i]];
        k->be[i] = (float)(9.0 * kf * w * cF);
        k->so[i] = (float)(3.0 * kf * w * cF);
    }
}

void f32_consts(const lbm_params* p, double omega, const double* force, F32Consts* k) {
    *k = F32Consts{};
    if (p->lattice == LBM_D2Q9)
        f32_consts_for<D2Q9>(omega, force, k);
    else if (p->lattice == LBM_D3Q19)
        f32_consts_for<D3Q19>(omega, force, k);
}

StepLaunch select_step_f32(int lattice, int a, int model, int storage, int block_nodes, int persistent) {
    if (lattice == LBM_D2Q9) {
        if (a == 8) return pick_storage<D2Q9, 8>(model, storage, block_nodes, persistent);
        if (a == 16) return pick_storage<D2Q9, 16>(model, storage, block_nodes, persistent);
        if (a == 32) return pick_storage<D2Q9, 32>(model, storage, block_nodes, persistent);
    } else if (lattice == LBM_D3Q19) {
        if (a == 4) return pick_storage<D3Q19, 4>(model, storage, block_nodes, persistent);
        if (a == 8) return pick_storage<D3Q19, 8>(model, storage, block_nodes, persistent);
    }
    return nullptr;
}

}  // namespace lbm

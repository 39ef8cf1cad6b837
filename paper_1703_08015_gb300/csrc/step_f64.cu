// step_f64.cu -- the tiled step (Fig. 5) with native FP64 arithmetic: raw
// words are gathered, widened to FP64, collided, and stored into the node's
// own slots of the other copy.  One thread per fluid node (work list).
#include "collide_f64.cuh"
#include "tile.cuh"

namespace lbm {

template <class L, int A, int MODEL, class S>
__global__ void __launch_bounds__(work_threads<L, A>()) k_step_f64(const StepArgs a) {
    using TL = Tile<L, A>;
    using T = typename S::T;
    __shared__ NeighShared<TL, work_tiles()> sh;
    WorkNode wn;
    if (!stage_work<TL, work_tiles(), work_threads<L, A>()>(sh, a, wn)) return;
    const NodePos<A> p = node_pos<TL>(wn.node);
    T raw[L::Q];
    const int rank = gather<L, A, work_tiles(), T>(sh, a.src, wn.lt, wn.node, p, raw);
    const int stride = sh.loc[wn.lt][TL::CENTER].y;
    double f[L::Q];
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        f[i] = S::template to_f64<L, i>(raw[i], a.f16_inv_scale);
    });
    collide_f64<L, MODEL>(f, a.omega, a.force);
    T* out = own_slot<TL, work_tiles(), T>(sh, a.dst, wn.lt, rank);
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        out[i * stride] = S::template from_f64<L, i>(f[i], a.f16_scale);
    });
}

template <class L, int A, int MODEL, class S>
cudaError_t launch_step_f64(const StepArgs& a, cudaStream_t s) {
    if (a.n_work_blocks == 0) return cudaSuccess;
    k_step_f64<L, A, MODEL, S><<<a.n_work_blocks, work_threads<L, A>(), 0, s>>>(a);
    return cudaGetLastError();
}

template <class L, int A, class S>
static StepLaunch pick_model(int model) {
    return model == LBM_QUASI_COMPRESSIBLE ? &launch_step_f64<L, A, LBM_QUASI_COMPRESSIBLE, S>
                                           : &launch_step_f64<L, A, LBM_INCOMPRESSIBLE, S>;
}

StepLaunch select_step_f64(int lattice, int a, int model, int storage) {
#define LBM_PICK_STORE(L, A)                                                   \
    switch (storage) {                                                         \
        case LBM_STORE_F64: return pick_model<L, A, StoreF64>(model);          \
        default: return nullptr;                                               \
    }
    if (lattice == LBM_D2Q9) {
        if (a == 8) LBM_PICK_STORE(D2Q9, 8)
        if (a == 16) LBM_PICK_STORE(D2Q9, 16)
        if (a == 32) LBM_PICK_STORE(D2Q9, 32)
    } else if (lattice == LBM_D3Q19) {
        if (a == 4) LBM_PICK_STORE(D3Q19, 4)
        if (a == 8) LBM_PICK_STORE(D3Q19, 8)
    }
#undef LBM_PICK_STORE
    return nullptr;
}

}  // namespace lbm

// step_f64.cu -- the tiled step (Fig. 5) with native FP64 arithmetic, for
// every storage format: raw words are gathered, widened to FP64, collided,
// narrowed and stored back into the node's own slots of the other copy.
#include "collide_f64.cuh"
#include "tile.cuh"

namespace lbm {

template <class L, int A, int TPB, int MODEL, class S>
__global__ void __launch_bounds__(TPB* Tile<L, A>::NT) k_step_f64(const StepArgs a) {
    using TL = Tile<L, A>;
    using T = typename S::T;
    constexpr size_t TILE_BYTES = sizeof(T) * L::Q * TL::NT;
    __shared__ NeighShared<TL, TPB> sh;
    const int lt = threadIdx.x / TL::NT;
    const int node = threadIdx.x - lt * TL::NT;
    const int tile = blockIdx.x * TPB + lt;
    stage_neighbourhood<TL, TPB>(sh, a.nbr, a.tmask, static_cast<const unsigned char*>(a.src), TILE_BYTES,
                                 a.n_tiles, tile, lt, node);
    __syncthreads();  // the only barrier (Fig. 5, step 4)
    if (tile >= a.n_tiles || !mask_bit(sh, lt, TL::CENTER, node)) return;

    const NodePos<A> p = node_pos<TL>(node);
    T raw[L::Q];
    gather<L, A, TPB, T>(sh, lt, node, p, raw);
    double f[L::Q];
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        f[i] = S::template to_f64<L, i>(raw[i], a.f16_inv_scale);
    });
    collide_f64<L, MODEL>(f, a.omega, a.force);
    T* out = static_cast<T*>(a.dst) + (size_t)tile * L::Q * TL::NT + node;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        out[i * TL::NT] = S::template from_f64<L, i>(f[i], a.f16_scale);
    });
}

template <class L, int A, int MODEL, class S>
cudaError_t launch_step_f64(const StepArgs& a, cudaStream_t s) {
    constexpr int TPB = tiles_per_block<L, A>();
    const int blocks = (a.n_tiles + TPB - 1) / TPB;
    if (blocks == 0) return cudaSuccess;
    k_step_f64<L, A, TPB, MODEL, S><<<blocks, TPB * Tile<L, A>::NT, 0, s>>>(a);
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

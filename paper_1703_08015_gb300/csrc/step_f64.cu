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

// Native-FP64 update of the nodes the float-float or fixed-point step listed as
// out of its range (a state far from equilibrium).  Reads the same source copy
// and overwrites the listed nodes' values in the destination; the last block
// to finish clears the list for the next step.
template <class L, int A, int MODEL>
__global__ void __launch_bounds__(Tile<L, A>::NT) k_fp64_fallback(const StepArgs a) {
    using TL = Tile<L, A>;
    using T = unsigned long long;
    __shared__ NeighShared<TL, 1> sh;
    const unsigned n = min(*a.fb_count, a.fb_cap);
    for (unsigned e = blockIdx.x; e < n; e += gridDim.x) {
        const uint32_t ent = a.fb_list[e];
        const int tile = (int)(ent >> (TL::D * TL::LA)), node = (int)(ent & (TL::NT - 1));
        stage_neighbourhood<TL, 1>(sh, a.nbr, a.tmask, a.tile_off, a.tile_stride, tile, a.n_tiles, tile, 0,
                                   threadIdx.x);
        __syncthreads();
        if (threadIdx.x == 0) {
            const NodePos<A> p = node_pos<TL>(node);
            T b[L::Q];
            const int rank = gather<L, A, 1, T>(sh, a.src, 0, node, p, b);
            double f[L::Q];
            static_for<0, L::Q>([&](auto I) { f[decltype(I)::value] = __longlong_as_double((long long)b[decltype(I)::value]); });
            collide_f64<L, MODEL>(f, a.omega, a.force);
            T* out = own_slot<TL, 1, T>(sh, a.dst, 0, rank);
            const int stride = sh.loc[0][TL::CENTER].y;
            static_for<0, L::Q>([&](auto I) { out[decltype(I)::value * stride] = (T)__double_as_longlong(f[decltype(I)::value]); });
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.fb_done, 1u) == gridDim.x - 1) {
            *a.fb_count = 0;
            *a.fb_done = 0;
            __threadfence();
        }
    }
}

template <class L, int A, int MODEL>
cudaError_t launch_fp64_fallback(const StepArgs& a, cudaStream_t s) {
    k_fp64_fallback<L, A, MODEL><<<152, Tile<L, A>::NT, 0, s>>>(a);
    return cudaGetLastError();
}

template <class L, int A>
static StepLaunch pick_fallback(int model) {
    return model == LBM_QUASI_COMPRESSIBLE ? &launch_fp64_fallback<L, A, LBM_QUASI_COMPRESSIBLE>
                                           : &launch_fp64_fallback<L, A, LBM_INCOMPRESSIBLE>;
}

StepLaunch select_fp64_fallback(int lattice, int a, int model) {
    if (lattice == LBM_D2Q9) {
        if (a == 8) return pick_fallback<D2Q9, 8>(model);
        if (a == 16) return pick_fallback<D2Q9, 16>(model);
        if (a == 32) return pick_fallback<D2Q9, 32>(model);
    } else if (lattice == LBM_D3Q19) {
        if (a == 4) return pick_fallback<D3Q19, 4>(model);
        if (a == 8) return pick_fallback<D3Q19, 8>(model);
    }
    return nullptr;
}

}  // namespace lbm

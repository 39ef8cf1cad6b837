// tgb.cu -- the single-copy "tiles with ghost buffers" (TGB) form of the step
// (Sec. 3.1, Fig. 2-4): one PDF copy updated in place, plus two sets of ghost
// buffers through which tiles exchange the values that cross their edges.
//
// The copy holds the post-collision state f*(t) in the compact tile layout of
// the two-copy (T2C) form, so initialisation, moments, export and import are
// the T2C kernels.  Ghost set G holds, for every non-empty tile and every link
// i, the values f*_i of the nodes on the tile's downstream boundary for i (the
// nodes whose r + c_i lies outside the tile), a^d - a^(d-k) (a-1)^k entries for
// a link with k nonzero components.  A step reads f*(t) of its own tile from
// the copy and the values arriving from neighbour tiles from ghost set t,
// collides, and after one barrier writes f*(t+1) in place and the tile's
// boundary values into ghost set t+1; tiles never read each other's copy, so
// blocks need no ordering.  A source node that is solid, in a removed tile or
// beyond a wall gives halfway bounce-back exactly as in T2C (the receiver
// tests the source's fluid bit, so ghost entries of solid nodes are never
// read).  The update of every node is the T2C update bit for bit.
#include <cmath>

#include "collide_f32.cuh"
#include "collide_ff.cuh"

namespace lbm {

template <class L, int A, int I>
struct Ghost {
    using K = Link<L, I>;
    static constexpr int D = L::D;
    static constexpr int NZ = (K::cx != 0) + (K::cy != 0) + (K::cz != 0);
    static constexpr int pw(int b, int e) { return e == 0 ? 1 : b * pw(b, e - 1); }
    // entries of link I: the downstream boundary of the tile for I
    static constexpr int count = I == 0 ? 0 : pw(A, D) - pw(A, D - NZ) * pw(A - 1, NZ);
    // first entry of link I within a tile's ghost block
    static constexpr int offset() {
        int o = 0;
        for (int j = 1; j < I; j++) {
            const int nz = (L::cx_[j] != 0) + (L::cy_[j] != 0) + (L::cz_[j] != 0);
            o += pw(A, D) - pw(A, D - nz) * pw(A - 1, nz);
        }
        return o;
    }
    // is r + c_I outside the tile?
    __host__ __device__ static __forceinline__ bool downstream(int lx, int ly, int lz) {
        bool b = false;
        if constexpr (K::cx > 0) b |= lx == A - 1;
        if constexpr (K::cx < 0) b |= lx == 0;
        if constexpr (K::cy > 0) b |= ly == A - 1;
        if constexpr (K::cy < 0) b |= ly == 0;
        if constexpr (K::cz > 0) b |= lz == A - 1;
        if constexpr (K::cz < 0) b |= lz == 0;
        return b;
    }
    // index among the link's entries of a node on its downstream boundary:
    // first the face of the first nonzero axis (other coordinates, lowest axis
    // fastest), then the face of the second nonzero axis without the shared edge
    __host__ __device__ static __forceinline__ int entry(int lx, int ly, int lz) {
        const int c[3] = {K::cx, K::cy, K::cz};
        const int x[3] = {lx, ly, lz};
        constexpr int ax0 = K::cx != 0 ? 0 : (K::cy != 0 ? 1 : 2);
        constexpr int ax1 = NZ == 2 ? (ax0 == 0 ? (K::cy != 0 ? 1 : 2) : 2) : -1;
        const int b0 = c[ax0] > 0 ? A - 1 : 0;
        auto face = [&](int ax) {  // index over the other axes of a face normal to ax
            int idx = 0, mul = 1;
            for (int k = 0; k < D; k++)
                if (k != ax) {
                    idx += x[k] * mul;
                    mul *= A;
                }
            return idx;
        };
        if constexpr (NZ == 1) {
            return face(ax0);
        } else {
            if (x[ax0] == b0) return face(ax0);
            const int a0 = c[ax0] > 0 ? x[ax0] : x[ax0] - 1;  // 0 .. A-2 off the shared edge
            int idx = a0, mul = A - 1;
            for (int k = 0; k < D; k++)
                if (k != ax0 && k != ax1) {
                    idx += x[k] * mul;
                    mul *= A;
                }
            return pw(A, D - 1) + idx;
        }
    }
};

template <class L, int A>
constexpr int ghost_per_tile() {
    int e = 0;
    for (int j = 1; j < L::Q; j++) {
        const int nz = (L::cx_[j] != 0) + (L::cy_[j] != 0) + (L::cz_[j] != 0);
        e += Ghost<L, A, 1>::pw(A, L::D) - Ghost<L, A, 1>::pw(A, L::D - nz) * Ghost<L, A, 1>::pw(A - 1, nz);
    }
    return e;
}

// Gather the q post-collision words that arrive at `node`: from the tile's own
// copy when the source is inside the tile, from the neighbour's ghost entries
// when it is outside, bounce-back when the source is not a fluid node.
template <class L, int A, int KMAX, class T>
__device__ __forceinline__ int gather_tgb(const NeighShared<Tile<L, A>, KMAX>& sh, const int (&nbt)[KMAX][Tile<L, A>::NN],
                                          const T* copy, const T* __restrict__ ghost_in, int lt, int node,
                                          const NodePos<A>& p, T (&f)[L::Q]) {
    using TL = Tile<L, A>;
    constexpr int E = ghost_per_tile<L, A>();
    const T* own = copy + sh.origin + sh.loc[lt][TL::CENTER].x;
    const int own_stride = sh.loc[lt][TL::CENTER].y;
    const int own_rank = fluid_rank<TL::W>(sh.m[lt][TL::CENTER], node);
    f[0] = own[own_rank];
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using G = Ghost<L, A, i>;
        const PullSource<L, A, i> s(p);
        bool fl;
        const int r = fluid_bit_rank<TL::W>(sh.m[lt][s.slot], s.sn, fl);
        const T* src = own + Link<L, i>::opp * own_stride + own_rank;  // bounce-back
        if (fl) {
            if (s.slot == TL::CENTER) {
                src = own + i * own_stride + r;
            } else {
                const int sx = s.sn & (A - 1), sy = (s.sn >> TL::LA) & (A - 1), sz = s.sn >> (2 * TL::LA);
                src = ghost_in + (size_t)nbt[lt][s.slot] * E + G::offset() + G::entry(sx, sy, sz);
            }
        }
        f[i] = *src;
    });
    return own_rank;
}

// The q FP64 words of a node's update in native FP64, for the nodes outside
// the range of the float-float arithmetic: a call rather than inline code, so
// that its registers do not weigh on the step.
template <int Q>
struct Words {
    unsigned long long v[Q];
};

template <class L, int A, int MODEL, int KMAX>
__device__ __noinline__ Words<L::Q> tgb_update_fp64(const NeighShared<Tile<L, A>, KMAX>& sh,
                                                    const int (&nbt)[KMAX][Tile<L, A>::NN], const StepArgs& a,
                                                    int lt, int node, const NodePos<A>& p) {
    unsigned long long raw[L::Q];
    gather_tgb<L, A, KMAX, unsigned long long>(sh, nbt, static_cast<const unsigned long long*>(a.dst),
                                               static_cast<const unsigned long long*>(a.ghost_in), lt, node, p, raw);
    double f[L::Q];
    static_for<0, L::Q>([&](auto I) { f[decltype(I)::value] = __longlong_as_double((long long)raw[decltype(I)::value]); });
    collide_f64<L, MODEL>(f, a.omega, a.force);
    Words<L::Q> w;
    static_for<0, L::Q>([&](auto I) { w.v[decltype(I)::value] = (unsigned long long)__double_as_longlong(f[decltype(I)::value]); });
    return w;
}

// Resident blocks per SM requested (register cap) for each arithmetic.
template <class L, int A, int ARITH>
constexpr int tgb_min_blocks() {
    return work_threads<L, A>() > 256 ? 1 : (ARITH == 0 ? 1280 / work_threads<L, A>() : (ARITH == 1 ? 3 : 2));
}

// ARITH: 0 = FP32 collision on deviations (reduced storage), 1 = float-float
// FP64 (native FP64 for nodes out of its range), 2 = native FP64.
template <class L, int A, int MODEL, class S, int ARITH>
__global__ void __launch_bounds__(work_threads<L, A>(), tgb_min_blocks<L, A, ARITH>()) k_step_tgb(const StepArgs a) {
    using TL = Tile<L, A>;
    using T = typename S::T;
    constexpr int E = ghost_per_tile<L, A>();
    __shared__ NeighShared<TL, work_tiles()> sh;
    __shared__ int nbt[work_tiles()][TL::NN];
    const WorkBlock wb = a.blocks[blockIdx.x];
    T* copy = static_cast<T*>(a.dst);  // the single copy (src == dst)
    const bool active = (int)threadIdx.x < wb.count;
    const uint32_t e = active ? __ldg(a.nodes + wb.node_begin + threadIdx.x) : 0u;  // in flight during the staging
    stage_tables<TL, work_tiles(), work_threads<L, A>()>(sh, a, wb, nbt);
    __syncthreads();
    T vals[L::Q];
    int tile = 0, lt = 0, node = 0, rank = 0;
    NodePos<A> p{0, 0, 0};
    if (active) {
        tile = (int)(e >> (TL::D * TL::LA));
        node = (int)(e & (TL::NT - 1));
        lt = tile - wb.tile_begin;
        p = node_pos<TL>(node);
        T raw[L::Q];
        rank = gather_tgb<L, A, work_tiles(), T>(sh, nbt, copy, static_cast<const T*>(a.ghost_in), lt, node, p, raw);
        if constexpr (ARITH == 0) {
            using IO = F32Io<L, S>;
            float g[L::Q];
            static_for<0, L::Q>([&](auto I) { g[decltype(I)::value] = IO::template dev<decltype(I)::value>(raw[decltype(I)::value], a); });
            collide_f32<L, MODEL>(g, a.f32c, a.force_f);
            static_for<0, L::Q>([&](auto I) { vals[decltype(I)::value] = IO::template raw<decltype(I)::value>(g[decltype(I)::value], a); });
        } else {
            if constexpr (ARITH == 1) {
                if (!collide_ff<L, MODEL>(raw, a.fx, a.ffc, vals, 1)) {
                    const Words<L::Q> w = tgb_update_fp64<L, A, MODEL, work_tiles()>(sh, nbt, a, lt, node, p);
                    static_for<0, L::Q>([&](auto I) { vals[decltype(I)::value] = w.v[decltype(I)::value]; });
                }
            } else {
                double f[L::Q];
                static_for<0, L::Q>([&](auto I) { f[decltype(I)::value] = __longlong_as_double((long long)raw[decltype(I)::value]); });
                collide_f64<L, MODEL>(f, a.omega, a.force);
                static_for<0, L::Q>([&](auto I) { vals[decltype(I)::value] = (T)__double_as_longlong(f[decltype(I)::value]); });
            }
        }
    }
    __syncthreads();  // every read of this block's tiles is done: update in place
    if (active) {
        T* own = copy + sh.origin + sh.loc[lt][TL::CENTER].x;
        const int stride = sh.loc[lt][TL::CENTER].y;
        T* gout = static_cast<T*>(a.ghost_out) + (size_t)tile * E;
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            own[i * stride + rank] = vals[i];
            if constexpr (i > 0) {
                using G = Ghost<L, A, i>;
                if (G::downstream(p.lx, p.ly, p.lz)) gout[G::offset() + G::entry(p.lx, p.ly, p.lz)] = vals[i];
            }
        });
    }
}

// Fill a ghost set from the copy (after initialisation or import).
template <class L, int A, class S>
__global__ void k_tgb_publish(const StepArgs a) {
    using TL = Tile<L, A>;
    using T = typename S::T;
    constexpr int E = ghost_per_tile<L, A>();
    const WorkBlock wb = a.blocks[blockIdx.x];
    if ((int)threadIdx.x >= wb.count) return;
    const uint32_t e = __ldg(a.nodes + wb.node_begin + threadIdx.x);
    const int tile = (int)(e >> (TL::D * TL::LA));
    const int node = (int)(e & (TL::NT - 1));
    const NodePos<A> p = node_pos<TL>(node);
    const T* own = static_cast<const T*>(a.src) + a.tile_off[tile] + fluid_rank<TL::W>(a.tmask + (size_t)tile * TL::W, node);
    const int stride = a.tile_stride[tile];
    T* gout = static_cast<T*>(a.ghost_out) + (size_t)tile * E;
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        using G = Ghost<L, A, i>;
        if (G::downstream(p.lx, p.ly, p.lz)) gout[G::offset() + G::entry(p.lx, p.ly, p.lz)] = own[i * stride];
    });
}

template <class L, int A, int MODEL, class S, int ARITH>
cudaError_t launch_step_tgb(const StepArgs& a, cudaStream_t s) {
    if (a.n_work_blocks == 0) return cudaSuccess;
    k_step_tgb<L, A, MODEL, S, ARITH><<<a.n_work_blocks, work_threads<L, A>(), 0, s>>>(a);
    return cudaGetLastError();
}

template <class L, int A, class S>
cudaError_t launch_tgb_publish(const StepArgs& a, cudaStream_t s) {
    if (a.n_work_blocks == 0) return cudaSuccess;
    k_tgb_publish<L, A, S><<<a.n_work_blocks, work_threads<L, A>(), 0, s>>>(a);
    return cudaGetLastError();
}

template <class L, int A, int MODEL>
static StepLaunch pick_tgb(int storage, int arith) {
    if (storage == LBM_STORE_F64) {
        if (arith == LBM_ARITH_F64) return &launch_step_tgb<L, A, MODEL, StoreF64, 2>;
        if (arith == LBM_ARITH_FF || arith == LBM_ARITH_AUTO || arith == LBM_ARITH_FF_TABLE)
            return &launch_step_tgb<L, A, MODEL, StoreF64, 1>;
        return nullptr;
    }
    if (storage == LBM_STORE_F32) return &launch_step_tgb<L, A, MODEL, StoreF32, 0>;
    if (storage == LBM_STORE_F32S) return &launch_step_tgb<L, A, MODEL, StoreF32S, 0>;
    if (storage == LBM_STORE_F16S) return &launch_step_tgb<L, A, MODEL, StoreF16S, 0>;
    return nullptr;
}

template <class L, int A>
static StepLaunch pick_tgb_model(int model, int storage, int arith) {
    return model == LBM_QUASI_COMPRESSIBLE ? pick_tgb<L, A, LBM_QUASI_COMPRESSIBLE>(storage, arith)
                                           : pick_tgb<L, A, LBM_INCOMPRESSIBLE>(storage, arith);
}

StepLaunch select_step_tgb(const lbm_params* p) {
    if (p->persistent || (p->block_nodes && p->block_nodes != work_threads_for(p->lattice, p->tile_a)))
        return nullptr;
    if (p->lattice == LBM_D2Q9) {
        if (p->tile_a == 8) return pick_tgb_model<D2Q9, 8>(p->model, p->storage, p->arith);
        if (p->tile_a == 16) return pick_tgb_model<D2Q9, 16>(p->model, p->storage, p->arith);
        if (p->tile_a == 32) return pick_tgb_model<D2Q9, 32>(p->model, p->storage, p->arith);
    } else if (p->lattice == LBM_D3Q19) {
        if (p->tile_a == 4) return pick_tgb_model<D3Q19, 4>(p->model, p->storage, p->arith);
        if (p->tile_a == 8) return pick_tgb_model<D3Q19, 8>(p->model, p->storage, p->arith);
    }
    return nullptr;
}

template <class L, int A>
static StepLaunch pick_publish(int storage) {
    if (storage == LBM_STORE_F64) return &launch_tgb_publish<L, A, StoreF64>;
    if (storage == LBM_STORE_F32) return &launch_tgb_publish<L, A, StoreF32>;
    if (storage == LBM_STORE_F32S) return &launch_tgb_publish<L, A, StoreF32S>;
    if (storage == LBM_STORE_F16S) return &launch_tgb_publish<L, A, StoreF16S>;
    return nullptr;
}

StepLaunch select_tgb_publish(int lattice, int a, int storage) {
    if (lattice == LBM_D2Q9) {
        if (a == 8) return pick_publish<D2Q9, 8>(storage);
        if (a == 16) return pick_publish<D2Q9, 16>(storage);
        if (a == 32) return pick_publish<D2Q9, 32>(storage);
    } else if (lattice == LBM_D3Q19) {
        if (a == 4) return pick_publish<D3Q19, 4>(storage);
        if (a == 8) return pick_publish<D3Q19, 8>(storage);
    }
    return nullptr;
}

long long tgb_ghost_per_tile(int lattice, int a) {
    if (lattice == LBM_D2Q9) {
        if (a == 8) return ghost_per_tile<D2Q9, 8>();
        if (a == 16) return ghost_per_tile<D2Q9, 16>();
        if (a == 32) return ghost_per_tile<D2Q9, 32>();
    } else if (lattice == LBM_D3Q19) {
        if (a == 4) return ghost_per_tile<D3Q19, 4>();
        if (a == 8) return ghost_per_tile<D3Q19, 8>();
    }
    return 0;
}

}  // namespace lbm

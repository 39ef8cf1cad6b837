// step_ff_table.cu -- the FP64 float-float step through a per-node gather
// table (LBM_ARITH_FF_TABLE): the connectivity-matrix scheme the paper sets
// against its tiles (Sec. 2.3.1, Eqs. 13-14), kept on the compact tiles as an
// opt-in for comparison.  The collision is collide_ff, the rule of each
// node's sources that of gather() (tile.cuh).
#include "collide_ff.cuh"

namespace lbm {

// ---- the gather table: the FP64 step without staging ---------------------------
// The sources of every node's gather depend only on the geometry, so they are
// computed once: for the node at work-list position n, row 0 of the table
// holds its own slot, row i (1 .. q-1) the slot f*_i(r - c_i) is pulled from
// (its own f*_opp(i) slot when r - c_i is solid, removed or beyond a wall:
// halfway bounce-back), row q its tile's stride (values per link); slots are
// int32 value indices into a PDF copy (both copies share the layout).  The
// step then reads q + 1 coalesced table words per node instead of staging the
// neighbourhood: no shared memory, no barrier and no index arithmetic, at
// 4 (q + 1) bytes more per node update.  The rule is the one of gather().
template <class L, int A>
__global__ void __launch_bounds__(work_threads<L, A>()) k_gather_table(const StepArgs a) {
    using TL = Tile<L, A>;
    __shared__ NeighShared<TL, work_tiles()> sh;
    WorkNode wn;
    if (!stage_work<TL, work_tiles(), work_threads<L, A>()>(sh, a, wn)) return;
    const long long pos = (long long)a.blocks[blockIdx.x].node_begin + threadIdx.x;
    const long long P = a.gtab_pitch;
    const NodePos<A> p = node_pos<TL>(wn.node);
    const int2 own = sh.loc[wn.lt][TL::CENTER];
    const int own_rank = fluid_rank<TL::W>(sh.m[wn.lt][TL::CENTER], wn.node);
    const long long own_r = sh.origin + own.x + own_rank;
    int32_t* t = a.gtab_out + pos;
    t[0] = (int32_t)own_r;
    const PullBase<L, A> pb(p);
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const PullSource<L, A, i> s(pb);
        bool fl;
        const int r = fluid_bit_rank<TL::W>(sh.m[wn.lt][s.slot], s.sn, fl);
        const int2 nb = sh.loc[wn.lt][s.slot];
        const long long idx = fl ? sh.origin + nb.x + i * nb.y + r : own_r + Link<L, i>::opp * own.y;
        t[i * P] = (int32_t)idx;
    });
    t[L::Q * P] = own.y;
}

// Native-FP64 update of one node through the table (the range fallback).
template <class L, int MODEL>
__device__ __noinline__ void update_fp64_table(const StepArgs& a, const int32_t* t, unsigned long long* out,
                                               int stride) {
    using T = unsigned long long;
    const T* src = static_cast<const T*>(a.src);
    double f[L::Q];
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        f[i] = __longlong_as_double((long long)src[__ldg(t + i * a.gtab_pitch)]);
    });
    collide_f64<L, MODEL>(f, a.omega, a.force);
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        out[i * stride] = (T)__double_as_longlong(f[i]);
    });
}

// Blocks of 128 threads, seven per SM (72 registers): 290 against 310 us per
// 256^3 step for three blocks of 256 at 80 registers.
constexpr int kTableThreads = 128;

template <class L, int MODEL>
__global__ void __launch_bounds__(kTableThreads, 7) k_step_ff_table(const StepArgs a) {
    using T = unsigned long long;
    const long long pos = (long long)blockIdx.x * kTableThreads + threadIdx.x;
    if (pos >= a.n_nodes) return;
    const long long P = a.gtab_pitch;
    const int32_t* t = a.gtab + pos;
    const T* src = static_cast<const T*>(a.src);
    const int own = __ldg(t);
    T b[L::Q];
    b[0] = __ldg(src + own);
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        b[i] = __ldg(src + __ldg(t + i * P));
    });
    const int stride = __ldg(t + L::Q * P);
    T* out = static_cast<T*>(a.dst) + own;
    if (!collide_ff<L, MODEL>(b, a.fx, a.ffc, out, stride)) {
        // out of range: the same update in native FP64 (a call, off the hot path)
        update_fp64_table<L, MODEL>(a, t, out, stride);
    }
}

template <class L, int MODEL>
cudaError_t launch_step_ff_table(const StepArgs& a, cudaStream_t s) {
    if (a.n_nodes == 0) return cudaSuccess;
    k_step_ff_table<L, MODEL><<<(unsigned)((a.n_nodes + kTableThreads - 1) / kTableThreads), kTableThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class L, int A>
cudaError_t launch_gather_table(const StepArgs& a, cudaStream_t s) {
    if (a.n_work_blocks == 0) return cudaSuccess;
    k_gather_table<L, A><<<a.n_work_blocks, work_threads<L, A>(), 0, s>>>(a);
    return cudaGetLastError();
}

StepLaunch select_step_ff_table(int lattice, int a, int model) {
    const bool qc = model == LBM_QUASI_COMPRESSIBLE;
    if (lattice == LBM_D2Q9 && (a == 8 || a == 16 || a == 32))
        return qc ? &launch_step_ff_table<D2Q9, LBM_QUASI_COMPRESSIBLE> : &launch_step_ff_table<D2Q9, LBM_INCOMPRESSIBLE>;
    if (lattice == LBM_D3Q19 && (a == 4 || a == 8))
        return qc ? &launch_step_ff_table<D3Q19, LBM_QUASI_COMPRESSIBLE> : &launch_step_ff_table<D3Q19, LBM_INCOMPRESSIBLE>;
    return nullptr;
}

StepLaunch select_gather_table_builder(int lattice, int a) {
    if (lattice == LBM_D2Q9) {
        if (a == 8) return &launch_gather_table<D2Q9, 8>;
        if (a == 16) return &launch_gather_table<D2Q9, 16>;
        if (a == 32) return &launch_gather_table<D2Q9, 32>;
    } else if (lattice == LBM_D3Q19) {
        if (a == 4) return &launch_gather_table<D3Q19, 4>;
        if (a == 8) return &launch_gather_table<D3Q19, 8>;
    }
    return nullptr;
}

}  // namespace lbm

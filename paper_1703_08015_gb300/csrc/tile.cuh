// tile.cuh -- device side of the tiled step: staging of a tile's
// neighbourhood in shared memory and the gather (streaming) of Fig. 5.
//
// One thread owns one fluid node; a block takes the fluid nodes of up to 16
// consecutive tiles (a work block).  Before the single barrier, the block's
// threads copy the 3^d neighbour record of each of its tiles into shared
// memory as offsets of the neighbours' PDF blocks, together with the
// neighbours' fluid-node bit masks (the copy of the tile bitmap and the node
// types of the tile and its halo that Fig. 5 stages).  After the barrier every
// fluid node pulls f*_i(r - c_i) from the tile that holds r - c_i, or, when
// that node is solid, in a removed tile or beyond a wall, its own
// f*_{opp(i)}(r) (halfway bounce-back).
#pragma once

#include <cuda_fp16.h>

#include "internal.h"
#include "lattice.cuh"

namespace lbm {

// The neighbourhood of the tiles of one block.  PDF blocks are addressed from
// the block's origin (the compact offset of its first tile) with 32-bit value
// offsets; the tiling checks that every neighbour lies within 2^30 values.
template <class TL, int TPB>
struct NeighShared {
    int2 loc[TPB][TL::NN];           // x: the slot's PDF block, values from the origin; y: values per link
    uint64_t m[TPB][TL::NN][TL::W];  // its fluid-node bits (0 when removed)
    long long origin;                // compact offset of the block's first tile (values)
};

// Rank of node n among the fluid nodes of a tile (its slot in the compact
// layout): the number of fluid bits below bit n.
template <int W>
__device__ __forceinline__ int fluid_rank(const uint64_t* m, int n) {
    const int w = n >> 6;
    int r = __popcll(m[w] & ((1ull << (n & 63)) - 1ull));
    if constexpr (W > 1) {
#pragma unroll
        for (int k = 0; k < W - 1; k++)
            if (k < w) r += __popcll(m[k]);
    }
    return r;
}

// Fluid bit of node n and, when set, its rank (see fluid_rank): the word is
// shifted so that bit n lands in the sign bit; the popcount then counts the
// bits at and below n.
template <int W>
__device__ __forceinline__ int fluid_bit_rank(const uint64_t* m, int n, bool& fl) {
    const unsigned long long t = (W == 1 ? m[0] : m[n >> 6]) << (63 - (n & 63));
    fl = (long long)t < 0;
    int r = __popcll(t) - (int)fl;
    if constexpr (W > 1) {
        const int w = n >> 6;
#pragma unroll
        for (int k = 0; k < W - 1; k++)
            if (k < w) r += __popcll(m[k]);
    }
    return r;
}

template <class TL, int TPB>
__device__ __forceinline__ bool mask_bit(const NeighShared<TL, TPB>& sh, int lt, int slot, int n) {
    if constexpr (TL::W == 1)
        return (sh.m[lt][slot][0] >> n) & 1ull;
    else
        return (sh.m[lt][slot][n >> 6] >> (n & 63)) & 1ull;
}

template <int A>
struct NodePos {
    int lx, ly, lz;
};

template <class TL>
__device__ __forceinline__ NodePos<(1 << TL::LA)> node_pos(int node) {
    constexpr int A = 1 << TL::LA;
    NodePos<A> p;
    p.lx = node & (A - 1);
    p.ly = (node >> TL::LA) & (A - 1);
    p.lz = TL::D == 3 ? node >> (2 * TL::LA) : 0;
    return p;
}

// Per node, once: for each axis and each link component c in {-1, 0, +1}
// (index c + 1), the source coordinate (r - c) mod A already shifted into the
// node index, and the step to the neighbour slot (in slot units of that axis)
// when r - c leaves the tile.
template <class L, int A>
struct PullBase {
    using TL = Tile<L, A>;
    int nx[3], ny[3], nz[3];  // shifted source coordinates
    int tx[3], ty[3], tz[3];  // slot steps: 1, 3, 9 per tile along x, y, z
    __device__ __forceinline__ PullBase(const NodePos<A>& p) {
        nx[0] = (p.lx + 1) & (A - 1);
        nx[1] = p.lx;
        nx[2] = (p.lx - 1) & (A - 1);
        ny[0] = ((p.ly + 1) & (A - 1)) << TL::LA;
        ny[1] = p.ly << TL::LA;
        ny[2] = ((p.ly - 1) & (A - 1)) << TL::LA;
        tx[0] = p.lx == A - 1;
        tx[1] = 0;
        tx[2] = -(p.lx == 0);
        ty[0] = 3 * (p.ly == A - 1);
        ty[1] = 0;
        ty[2] = -3 * (p.ly == 0);
        if (TL::D == 3) {
            nz[0] = ((p.lz + 1) & (A - 1)) << (2 * TL::LA);
            nz[1] = p.lz << (2 * TL::LA);
            nz[2] = ((p.lz - 1) & (A - 1)) << (2 * TL::LA);
            tz[0] = 9 * (p.lz == A - 1);
            tz[1] = 0;
            tz[2] = -9 * (p.lz == 0);
        } else {
            nz[0] = nz[1] = nz[2] = 0;
            tz[0] = tz[1] = tz[2] = 0;
        }
    }
};

// Source of the pull along link I: the neighbour slot and node index that
// hold r - c_I.
template <class L, int A, int I>
struct PullSource {
    using TL = Tile<L, A>;
    using K = Link<L, I>;
    int slot, sn;
    __device__ __forceinline__ PullSource(const PullBase<L, A>& b) {
        slot = TL::CENTER + b.tx[K::cx + 1] + b.ty[K::cy + 1] + b.tz[K::cz + 1];
        sn = b.nx[K::cx + 1] | b.ny[K::cy + 1] | b.nz[K::cz + 1];
    }
    __device__ __forceinline__ PullSource(const NodePos<A>& p) {
        const int sx = p.lx - K::cx, sy = p.ly - K::cy, sz = p.lz - K::cz;
        const int tx = K::cx > 0 ? -(sx < 0) : (K::cx < 0 ? (sx >= A) : 0);
        const int ty = K::cy > 0 ? -(sy < 0) : (K::cy < 0 ? (sy >= A) : 0);
        const int tz = K::cz > 0 ? -(sz < 0) : (K::cz < 0 ? (sz >= A) : 0);
        slot = TL::CENTER + tx + 3 * ty + 9 * tz;
        sn = (sx & (A - 1)) | ((sy & (A - 1)) << TL::LA) | ((sz & (A - 1)) << (2 * TL::LA));
    }
};

// Gather the q post-collision words that arrive at `node` (raw storage words)
// from the compact blocks; returns the node's own slot (its fluid rank).
template <class L, int A, int TPB, class T>
__device__ __forceinline__ int gather(const NeighShared<Tile<L, A>, TPB>& sh, const void* pdf, int lt, int node,
                                      const NodePos<A>& p, T (&f)[L::Q]) {
    using TL = Tile<L, A>;
    const T* org = static_cast<const T*>(pdf) + sh.origin;
    const int2 own = sh.loc[lt][TL::CENTER];
    const int own_rank = fluid_rank<TL::W>(sh.m[lt][TL::CENTER], node);
    const int own_r = own.x + own_rank;  // bounce-back sources: own_r + opp * own.y
    f[0] = __ldg(org + own_r);
    const PullBase<L, A> pb(p);
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const PullSource<L, A, i> s(pb);
        bool fl;
        const int r = fluid_bit_rank<TL::W>(sh.m[lt][s.slot], s.sn, fl);
        const int2 nb = sh.loc[lt][s.slot];
        const int idx = fl ? nb.x + i * nb.y + r : own_r + Link<L, i>::opp * own.y;
        f[i] = __ldg(org + idx);
    });
    return own_rank;
}

// The node's own values in a copy laid out like the source: base + i * stride.
template <class TL, int TPB, class T>
__device__ __forceinline__ T* own_slot(const NeighShared<TL, TPB>& sh, void* pdf, int lt, int rank) {
    return static_cast<T*>(pdf) + sh.origin + sh.loc[lt][TL::CENTER].x + rank;
}

// ---- storage policies: raw words <-> FP64 values ------------------------------
struct StoreF64 {
    using T = unsigned long long;
    static constexpr int id = LBM_STORE_F64;
    template <class L, int I>
    __device__ static __forceinline__ double to_f64(T r, double) { return __longlong_as_double((long long)r); }
    template <class L, int I>
    __device__ static __forceinline__ T from_f64(double v, double) { return (T)__double_as_longlong(v); }
};

struct StoreF32 {
    using T = unsigned int;
    static constexpr int id = LBM_STORE_F32;
    template <class L, int I>
    __device__ static __forceinline__ double to_f64(T r, double) { return (double)__uint_as_float(r); }
    template <class L, int I>
    __device__ static __forceinline__ T from_f64(double v, double) { return __float_as_uint((float)v); }
};

// FP32 holding the deviation f_i - w_i.
struct StoreF32S {
    using T = unsigned int;
    static constexpr int id = LBM_STORE_F32S;
    template <class L, int I>
    __device__ static __forceinline__ double to_f64(T r, double) {
        return Link<L, I>::w + (double)__uint_as_float(r);
    }
    template <class L, int I>
    __device__ static __forceinline__ T from_f64(double v, double) {
        return __float_as_uint((float)(v - Link<L, I>::w));
    }
};

// FP16 holding the scaled deviation (f_i - w_i) * scale.
struct StoreF16S {
    using T = unsigned short;
    static constexpr int id = LBM_STORE_F16S;
    template <class L, int I>
    __device__ static __forceinline__ double to_f64(T r, double inv_scale) {
        return Link<L, I>::w + (double)__half2float(__ushort_as_half(r)) * inv_scale;
    }
    template <class L, int I>
    __device__ static __forceinline__ T from_f64(double v, double scale) {
        return __half_as_ushort(__float2half_rn((float)((v - Link<L, I>::w) * scale)));
    }
};

template <class L, int A>
constexpr int tiles_per_block() {
    return Tile<L, A>::NT >= 256 ? 1 : 256 / Tile<L, A>::NT;
}

// ---- work lists: one thread per fluid node ------------------------------------
// The host packs the fluid nodes of consecutive tiles into blocks of at most
// work_threads<L,A>() nodes and work_tiles() tiles (see WorkBlock in
// internal.h), so no lane of the step kernels idles on a solid node.
template <class L, int A>
constexpr int work_threads() {
    return Tile<L, A>::NT > 256 ? Tile<L, A>::NT : 256;
}
constexpr int work_tiles() { return 16; }

struct WorkNode {
    int lt, tile, node;
};

// Resident blocks per SM the float-float and fixed-point FP64 steps ask the
// compiler to allow (it caps their registers): three blocks of 256 threads
// (80 registers; two blocks measured slower), two of 512 (64 registers: the
// 8^3-tile D3Q19 step spills 168 B but runs at 644 against 909 us per 256^3
// step with one block of 128 registers).
template <class L, int A>
constexpr int fp64_step_min_blocks() {
    return work_threads<L, A>() <= 256 ? 3 : (work_threads<L, A>() <= 512 ? 2 : 1);
}

// The block's BT threads copy the neighbourhoods of work block `wb`'s tiles
// into `sh` (visible to the block after the next barrier), and the neighbour
// tile indices into `nbt` when given.  The entries a thread copies are
// unrolled so that the loads of all of them are in flight together: one round
// trip for the neighbour indices, one for what they point at, whatever the
// number of entries per thread.
template <class TL, int KMAX, int BT>
__device__ __forceinline__ void stage_tables(NeighShared<TL, KMAX>& sh, const StepArgs& a, const WorkBlock& wb,
                                             int (*nbt)[TL::NN] = nullptr) {
    constexpr int PER_TILE = TL::NN * TL::W;
    constexpr int R = (KMAX * PER_TILE + BT - 1) / BT;  // entries per thread, at most
    const long long origin = __ldg(a.tile_off + wb.tile_begin);
    if (threadIdx.x == 0) sh.origin = origin;
    const int total = wb.n_tiles * PER_TILE;
    int nb[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int k = (int)threadIdx.x + r * BT;
        nb[r] = -1;
        if (k < total) {
            const int lt = k / PER_TILE, slot = (k - lt * PER_TILE) / TL::W;
            nb[r] = __ldg(a.nbr + (size_t)(wb.tile_begin + lt) * TL::NN + slot);
        }
    }
    uint64_t m[R];
    int2 loc[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int k = (int)threadIdx.x + r * BT;
        const int w = k % TL::W;
        m[r] = 0ull;
        loc[r] = make_int2(0, 0);
        if (nb[r] >= 0) {
            if (w == 0) {  // mask word 0, offset and stride in one record
                const ulonglong2 t = __ldg(a.tinfo + nb[r]);
                m[r] = t.x;
                loc[r] = make_int2((int)((long long)(t.y >> 24) - origin), (int)(t.y & 0xFFFFFFull));
            } else {
                m[r] = __ldg(a.tmask + (size_t)nb[r] * TL::W + w);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int k = (int)threadIdx.x + r * BT;
        if (k < total) {
            const int lt = k / PER_TILE, rem = k - lt * PER_TILE;
            const int slot = rem / TL::W, w = rem - slot * TL::W;
            sh.m[lt][slot][w] = m[r];
            if (w == 0) {
                sh.loc[lt][slot] = loc[r];
                if (nbt) nbt[lt][slot] = nb[r];
            }
        }
    }
}

// Stage the neighbourhoods of the block's tiles, then decode this thread's
// fluid node.  Every thread of the block must call it (it holds the barrier);
// returns false for threads beyond the block's node count.
template <class TL, int KMAX, int BT>
__device__ __forceinline__ bool stage_work_at(NeighShared<TL, KMAX>& sh, const StepArgs& a, int wbi,
                                              WorkNode& wn) {
    const WorkBlock wb = a.blocks[wbi];
    const bool active = (int)threadIdx.x < wb.count;
    const uint32_t e = active ? __ldg(a.nodes + wb.node_begin + threadIdx.x) : 0u;  // in flight during the staging
    stage_tables<TL, KMAX, BT>(sh, a, wb);
    __syncthreads();  // the only barrier of the step (Fig. 5)
    if (!active) return false;
    wn.tile = (int)(e >> (TL::D * TL::LA));
    wn.node = (int)(e & (TL::NT - 1));
    wn.lt = wn.tile - wb.tile_begin;
    return true;
}

template <class TL, int KMAX, int BT>
__device__ __forceinline__ bool stage_work(NeighShared<TL, KMAX>& sh, const StepArgs& a, WorkNode& wn) {
    return stage_work_at<TL, KMAX, BT>(sh, a, blockIdx.x, wn);
}

// ---- staging from the per-tile neighbour table (tiles of one mask word) ---------
// The neighbour records of a work block's tiles lie back to back in the table
// (NRec, built once at initialisation), so the block copies them with one
// dependent load instead of two (neighbour index, then that tile's record),
// as asynchronous 16-byte copies that hold no registers; offsets are relative
// to each tile's own PDF block.
template <class TL, int TPB>
struct RecShared {
    static_assert(TL::W == 1, "neighbour records hold one mask word");
    NRec rec[TPB][TL::NN];
    long long toff[TPB];  // each tile's own PDF block (values)
};

__device__ __forceinline__ void cp_async16_l2(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async8_l1(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Ask the L2 for [p, p + bytes) (16-byte aligned, a multiple of 16 bytes);
// no registers or shared memory are held while the lines arrive.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// [b0, b1) of an array of `limit` bytes, widened to 16-byte bounds (the end
// clamped to the last whole 16 bytes), requested from the L2.
__device__ __forceinline__ void prefetch_l2_range(const void* base, long long b0, long long b1, long long limit) {
    b0 &= ~15ll;
    b1 = (b1 + 15) & ~15ll;
    if (b1 > (limit & ~15ll)) b1 = limit & ~15ll;
    if (b1 > b0) prefetch_l2_bulk(static_cast<const char*>(base) + b0, (unsigned)(b1 - b0));
}

// What work block `w` will read, requested from the L2 ahead of its run (see
// StepArgs::pf_ahead): its source range and, with pf_tables, its entries of
// the node list and its tiles' neighbour records (or neighbour indices).
template <int NN>
__device__ __forceinline__ void prefetch_work_block(const StepArgs& a, const WorkBlock& w) {
    const long long nb = a.pf_node_bytes;
    prefetch_l2_range(a.src, w.node_begin * nb, (long long)(w.node_begin + w.count) * nb, a.pf_limit);
    if (a.pf_tables) {
        prefetch_l2_range(a.nodes, 4ll * w.node_begin, 4ll * (w.node_begin + w.count), 4ll * a.n_nodes);
        const long long t0 = (long long)w.tile_begin * NN, t1 = (long long)(w.tile_begin + w.n_tiles) * NN;
        if (a.ntab)
            prefetch_l2_range(a.ntab, t0 * (long long)sizeof(NRec), t1 * (long long)sizeof(NRec),
                              (long long)a.n_tiles * NN * (long long)sizeof(NRec));
        else
            prefetch_l2_range(a.nbr, 4 * t0, 4 * t1, 4ll * a.n_tiles * NN);
    }
}

template <class TL, int KMAX, int BT>
__device__ __forceinline__ bool stage_work_rec(RecShared<TL, KMAX>& sh, const StepArgs& a, WorkNode& wn) {
    const WorkBlock wb = a.blocks[blockIdx.x];
    const bool active = (int)threadIdx.x < wb.count;
    const uint32_t e = active ? __ldg(a.nodes + wb.node_begin + threadIdx.x) : 0u;  // in flight during the copies
    const int total = wb.n_tiles * TL::NN;
    const NRec* src = a.ntab + (size_t)wb.tile_begin * TL::NN;
    for (int k = (int)threadIdx.x; k < total; k += BT) cp_async16_l2(&sh.rec[0][0] + k, src + k);
    if ((int)threadIdx.x < wb.n_tiles) cp_async8_l1(&sh.toff[threadIdx.x], a.tile_off + wb.tile_begin + threadIdx.x);
    cp_async_wait_all();
    __syncthreads();  // the only barrier of the step (Fig. 5)
    if (!active) return false;
    wn.tile = (int)(e >> (TL::D * TL::LA));
    wn.node = (int)(e & (TL::NT - 1));
    wn.lt = wn.tile - wb.tile_begin;
    return true;
}

// gather() from the staged records: the q post-collision words that arrive
// at `node`; returns the node's values in the copy `dst` and sets its values
// per link.
template <class L, int A, int TPB, class T>
__device__ __forceinline__ T* gather_rec(const RecShared<Tile<L, A>, TPB>& sh, const void* pdf, void* dst, int lt,
                                         int node, const NodePos<A>& p, T (&f)[L::Q], int& stride) {
    using TL = Tile<L, A>;
    const long long toff = sh.toff[lt];
    const T* org = static_cast<const T*>(pdf) + toff;
    const NRec own = sh.rec[lt][TL::CENTER];  // offset 0: the tile itself
    const int own_r = __popcll(own.m & ((1ull << node) - 1ull));
    f[0] = __ldg(org + own_r);
    const PullBase<L, A> pb(p);
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const PullSource<L, A, i> s(pb);
        const NRec nb = sh.rec[lt][s.slot];
        // bit s.sn into the sign bit: the popcount counts the bits at and below it
        const unsigned long long t = nb.m << (63 - s.sn);
        const bool fl = (long long)t < 0;
        const int r = __popcll(t) - (int)fl;
        const int idx = fl ? nb.off + i * nb.stride + r : own_r + Link<L, i>::opp * own.stride;
        f[i] = __ldg(org + idx);
    });
    stride = own.stride;
    return static_cast<T*>(dst) + toff + own_r;
}

}  // namespace lbm

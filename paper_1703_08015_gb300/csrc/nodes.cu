// nodes.cu -- kernels that visit every node of every non-empty tile once:
// equilibrium start, moments with FP64 reductions, and dense export/import
// of the PDFs.  None of them is on the per-step path.
#include <cmath>

#include "collide_f64.cuh"
#include "tile.cuh"

namespace lbm {

constexpr int kStats = 8;  // mass, momentum x/y/z, |u|^2, |u - u_saved|^2, fluid count, spare

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
template <class L, int A, int TPB, int MODEL, class S>
__global__ void __launch_bounds__(TPB* Tile<L, A>::NT) k_moments(const NodeArgs a) {
    using TL = Tile<L, A>;
    using T = typename S::T;
    constexpr int NTH = TPB * TL::NT;
    __shared__ NeighShared<TL, TPB> sh;
    __shared__ double red[NTH / 32][kStats];
    const int lt = threadIdx.x / TL::NT;
    const int node = threadIdx.x - lt * TL::NT;
    const int tile = a.tile_begin + blockIdx.x * TPB + lt;
    const int tile_end = a.tile_begin + a.n_tiles;
    stage_neighbourhood<TL, TPB>(sh, a.nbr, a.tmask, a.tile_off, a.tile_stride, a.tile_begin + blockIdx.x * TPB,
                                 tile_end, tile, lt, node);
    __syncthreads();
    double acc[kStats];
#pragma unroll
    for (int k = 0; k < kStats; k++) acc[k] = 0.0;
    const NodePos<A> p = node_pos<TL>(node);
    size_t n = 0;
    const bool want_fields = a.rho_out || a.u_out;
    if (tile < tile_end && mask_bit(sh, lt, TL::CENTER, node) && (!want_fields || dense_index<L, A>(a, tile, p, n))) {
        T raw[L::Q];
        gather<L, A, TPB, T>(sh, a.pdf, lt, node, p, raw);
        double f[L::Q];
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            f[i] = S::template to_f64<L, i>(raw[i], a.f16_inv_scale);
        });
        double rho, jx, jy, jz, ux, uy, uz;
        moments_f64<L>(f, rho, jx, jy, jz);
        velocity_f64<L, MODEL>(rho, jx, jy, jz, a.force, ux, uy, uz);
        const size_t N = (size_t)a.nx * a.ny * a.nz;  // fields only for a single-sample launch
        if (a.rho_out) a.rho_out[n] = rho;
        if (a.u_out) {
            a.u_out[n] = ux;
            a.u_out[N + n] = uy;
            if (L::D == 3) a.u_out[2 * N + n] = uz;
        }
        acc[0] = rho;
        acc[1] = rho * ux;
        acc[2] = rho * uy;
        acc[3] = rho * uz;
        acc[4] = ux * ux + uy * uy + uz * uz;
        if (a.residual && a.u_saved) {
            double* us = a.u_saved + (size_t)tile * 3 * TL::NT + node;
            const double dx = ux - us[0], dy = uy - us[TL::NT], dz = uz - us[2 * TL::NT];
            acc[5] = dx * dx + dy * dy + dz * dz;
            us[0] = ux;
            us[TL::NT] = uy;
            us[2 * TL::NT] = uz;
        }
        acc[6] = 1.0;
    }
    // deterministic block sum: butterfly within each warp, then warps in order
#pragma unroll
    for (int k = 0; k < kStats; k++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kStats; k++) red[warp][k] = acc[k];
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
    const int blocks = (a.n_tiles + TPB - 1) / TPB;
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
    return (n_tiles + tpb - 1) / tpb;
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

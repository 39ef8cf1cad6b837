// internal.h -- host-side declarations shared by the library's translation
// units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <utility>
#include <vector>

#include "lbm.h"

namespace lbm {

// ---- errors ---------------------------------------------------------------
int fail(int code, const char* fmt, ...);          // records a message, returns code
int cuda_fail(cudaError_t e, const char* what);    // LBM_ERR_CUDA or LBM_ERR_OOM

#define LBM_CUDA_TRY(call)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ::lbm::cuda_fail(e_, #call); \
    } while (0)

// A block of the step kernels: `count` consecutive entries of the fluid-node
// list starting at `node_begin`, drawn from the `n_tiles` consecutive
// non-empty tiles starting at `tile_begin`.
struct WorkBlock {
    int node_begin, count, tile_begin, n_tiles;
};

// One neighbour slot of a tile whose fluid nodes fit one mask word (the
// per-tile neighbourhood table of the float-float step): the neighbour's
// fluid-node bits, its PDF block relative to the tile's own (values; the
// tiling keeps every neighbour within 2^30 values), its values per link.
// All zero for an empty slot.
struct alignas(16) NRec {
    unsigned long long m;
    int off, stride;
};

// ---- host tiling ------------------------------------------------------------
// An allocator whose default construction leaves trivial elements as they
// are: resize() of a vector the tiling then fills completely (in parallel)
// skips a serial zero fill and its first-touch page faults.
template <class T>
struct fill_later_alloc : std::allocator<T> {
    fill_later_alloc() = default;
    template <class U>
    fill_later_alloc(const fill_later_alloc<U>&) noexcept {}
    template <class U>
    struct rebind {
        using other = fill_later_alloc<U>;
    };
    template <class U>
    void construct(U* p) noexcept {
        ::new (static_cast<void*>(p)) U;
    }
    template <class U, class... Args>
    void construct(U* p, Args&&... args) {
        ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
    }
};
template <class T>
using fill_vector = std::vector<T, fill_later_alloc<T>>;

struct HostTiling {
    lbm_tiling info{};
    int a = 0, d = 0, nn = 0, words = 0;     // edge, dimension, 3^d, mask words per tile
    std::vector<int32_t> tile_map;           // [n_tiles]
    fill_vector<int32_t> nbr;                // [n_ftiles][nn]
    fill_vector<uint64_t> tmask;             // [n_ftiles][words], bit n = node n fluid
    fill_vector<int32_t> coords;             // [n_ftiles][3] tile coordinates
    std::vector<long long> tile_off;         // [n_ftiles] first value of the tile's PDF block
    std::vector<int32_t> tile_stride;        // [n_ftiles] values per link (fluid count, sector-padded)
    std::vector<uint32_t> nodes;             // fluid nodes, tile-major: tile * NT + node
    std::vector<WorkBlock> blocks;           // step-kernel blocks over `nodes`
};
// The tiles of one sample of a batch (a single geometry is a batch of one).
struct SampleRange {
    int nx, ny, nz;
    int tile_begin, n_tiles;
    long long n_fluid;
};
int build_batch_tiling(const lbm_params* p, int n, const int* dims, const uint8_t* const* masks, HostTiling* T,
                       std::vector<SampleRange>* samples);
int validate_params(const lbm_params* p);
// host_nbr false: no neighbour records (T->nbr stays empty) and no check of
// neighbour distances; the caller builds both on the device (launch_build_nbr)
int build_tiling(const lbm_params* p, const uint8_t* mask, HostTiling* out, bool host_nbr = true);
// Step-kernel blocks of at most `threads` nodes and `max_tiles` tiles each,
// and (want_nodes) the fluid-node list on the host; returns the number of
// fluid nodes (entries of the list).  With split_tiles a tile's nodes may be
// shared by two consecutive blocks, so that every block but the last holds
// `threads` nodes (only for steps that read one copy and write the other:
// the in-place ghost-buffer step updates a tile from one block).
long long build_work_list(HostTiling* T, int threads, int max_tiles, bool want_nodes = true, bool split_tiles = false);
int work_threads_for(int lattice, int a);
int lattice_q(int lattice);
size_t bytes_per_value(int storage);

// ---- kernel arguments --------------------------------------------------------
// Constants of the fixed-point FP64 path (values scaled by 2^60 = "Q60"
// unless stated; w = 1/tau, c = weight class, i = link).
struct FixedConsts {
    long long w_bits[3];  // FP64 bit patterns of the class weights w_c
    long long w60[3];     // w_c in Q60 (exact)
    long long kw[3];      // w_c * 2^62
    long long k_keep;     // (1 - w) * 2^62
    long long k_rho[3];   // w * w_c * 2^62
    long long k_j[3];     // 3 w w_c * 2^61
    long long alpha;      // 4.5 w * 2^59
    long long g1;         // 1.5 w * 2^61
    long long kf[3];      // 3 (1 - w/2) F_a in Q60
    long long half_f[3];  // F_a / 2 in Q60
    long long beta[19];   // 9 (1 - w/2) (c_i.F) in Q60
    long long so[19];     // 3 (1 - w/2) w_i (c_i.F) in Q60
    long long dws;        // sum_i w_i in Q60, minus 2^60 (exact)
};

// Two float-float constants laid out for the f32x2 instructions: the high
// parts of lanes 0 and 1, then their low parts.
struct FF2C {
    float2 h, l;
};

// Constants of the float-float FP64 path: each a (hi, lo) pair of floats.
struct FFConsts {      // u_c = 1 / ulp(w_c): class quantities in ulps of w_c
    float2 w[3];       // w_c u_c
    float2 rho[3];     // w * w_c u_c
    float2 j[3];       // 3 w w_c u_c
    float2 keep;       // 1 - w
    float2 alpha;      // 4.5 w
    float2 g1;         // 1.5 w
    float2 kf[3];      // 3 (1 - w/2) F_a
    float2 beta[19];   // 9 (1 - w/2) (c_i.F)
    float2 so[19];     // 3 (1 - w/2) w_i (c_i.F) u_c
    // the same, two lanes at a time: (x, x) for keep and alpha, classes (1, 2)
    // for w and rho, (kf_x, kf_y), and per group of two pairs of opposite
    // links (first links a_g, b_g) beta, j of their classes and so
    FF2C keep2, alpha2, w12, rho12, kf01;
    FF2C w11, w22, rho11, rho22;  // (w_c, w_c) and (w w_c, w w_c) of classes 1 and 2
    FF2C beta2[4], j2[4], so2[4];
};

// Constants of the FP32 collision (reduced storage forms), per weight class c
// and per link i.
struct F32Consts {
    float keep;      // 1 - w
    float ow[3];     // w * w_c
    float kw3[3];    // 3 (1 - w/2) w_c
    float be[19];    // 9 (1 - w/2) w_i (c_i.F)
    float so[19];    // 3 (1 - w/2) w_i (c_i.F)
};

struct StepArgs {
    const WorkBlock* blocks;  // [n_work_blocks]
    const uint32_t* nodes;    // fluid-node list: tile * NT + node
    int n_work_blocks;
    const void* src;
    void* dst;
    const void* ghost_in;  // ghost-buffer form: the set written by the previous step
    void* ghost_out;       // ghost-buffer form: the set this step writes
    const int32_t* nbr;
    const uint64_t* tmask;
    const long long* tile_off;  // compact layout: PDF block of each tile (in values)
    const int32_t* tile_stride; // compact layout: values per link of each tile
    const ulonglong2* tinfo;    // per tile, one 16-byte record: {first fluid-mask word, tile_off << 24 | tile_stride}
    const NRec* ntab;           // [n_tiles][3^d] neighbour records (one-word tiles, float-float step) or NULL
    // L2 prefetch of the source values ahead of the blocks that read them:
    // block b asks the L2 for the range of work block b + pf_ahead (0: off).
    // A copy holds pf_node_bytes per fluid node with the tiles in work-list
    // order, so the ranges [node_begin, node_begin + count) * pf_node_bytes
    // of the work blocks partition it, each about its own tiles' values;
    // clamped to pf_limit bytes
    int pf_ahead;
    int pf_tables;  // also the block's node-list entries and neighbour records
    int pf_node_bytes;
    long long pf_limit;
    int n_tiles;
    long long n_nodes;          // fluid nodes (entries of the work list)
    const int32_t* gtab;        // FP64 gather table [q + 1][gtab_pitch] (see k_gather_table) or NULL
    int32_t* gtab_out;          // the same table, written once at initialisation
    long long gtab_pitch;
    double omega;         // 1 / tau
    double tau;
    double force[3];
    double f16_scale;     // storage scale for LBM_STORE_F16S
    double f16_inv_scale;
    float omega_f, force_f[3], f16_scale_f, f16_inv_scale_f;
    FixedConsts fx;
    FFConsts ffc;
    F32Consts f32c;
};

struct NodeArgs {         // kernels that visit every node of every tile
    const void* pdf;      // current copy
    void* pdf_out;        // second copy (init writes both)
    const int32_t* nbr;
    const uint64_t* tmask;
    const int32_t* coords;
    const long long* tile_off;
    const int32_t* tile_stride;
    int tile_begin;           // first tile of this launch (a sample of a batch)
    int n_tiles;              // tiles of this launch
    int nx, ny, nz;
    double force[3];
    double rho0;
    double f16_scale, f16_inv_scale;
    const double* rho_in;     // dense or NULL
    const double* u_in;       // dense [3][N] or NULL
    double* rho_out;          // dense or NULL
    double* u_out;            // dense [3][N] or NULL
    double* dense_pdf;        // dense [q][N]
    const double* dense_pdf_in;
    const ulonglong2* tinfo;  // per tile: {first fluid-mask word, tile_off << 24 | tile_stride}
    long long n_slots;        // fluid-node slots of one link (values of a PDF copy / q)
    float2* u_saved;          // [3][n_slots] velocity of the last residual check (float-float) or NULL
    int residual;             // compare and save velocity
    double* partials;         // [blocks][8]
};

using StepLaunch = cudaError_t (*)(const StepArgs&, cudaStream_t);
// The fluid-node list of build_work_list written on the device from the tile
// masks and compact offsets (nullptr when a geometry is not compiled).
using NodeListLaunch = cudaError_t (*)(const uint64_t* tmask, const long long* tile_off, int n_tiles,
                                       uint32_t* nodes, cudaStream_t);
NodeListLaunch select_node_list(int lattice, int a);
using NodeLaunch = cudaError_t (*)(const NodeArgs&, cudaStream_t);

// Kernel selection (nullptr when a combination is not compiled).
StepLaunch select_step(const lbm_params* p);
void f32_consts(const lbm_params* p, double omega, const double* force, F32Consts* k);
StepLaunch select_step_tgb(const lbm_params* p);
// The float-float FP64 step that reads its sources from a gather table, and
// the kernel that builds the table once (nullptr when not compiled).
StepLaunch select_step_ff_table(int lattice, int a, int model);
// The axis of a D3Q19 body force with one nonzero component (0 for no force),
// else -1: the float-float step then leaves out the forcing terms of the
// links with c_i . F = 0.
int ff_force_axis(int lattice, const double force[3]);
StepLaunch select_gather_table_builder(int lattice, int a);
StepLaunch select_tgb_publish(int lattice, int a, int storage);
long long tgb_ghost_per_tile(int lattice, int a);
NodeLaunch select_init(int lattice, int a, int model, int storage);
NodeLaunch select_moments(int lattice, int a, int model, int storage);
NodeLaunch select_export(int lattice, int a, int storage);
NodeLaunch select_import(int lattice, int a, int storage);
int node_blocks(int lattice, int a, int n_tiles);  // grid (= partial sums) of the moments kernel
cudaError_t launch_fill_nan(double* p, size_t n, cudaStream_t s);
// the neighbour records of the compact tiles from their coordinates and the
// dense tile map (build_tiling's rule); a check that no neighbour lies more
// than 2^30 values away (*far set to 1, else left as it is)
cudaError_t launch_build_nbr(const int32_t* coords, const int32_t* tile_map, int n_ftiles, int d, int ntx, int nty,
                             int ntz, const int per[3], int32_t* nbr, cudaStream_t s);
cudaError_t launch_far_check(const int32_t* nbr, const long long* tile_off, int n_ftiles, int nn, unsigned* far,
                             cudaStream_t s);
// ntab[t][slot] from nbr, tmask (one word per tile), tile_off, tile_stride
cudaError_t launch_build_ntab(const int32_t* nbr, const uint64_t* tmask, const long long* tile_off,
                              const int32_t* tile_stride, int n_tiles, int nn, NRec* ntab, cudaStream_t s);
cudaError_t launch_average(void* cur, const void* prev, size_t bytes, int storage, cudaStream_t s);
cudaError_t launch_reduce(const double* partials, int nblocks, double* result, cudaStream_t s);

void fixed_consts(const lbm_params* p, FixedConsts* k);
void ff_consts(const lbm_params* p, FFConsts* k);

}  // namespace lbm

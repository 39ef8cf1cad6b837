// api.cu -- the C ABI of include/lbm.h: context life cycle, stepping (with a
// captured CUDA graph of several steps), moments and PDF export/import.
#include <cmath>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>

#include "internal.h"

namespace lbm {
StepLaunch select_step_f64(int lattice, int a, int model, int storage);
StepLaunch select_step_fixed(int lattice, int a, int model);
StepLaunch select_step_f32(int lattice, int a, int model, int storage, int block_nodes, int persistent);

StepLaunch select_step_ff(int lattice, int a, int model, int block_nodes, int fax);

// Fluid nodes per work block of the step kernel: the caller's choice, else
// 128 for the float-float FP64 step on tiles of at most 128 nodes where a
// block would hold 256 (six blocks
// of 128 per SM interleave staging, gather and collision more finely than
// three of 256: 2-6 % faster, the same bits), else work_threads_for.
int step_block_nodes(const lbm_params* p) {
    if (p->block_nodes) return p->block_nodes;
    const int bd = work_threads_for(p->lattice, p->tile_a);
    const int nt = p->lattice == LBM_D3Q19 ? p->tile_a * p->tile_a * p->tile_a : p->tile_a * p->tile_a;
    if (p->layout != LBM_LAYOUT_TGB && p->storage == LBM_STORE_F64 && !p->persistent && bd == 256 && nt <= 128 &&
        (p->arith == LBM_ARITH_FF || p->arith == LBM_ARITH_AUTO))
        return 128;  // a work block never splits a tile: only tiles of up to 128 nodes
    return bd;
}

StepLaunch select_step(const lbm_params* p) {
    const int lattice = p->lattice, a = p->tile_a, model = p->model, storage = p->storage, arith = p->arith;
    if (storage == LBM_STORE_F64) {
        if (p->persistent) return nullptr;
        const bool ff = arith == LBM_ARITH_FF || arith == LBM_ARITH_AUTO || arith == LBM_ARITH_FF_TABLE;
        const int bn = step_block_nodes(p);
        if (bn != work_threads_for(lattice, a))  // 128-node work blocks: float-float only
            return ff ? select_step_ff(lattice, a, model, bn, ff_force_axis(lattice, p->force)) : nullptr;
        StepLaunch f = nullptr;
        if (arith == LBM_ARITH_F64) return select_step_f64(lattice, a, model, storage);
        if (arith == LBM_ARITH_FIXED) f = select_step_fixed(lattice, a, model);
        if (ff) f = select_step_ff(lattice, a, model, 0, ff_force_axis(lattice, p->force));
        return f ? f : select_step_f64(lattice, a, model, storage);
    }
    return select_step_f32(lattice, a, model, storage, p->block_nodes, p->persistent);
}
}  // namespace lbm

using namespace lbm;

struct lbm_ctx {
    lbm_params p{};
    lbm_tiling info{};
    int q = 0, nt = 0;
    void* pdf[2] = {nullptr, nullptr};
    size_t pdf_bytes = 0;
    int cur = 0;  // copy holding the current post-collision state
    int64_t step = 0;
    int32_t* d_nbr = nullptr;
    int32_t* d_tile_map = nullptr;  // dense tile map (single geometry, neighbour records built on the device)
    int32_t* d_gtab = nullptr;  // gather table of the FP64 float-float step
    uint64_t* d_tmask = nullptr;
    int32_t* d_coords = nullptr;
    uint32_t* d_nodes = nullptr;
    WorkBlock* d_blocks = nullptr;
    long long* d_tile_off = nullptr;
    int32_t* d_tile_stride = nullptr;
    ulonglong2* d_tinfo = nullptr;  // packed per-tile record of the step kernels' staging
    NRec* d_ntab = nullptr;         // per-tile neighbour records of the float-float step (one-word tiles)
    double* d_partials = nullptr;
    double* d_result = nullptr;
    float2* d_u_saved = nullptr;
    double* d_stage = nullptr;  // dense staging for host outputs
    size_t stage_bytes = 0;
    int nblocks = 0;            // blocks of the node kernels (= partial sums)
    bool u_saved_valid = false;
    bool prev_valid = false;  // the other copy holds the state one step before the current one
    bool tgb = false;         // LBM_LAYOUT_TGB: pdf[0] is the only copy, pdf[1] the two ghost sets
    int gset = 0;             // TGB: ghost set written by the last step (read by the next)
    size_t ghost_set = 0;     // TGB: bytes of one ghost set
    StepLaunch publish_fn = nullptr;
    std::vector<SampleRange> samples;     // one entry per geometry of a batch
    std::vector<int> part_begin, part_blocks;  // their slices of the partial sums
    StepArgs sa{};
    NodeArgs na{};
    StepLaunch step_fn = nullptr;
    NodeLaunch moments_fn = nullptr, export_fn = nullptr, import_fn = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_pairs = 8;  // each graph replays 2 * graph_pairs steps
    bool use_graph = true;
    int device = 0;       // the CUDA device current at lbm_init (the tables live there)
    // single geometry: per layer of tiles along the slowest tile axis (z in 3D,
    // y in 2D), the index of its first non-empty tile and the value offset of
    // that tile's PDF block (entry n_layers: the totals)
    std::vector<int> layer_first;
    std::vector<long long> layer_off;
};

static cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

// The state that alternates every step: the current copy (T2C) or the ghost
// set (TGB, whose copy never moves).
static int& parity(lbm_ctx* c) { return c->tgb ? c->gset : c->cur; }

static unsigned char* ghost(lbm_ctx* c, int set) { return static_cast<unsigned char*>(c->pdf[1]) + set * c->ghost_set; }

static int launch_one(lbm_ctx* c, cudaStream_t s) {
    StepArgs a = c->sa;
    if (c->tgb) {
        a.src = a.dst = c->pdf[0];
        a.ghost_in = ghost(c, c->gset);
        a.ghost_out = ghost(c, 1 - c->gset);
    } else {
        a.src = c->pdf[c->cur];
        a.dst = c->pdf[1 - c->cur];
    }
    cudaError_t e = c->step_fn(a, s);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    parity(c) = 1 - parity(c);
    return LBM_OK;
}

// TGB: fill the current ghost set from the copy (after init or import).
static int publish_ghosts(lbm_ctx* c, cudaStream_t s) {
    if (!c->tgb) return LBM_OK;
    StepArgs a = c->sa;
    a.src = a.dst = c->pdf[0];
    a.ghost_out = ghost(c, c->gset);
    LBM_CUDA_TRY(c->publish_fn(a, s));
    return LBM_OK;
}

static int build_graph(lbm_ctx* c, int start) {
    LBM_CUDA_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    const int saved = parity(c);
    parity(c) = start;
    int rc = LBM_OK;
    for (int k = 0; k < 2 * c->graph_pairs && rc == LBM_OK; k++) rc = launch_one(c, c->cap);
    parity(c) = saved;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph[start], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return LBM_OK;
}

static void release(lbm_ctx* c) {
    if (!c) return;
    for (int k = 0; k < 2; k++)
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
    if (c->cap) cudaStreamDestroy(c->cap);
    cudaFree(c->d_nbr);
    cudaFree(c->d_gtab);
    cudaFree(c->d_tmask);
    cudaFree(c->d_coords);
    cudaFree(c->d_nodes);
    cudaFree(c->d_blocks);
    cudaFree(c->d_tile_off);
    cudaFree(c->d_tile_stride);
    cudaFree(c->d_tinfo);
    cudaFree(c->d_tile_map);
    cudaFree(c->d_ntab);
    cudaFree(c->d_partials);
    cudaFree(c->d_result);
    cudaFree(c->d_u_saved);
    cudaFree(c->d_stage);
    delete c;
}

template <class T, class Alloc>
static int upload(T** dst, const std::vector<T, Alloc>& v, cudaStream_t s) {
    const size_t bytes = (v.empty() ? 1 : v.size()) * sizeof(T);
    LBM_CUDA_TRY(cudaMalloc(dst, bytes));
    if (!v.empty()) LBM_CUDA_TRY(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return LBM_OK;
}

static int ensure_stage(lbm_ctx* c, size_t bytes) {
    if (c->stage_bytes >= bytes) return LBM_OK;
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_bytes = 0;
    LBM_CUDA_TRY(cudaMalloc(&c->d_stage, bytes));
    c->stage_bytes = bytes;
    return LBM_OK;
}

static int init_ctx(lbm_ctx** out, const lbm_params* p, HostTiling& T, const std::vector<SampleRange>& samples,
                    void* pdf_a, void* pdf_b, size_t pdf_bytes, const double* rho_init, const double* u_init,
                    void* stream) {
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return fail(LBM_ERR_ARG, "tau must be > 1/2");
    if (!pdf_a || !pdf_b || pdf_a == pdf_b) return fail(LBM_ERR_ARG, "two distinct PDF buffers are required");
    if ((reinterpret_cast<uintptr_t>(pdf_a) | reinterpret_cast<uintptr_t>(pdf_b)) & 255)
        return fail(LBM_ERR_ARG, "PDF buffers must be 256-byte aligned");
    if (pdf_bytes < T.info.pdf_bytes)
        return fail(LBM_ERR_ARG, "PDF buffers hold %zu bytes, %zu needed", pdf_bytes, T.info.pdf_bytes);
    if (p->layout != LBM_LAYOUT_T2C && p->layout != LBM_LAYOUT_TGB)
        return fail(LBM_ERR_ARG, "unknown layout %d", p->layout);

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(LBM_ERR_OOM, "host allocation failed");
    c->p = *p;
    if (c->p.storage == LBM_STORE_F16S && !(c->p.f16_scale > 0.0)) c->p.f16_scale = 65536.0;
    c->info = T.info;
    c->samples = samples;
    c->q = lattice_q(p->lattice);
    c->nt = T.a * T.a * (T.d == 3 ? T.a : 1);
    c->pdf[0] = pdf_a;
    c->pdf[1] = pdf_b;
    c->pdf_bytes = pdf_bytes;
    const char* env = std::getenv("LBM_NO_GRAPH");
    c->use_graph = !(env && env[0] == '1');
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        release(c);
        return fail(LBM_ERR_CUDA, "cudaGetDevice failed");
    }

    c->tgb = p->layout == LBM_LAYOUT_TGB;
    c->ghost_set = T.info.ghost_bytes / 2;
    c->step_fn = c->tgb ? select_step_tgb(p) : select_step(p);
    if (c->tgb) c->publish_fn = select_tgb_publish(p->lattice, p->tile_a, p->storage);
    NodeLaunch init_fn = select_init(p->lattice, p->tile_a, p->model, p->storage);
    c->moments_fn = select_moments(p->lattice, p->tile_a, p->model, p->storage);
    c->export_fn = select_export(p->lattice, p->tile_a, p->storage);
    c->import_fn = select_import(p->lattice, p->tile_a, p->storage);
    if (!c->step_fn || !init_fn || !c->moments_fn || !c->export_fn || !c->import_fn || (c->tgb && !c->publish_fn)) {
        release(c);
        return fail(LBM_ERR_ARG, "no kernel for lattice %d, tile %d, model %d, storage %d, block %d, persistent %d",
                    p->lattice, p->tile_a, p->model, p->storage, p->block_nodes, p->persistent);
    }

    cudaStream_t s = S(stream);
    const int nf = T.info.n_ftiles;
    // partial sums: one launch over all tiles (lbm_stats_noalloc) or one per sample
    c->nblocks = node_blocks(p->lattice, p->tile_a, nf);
    int acc = 0;
    for (const SampleRange& r : samples) {
        c->part_begin.push_back(acc);
        c->part_blocks.push_back(node_blocks(p->lattice, p->tile_a, r.n_tiles));
        acc += c->part_blocks.back();
    }
    const int n_partials = std::max(std::max(c->nblocks, acc), 1);
#define TRY(x)                \
    do {                      \
        int r_ = (x);         \
        if (r_) {             \
            release(c);       \
            return r_;        \
        }                     \
    } while (0)
#define CTRY(x)                                                   \
    do {                                                          \
        cudaError_t ce_ = (x);                                    \
        if (ce_ != cudaSuccess) TRY(cuda_fail(ce_, #x));          \
    } while (0)
    TRY(upload(&c->d_tmask, T.tmask, s));
    TRY(upload(&c->d_coords, T.coords, s));
    const bool device_nbr = T.nbr.empty() && nf > 0;  // tiled without host neighbour records
    if (device_nbr) {
        // from the dense tile map (4 B per tile instead of 4 * 3^d B per non-empty tile)
        TRY(upload(&c->d_tile_map, T.tile_map, s));
        CTRY(cudaMalloc(&c->d_nbr, (size_t)nf * T.nn * sizeof(int32_t)));
        const int per[3] = {p->periodic[0] ? 1 : 0, p->periodic[1] ? 1 : 0,
                            T.d == 3 && p->periodic[2] ? 1 : 0};
        CTRY(launch_build_nbr(c->d_coords, c->d_tile_map, nf, T.d, T.info.ntx, T.info.nty, T.info.ntz, per,
                              c->d_nbr, s));
    } else {
        TRY(upload(&c->d_nbr, T.nbr, s));
    }
    // work blocks on the host; the fluid-node list they index is written on
    // the device from the tile masks (20 MB for 5 M fluid nodes not copied)
    const long long n_nodes =
        build_work_list(&T, step_block_nodes(p), 16, false, !c->tgb);
    CTRY(cudaMalloc(&c->d_nodes, (size_t)std::max<long long>(n_nodes, 1) * sizeof(uint32_t)));
    TRY(upload(&c->d_blocks, T.blocks, s));
    TRY(upload(&c->d_tile_off, T.tile_off, s));
    if (device_nbr && (long long)c->q * T.info.n_fluid > (1ll << 30)) {
        // the step kernels address neighbours with 32-bit value offsets
        unsigned* d_far = nullptr;
        unsigned far = 0;
        CTRY(cudaMalloc(&d_far, sizeof(unsigned)));
        cudaError_t fe = cudaMemsetAsync(d_far, 0, sizeof(unsigned), s);
        if (fe == cudaSuccess) fe = launch_far_check(c->d_nbr, c->d_tile_off, nf, T.nn, d_far, s);
        if (fe == cudaSuccess) fe = cudaMemcpyAsync(&far, d_far, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (fe == cudaSuccess) fe = cudaStreamSynchronize(s);
        cudaFree(d_far);
        CTRY(fe);
        if (far) TRY(fail(LBM_ERR_CAPACITY, "neighbour tiles lie more than 2^30 values apart (tile plane too large)"));
    }
    {
        NodeListLaunch nl = select_node_list(p->lattice, p->tile_a);
        if (!nl) TRY(fail(LBM_ERR_ARG, "no node-list kernel for lattice %d, tile %d", p->lattice, p->tile_a));
        CTRY(nl(c->d_tmask, c->d_tile_off, nf, c->d_nodes, s));
    }
    if (samples.size() == 1) {
        // tiles are numbered with the slowest axis slowest: each layer is a
        // contiguous run of tile indices and of PDF values
        const int n_layers = T.d == 3 ? T.info.ntz : T.info.nty;
        const int ax = T.d == 3 ? 2 : 1;
        const long long total = nf > 0 ? T.tile_off[nf - 1] + (long long)c->q * T.tile_stride[nf - 1] : 0;
        c->layer_first.resize((size_t)n_layers + 1);
        c->layer_off.resize((size_t)n_layers + 1);
        int k = 0;
        for (int l = 0; l <= n_layers; l++) {
            while (k < nf && T.coords[(size_t)3 * k + ax] < l) k++;
            c->layer_first[l] = k;
            c->layer_off[l] = k < nf ? T.tile_off[k] : total;
        }
    }
    TRY(upload(&c->d_tile_stride, T.tile_stride, s));
    {
        // one 16-byte load per neighbour slot when the step kernels stage a neighbourhood
        std::vector<ulonglong2> rec((size_t)nf);
        for (int k = 0; k < nf; k++) {
            const long long off = T.tile_off[k];
            const int32_t st = T.tile_stride[k];
            if (off < 0 || off >= (1ll << 40) || st < 0 || st >= (1 << 24))
                TRY(fail(LBM_ERR_CAPACITY, "tile offset or stride beyond the packed tile record"));
            rec[k].x = T.tmask[(size_t)k * T.words];
            rec[k].y = ((unsigned long long)off << 24) | (unsigned long long)st;
        }
        TRY(upload(&c->d_tinfo, rec, s));
    }
    CTRY(cudaMalloc(&c->d_partials, (size_t)n_partials * 8 * sizeof(double)));
    CTRY(cudaMalloc(&c->d_result, 8 * sizeof(double) * samples.size()));
    CTRY(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));

    StepArgs& sa = c->sa;
    sa.blocks = c->d_blocks;
    sa.nodes = c->d_nodes;
    sa.n_work_blocks = (int)T.blocks.size();
    sa.nbr = c->d_nbr;
    sa.tmask = c->d_tmask;
    sa.tile_off = c->d_tile_off;
    sa.tile_stride = c->d_tile_stride;
    sa.tinfo = c->d_tinfo;
    sa.n_tiles = nf;
    sa.n_nodes = n_nodes;
    sa.tau = p->tau;
    sa.omega = 1.0 / p->tau;
    for (int k = 0; k < 3; k++) sa.force[k] = (k < 2 || p->lattice == LBM_D3Q19) ? p->force[k] : 0.0;
    sa.f16_scale = c->p.f16_scale;
    sa.f16_inv_scale = c->p.f16_scale > 0 ? 1.0 / c->p.f16_scale : 0.0;
    sa.omega_f = (float)sa.omega;
    for (int k = 0; k < 3; k++) sa.force_f[k] = (float)sa.force[k];
    f32_consts(&c->p, sa.omega, sa.force, &sa.f32c);
    sa.f16_scale_f = (float)sa.f16_scale;
    sa.f16_inv_scale_f = (float)sa.f16_inv_scale;
    fixed_consts(&c->p, &sa.fx);
    ff_consts(&c->p, &sa.ffc);
    // LBM_ARITH_FF_TABLE: the FP64 float-float step reads its sources from a
    // gather table built once here (4 (q + 1) bytes per fluid node, the
    // connectivity-matrix scheme of Sec. 2.3.1), when value indices fit int32;
    // LBM_ARITH_FF / LBM_ARITH_AUTO run the staged tile-map step (no table)
    if (!c->tgb && p->storage == LBM_STORE_F64 && p->arith == LBM_ARITH_FF_TABLE &&
        !p->persistent && (!p->block_nodes || p->block_nodes == work_threads_for(p->lattice, p->tile_a)) &&
        T.info.pdf_bytes / 8 < (size_t)INT32_MAX && sa.n_nodes > 0) {
        StepLaunch table_step = select_step_ff_table(p->lattice, p->tile_a, p->model);
        StepLaunch build = select_gather_table_builder(p->lattice, p->tile_a);
        const size_t bytes = (size_t)(c->q + 1) * (size_t)sa.n_nodes * sizeof(int32_t);
        cudaError_t ae = table_step && build ? cudaMalloc(&c->d_gtab, bytes) : cudaErrorInvalidValue;
        if (ae == cudaSuccess) {
            sa.gtab = c->d_gtab;
            sa.gtab_out = c->d_gtab;
            sa.gtab_pitch = sa.n_nodes;
            CTRY(build(sa, s));
            c->step_fn = table_step;
        } else if (ae == cudaErrorMemoryAllocation) {
            (void)cudaGetLastError();  // no room for the table: the staged step needs none
        }
    }
    // the staged float-float step on tiles of one mask word reads each
    // neighbourhood from a per-tile table of neighbour records (16 B per slot)
    if (!c->tgb && !sa.gtab && T.words == 1 && p->storage == LBM_STORE_F64 &&
        (p->arith == LBM_ARITH_FF || p->arith == LBM_ARITH_AUTO || p->arith == LBM_ARITH_FF_TABLE) && nf > 0) {
        const int nn = T.nn;
        CTRY(cudaMalloc(&c->d_ntab, (size_t)nf * nn * sizeof(NRec)));
        CTRY(launch_build_ntab(c->d_nbr, c->d_tmask, c->d_tile_off, c->d_tile_stride, nf, nn, c->d_ntab, s));
        sa.ntab = c->d_ntab;
    }
    sa.pf_node_bytes = (int)(bytes_per_value(p->storage) * (size_t)lattice_q(p->lattice));
    sa.pf_limit = (long long)(T.info.pdf_bytes & ~(size_t)15);
    {
        // L2 prefetch distance: about 0.6 of the FP64 step's resident blocks
        // (seven per SM), 0.7 of the FP32 forms' (six per SM); further ahead
        // the prefetched lines start to evict the ones still being read
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) sms = 0;
        sa.pf_ahead = p->prefetch_blocks < 0 ? 0 : (p->prefetch_blocks > 0 ? p->prefetch_blocks : 4 * sms);
        if (sa.pf_ahead > sa.n_work_blocks) sa.pf_ahead = sa.n_work_blocks;
        // the FP32 forms stage through neighbour indices (two dependent loads):
        // their tables gain from the prefetch, the FP64 records did not
        sa.pf_tables = p->storage != LBM_STORE_F64;
    }

    NodeArgs& na = c->na;  // a launch over every tile; sample launches narrow it
    na.nbr = c->d_nbr;
    na.tmask = c->d_tmask;
    na.coords = c->d_coords;
    na.tile_off = c->d_tile_off;
    na.tile_stride = c->d_tile_stride;
    na.tinfo = c->d_tinfo;
    na.n_slots = (long long)(T.info.pdf_bytes / (bytes_per_value(p->storage) * (size_t)lattice_q(p->lattice)));
    na.tile_begin = 0;
    na.n_tiles = nf;
    na.nx = samples[0].nx;
    na.ny = samples[0].ny;
    na.nz = samples[0].nz;
    for (int k = 0; k < 3; k++) na.force[k] = sa.force[k];
    na.rho0 = p->rho0;
    na.f16_scale = sa.f16_scale;
    na.f16_inv_scale = sa.f16_inv_scale;
    na.partials = c->d_partials;

    // equilibrium start in copy 0; copy 1 is zeroed
    const SampleRange& r0 = samples[0];
    const size_t N0 = (size_t)r0.nx * r0.ny * r0.nz;
    // the initial fields: device memory is read in place, host memory staged
    const double* d_rho = nullptr;
    const double* d_u = nullptr;
    bool staged = false;
    auto on_device = [&](const void* ptr) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == c->device;
    };
    if (rho_init) {
        if (on_device(rho_init)) {
            d_rho = rho_init;
        } else {
            TRY(ensure_stage(c, N0 * 4 * sizeof(double)));
            CTRY(cudaMemcpyAsync(c->d_stage, rho_init, N0 * sizeof(double), cudaMemcpyDefault, s));
            d_rho = c->d_stage;
            staged = true;
        }
    }
    if (u_init) {
        const size_t nu = (size_t)(p->lattice == LBM_D3Q19 ? 3 : 2) * N0;
        if (on_device(u_init)) {
            d_u = u_init;
        } else {
            TRY(ensure_stage(c, N0 * 4 * sizeof(double)));
            CTRY(cudaMemcpyAsync(c->d_stage + N0, u_init, nu * sizeof(double), cudaMemcpyDefault, s));
            d_u = c->d_stage + N0;
            staged = true;
        }
    }
    for (size_t k = 0; k < samples.size(); k++) {
        NodeArgs ia = na;
        ia.pdf = pdf_a;
        ia.tile_begin = samples[k].tile_begin;
        ia.n_tiles = samples[k].n_tiles;
        ia.nx = samples[k].nx;
        ia.ny = samples[k].ny;
        ia.nz = samples[k].nz;
        ia.rho_in = k == 0 ? d_rho : nullptr;
        ia.u_in = k == 0 ? d_u : nullptr;
        CTRY(init_fn(ia, s));
    }
    CTRY(cudaMemsetAsync(pdf_b, 0, c->tgb ? T.info.ghost_bytes : T.info.pdf_bytes, s));
    if (staged) CTRY(cudaStreamSynchronize(s));  // the host fields may be released on return
#undef CTRY
#undef TRY
    c->cur = 0;
    c->gset = 0;
    if (c->tgb) {
        int rc_ = publish_ghosts(c, s);
        if (rc_) {
            release(c);
            return rc_;
        }
    }
    *out = c;
    return LBM_OK;
}

extern "C" int lbm_init(lbm_ctx** out, const lbm_params* p, const uint8_t* mask, void* pdf_a, void* pdf_b,
                        size_t pdf_bytes, const double* rho_init, const double* u_init, void* stream) {
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    HostTiling T;
    int rc = build_tiling(p, mask, &T, false);  // neighbour records built on the device
    if (rc) return rc;
    std::vector<SampleRange> samples{SampleRange{p->nx, p->ny, p->nz, 0, T.info.n_ftiles, T.info.n_fluid}};
    return init_ctx(out, p, T, samples, pdf_a, pdf_b, pdf_bytes, rho_init, u_init, stream);
}

extern "C" int lbm_init_batch(lbm_ctx** out, const lbm_params* p, int n_samples, const int* dims,
                              const uint8_t* const* masks, void* pdf_a, void* pdf_b, size_t pdf_bytes,
                              void* stream) {
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    HostTiling T;
    std::vector<SampleRange> samples;
    int rc = build_batch_tiling(p, n_samples, dims, masks, &T, &samples);
    if (rc) return rc;
    return init_ctx(out, p, T, samples, pdf_a, pdf_b, pdf_bytes, nullptr, nullptr, stream);
}

extern "C" int lbm_step(lbm_ctx* c, int nsteps, void* stream) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps < 0");
    cudaStream_t s = S(stream);
    int left = nsteps;
    const int per_graph = 2 * c->graph_pairs;
    if (c->use_graph && left >= per_graph && c->info.n_ftiles > 0) {
        const int par = parity(c);
        if (!c->graph[par]) {
            int rc = build_graph(c, par);
            if (rc) return rc;
        }
        while (left >= per_graph) {
            LBM_CUDA_TRY(cudaGraphLaunch(c->graph[par], s));
            left -= per_graph;  // an even number of steps: the current copy is unchanged
        }
    }
    for (; left > 0; left--) {
        int rc = launch_one(c, s);
        if (rc) return rc;
    }
    c->step += nsteps;
    if (nsteps > 0) c->prev_valid = true;
    return LBM_OK;
}

extern "C" int lbm_filter_period2(lbm_ctx* c, void* stream) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
    if (c->tgb) return fail(LBM_ERR_ARG, "the period-2 filter needs the two-copy layout (LBM_LAYOUT_T2C)");
    if (!c->prev_valid)
        return fail(LBM_ERR_ARG, "no previous state: step at least once after init, import or a filter");
    LBM_CUDA_TRY(launch_average(c->pdf[c->cur], c->pdf[1 - c->cur], c->info.pdf_bytes, c->p.storage, S(stream)));
    c->prev_valid = false;
    return LBM_OK;
}

static NodeArgs sample_args(const lbm_ctx* c, size_t k) {
    NodeArgs a = c->na;
    const SampleRange& r = c->samples[k];
    a.pdf = c->pdf[c->cur];
    a.tile_begin = r.tile_begin;
    a.n_tiles = r.n_tiles;
    a.nx = r.nx;
    a.ny = r.ny;
    a.nz = r.nz;
    return a;
}

// Moments of every sample (fields only for a single sample), each reduced in
// a fixed order into d_result[8k .. 8k+7].
static int launch_sample_moments(lbm_ctx* c, double* d_rho, double* d_u, bool residual, cudaStream_t s) {
    if (residual && !c->d_u_saved)
        LBM_CUDA_TRY(cudaMalloc(&c->d_u_saved, (size_t)c->na.n_slots * 3 * sizeof(float2) + 8));
    for (size_t k = 0; k < c->samples.size(); k++) {
        NodeArgs a = sample_args(c, k);
        a.rho_out = d_rho;
        a.u_out = d_u;
        a.residual = residual ? 1 : 0;
        a.u_saved = residual ? c->d_u_saved : nullptr;
        a.partials = c->d_partials + (size_t)8 * c->part_begin[k];
        LBM_CUDA_TRY(c->moments_fn(a, s));
        LBM_CUDA_TRY(launch_reduce(a.partials, c->part_blocks[k], c->d_result + 8 * k, s));
    }
    return LBM_OK;
}

static void fill_stats(const lbm_ctx* c, const double* r, bool residual, bool had_saved, lbm_stats* st) {
    st->mass = r[0];
    st->momentum[0] = r[1];
    st->momentum[1] = r[2];
    st->momentum[2] = r[3];
    st->u2 = r[4];
    st->du2 = residual ? r[5] : 0.0;
    st->residual = residual && had_saved && r[4] > 0 ? std::sqrt(r[5] / r[4]) : INFINITY;
    st->n_fluid = (int64_t)r[6];
    st->step = c->step;
}

static bool finite_stats(const lbm_stats& st) {
    return std::isfinite(st.mass) && std::isfinite(st.momentum[0]) && std::isfinite(st.momentum[1]) &&
           std::isfinite(st.momentum[2]);
}

extern "C" int lbm_moments(lbm_ctx* c, double* rho, double* u, lbm_stats* stats, int flags, void* stream) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
    if ((rho || u) && c->samples.size() != 1)
        return fail(LBM_ERR_ARG, "rho/u fields need a single-geometry context");
    cudaStream_t s = S(stream);
    const size_t N = (size_t)c->p.nx * c->p.ny * c->p.nz;
    const int d = c->p.lattice == LBM_D3Q19 ? 3 : 2;
    const bool dev = flags & LBM_OUT_DEVICE;
    const bool residual = (flags & LBM_STATS_RESIDUAL) && stats;
    double* d_rho = nullptr;
    double* d_u = nullptr;
    if (rho || u) {
        if (dev) {
            d_rho = rho;
            d_u = u;
        } else {
            int rc = ensure_stage(c, N * (1 + d) * sizeof(double));
            if (rc) return rc;
            d_rho = rho ? c->d_stage : nullptr;
            d_u = u ? c->d_stage + N : nullptr;
        }
        if (d_rho) LBM_CUDA_TRY(launch_fill_nan(d_rho, N, s));
        if (d_u) LBM_CUDA_TRY(launch_fill_nan(d_u, d * N, s));
    }
    int rc = launch_sample_moments(c, d_rho, d_u, residual, s);
    if (rc) return rc;
    if (!dev && rho) LBM_CUDA_TRY(cudaMemcpyAsync(rho, d_rho, N * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!dev && u) LBM_CUDA_TRY(cudaMemcpyAsync(u, d_u, d * N * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (stats) {
        std::vector<double> r(8 * c->samples.size());
        LBM_CUDA_TRY(cudaMemcpyAsync(r.data(), c->d_result, r.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        LBM_CUDA_TRY(cudaStreamSynchronize(s));
        double sum[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (size_t k = 0; k < c->samples.size(); k++)
            for (int j = 0; j < 8; j++) sum[j] += r[8 * k + j];  // samples in order
        fill_stats(c, sum, residual, c->u_saved_valid, stats);
        if (residual) c->u_saved_valid = true;
        if (!finite_stats(*stats))
            return fail(LBM_ERR_DIVERGED, "mass or momentum is not finite at step %lld", (long long)c->step);
    } else if (!dev && (rho || u)) {
        LBM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return LBM_OK;
}

extern "C" int lbm_moments_sample(lbm_ctx* c, int sample, double* rho, double* u, int flags, void* stream) {
    if (!c || (!rho && !u)) return fail(LBM_ERR_ARG, "NULL argument");
    if (sample < 0 || sample >= (int)c->samples.size()) return fail(LBM_ERR_ARG, "no sample %d", sample);
    cudaStream_t s = S(stream);
    const SampleRange& r = c->samples[sample];
    const size_t N = (size_t)r.nx * r.ny * r.nz;
    const int d = c->p.lattice == LBM_D3Q19 ? 3 : 2;
    const bool dev = flags & LBM_OUT_DEVICE;
    double* d_rho = rho;
    double* d_u = u;
    if (!dev) {
        int rc = ensure_stage(c, N * (1 + d) * sizeof(double));
        if (rc) return rc;
        d_rho = rho ? c->d_stage : nullptr;
        d_u = u ? c->d_stage + N : nullptr;
    }
    if (d_rho) LBM_CUDA_TRY(launch_fill_nan(d_rho, N, s));
    if (d_u) LBM_CUDA_TRY(launch_fill_nan(d_u, d * N, s));
    NodeArgs a = sample_args(c, sample);
    a.rho_out = d_rho;
    a.u_out = d_u;
    a.partials = c->d_partials + (size_t)8 * c->part_begin[sample];
    LBM_CUDA_TRY(c->moments_fn(a, s));
    if (!dev) {
        if (rho) LBM_CUDA_TRY(cudaMemcpyAsync(rho, d_rho, N * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (u) LBM_CUDA_TRY(cudaMemcpyAsync(u, d_u, d * N * sizeof(double), cudaMemcpyDeviceToHost, s));
        LBM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return LBM_OK;
}

extern "C" int lbm_moments_batch(lbm_ctx* c, lbm_stats* stats, int flags, void* stream) {
    if (!c || !stats) return fail(LBM_ERR_ARG, "NULL argument");
    cudaStream_t s = S(stream);
    const bool residual = flags & LBM_STATS_RESIDUAL;
    int rc = launch_sample_moments(c, nullptr, nullptr, residual, s);
    if (rc) return rc;
    std::vector<double> r(8 * c->samples.size());
    LBM_CUDA_TRY(cudaMemcpyAsync(r.data(), c->d_result, r.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    LBM_CUDA_TRY(cudaStreamSynchronize(s));
    bool finite = true;
    for (size_t k = 0; k < c->samples.size(); k++) {
        fill_stats(c, &r[8 * k], residual, c->u_saved_valid, &stats[k]);
        finite &= finite_stats(stats[k]);
    }
    if (residual) c->u_saved_valid = true;
    if (!finite) return fail(LBM_ERR_DIVERGED, "a sample's mass or momentum is not finite at step %lld",
                             (long long)c->step);
    return LBM_OK;
}

extern "C" int lbm_export_pdfs_sample(lbm_ctx* c, int sample, double* pdfs, int flags, void* stream) {
    if (!c || !pdfs) return fail(LBM_ERR_ARG, "NULL argument");
    if (sample < 0 || sample >= (int)c->samples.size()) return fail(LBM_ERR_ARG, "no sample %d", sample);
    cudaStream_t s = S(stream);
    const SampleRange& r = c->samples[sample];
    const size_t n = (size_t)c->q * r.nx * r.ny * r.nz;
    const bool dev = flags & LBM_OUT_DEVICE;
    double* d = pdfs;
    if (!dev) {
        int rc = ensure_stage(c, n * sizeof(double));
        if (rc) return rc;
        d = c->d_stage;
    }
    LBM_CUDA_TRY(launch_fill_nan(d, n, s));
    NodeArgs a = sample_args(c, sample);
    a.dense_pdf = d;
    LBM_CUDA_TRY(c->export_fn(a, s));
    if (!dev) {
        LBM_CUDA_TRY(cudaMemcpyAsync(pdfs, d, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        LBM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return LBM_OK;
}

extern "C" int lbm_export_pdfs(lbm_ctx* c, double* pdfs, int flags, void* stream) {
    if (c && c->samples.size() != 1) return fail(LBM_ERR_ARG, "a batch exports per sample (lbm_export_pdfs_sample)");
    return lbm_export_pdfs_sample(c, 0, pdfs, flags, stream);
}

extern "C" int lbm_import_pdfs(lbm_ctx* c, const double* pdfs, int64_t step, int flags, void* stream) {
    if (!c || !pdfs) return fail(LBM_ERR_ARG, "NULL argument");
    if (c->samples.size() != 1) return fail(LBM_ERR_ARG, "import needs a single-geometry context");
    cudaStream_t s = S(stream);
    const size_t n = (size_t)c->q * c->p.nx * c->p.ny * c->p.nz;
    const double* d = pdfs;
    if (!(flags & LBM_OUT_DEVICE)) {
        int rc = ensure_stage(c, n * sizeof(double));
        if (rc) return rc;
        LBM_CUDA_TRY(cudaMemcpyAsync(c->d_stage, pdfs, n * sizeof(double), cudaMemcpyHostToDevice, s));
        d = c->d_stage;
    }
    NodeArgs a = sample_args(c, 0);
    a.dense_pdf_in = d;
    LBM_CUDA_TRY(c->import_fn(a, s));
    if (!(flags & LBM_OUT_DEVICE)) LBM_CUDA_TRY(cudaStreamSynchronize(s));
    c->step = step;
    c->u_saved_valid = false;
    c->prev_valid = false;
    return publish_ghosts(c, s);
}

static int check_layers(const lbm_ctx* c, int l_begin, int l_end) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
    if (c->layer_first.empty()) return fail(LBM_ERR_ARG, "tile layers need a single-geometry context");
    if (c->tgb) return fail(LBM_ERR_ARG, "tile layers need the two-copy layout (LBM_LAYOUT_T2C)");
    const int n = (int)c->layer_first.size() - 1;
    if (l_begin < 0 || l_end < l_begin || l_end > n)
        return fail(LBM_ERR_ARG, "tile layers [%d, %d) outside [0, %d)", l_begin, l_end, n);
    return LBM_OK;
}

extern "C" int lbm_layer_range(const lbm_ctx* c, int l_begin, int l_end, size_t* offset, size_t* bytes) {
    int rc = check_layers(c, l_begin, l_end);
    if (rc) return rc;
    if (!offset || !bytes) return fail(LBM_ERR_ARG, "NULL argument");
    const size_t bpv = bytes_per_value(c->p.storage);
    *offset = (size_t)c->layer_off[l_begin] * bpv;
    *bytes = (size_t)(c->layer_off[l_end] - c->layer_off[l_begin]) * bpv;
    return LBM_OK;
}

extern "C" int lbm_current_copy(const lbm_ctx* c) { return c ? c->cur : -1; }

extern "C" int lbm_moments_layers(lbm_ctx* c, int l_begin, int l_end, lbm_stats* stats, int flags, void* stream) {
    int rc = check_layers(c, l_begin, l_end);
    if (rc) return rc;
    if (!stats) return fail(LBM_ERR_ARG, "stats is NULL");
    cudaStream_t s = S(stream);
    const bool residual = flags & LBM_STATS_RESIDUAL;
    if (residual && !c->d_u_saved)
        LBM_CUDA_TRY(cudaMalloc(&c->d_u_saved, (size_t)c->na.n_slots * 3 * sizeof(float2) + 8));
    NodeArgs a = sample_args(c, 0);
    a.tile_begin = c->layer_first[l_begin];
    a.n_tiles = c->layer_first[l_end] - c->layer_first[l_begin];
    a.rho_out = nullptr;
    a.u_out = nullptr;
    a.residual = residual ? 1 : 0;
    a.u_saved = residual ? c->d_u_saved : nullptr;
    a.partials = c->d_partials;
    double r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (a.n_tiles > 0) {
        const int nb = node_blocks(c->p.lattice, c->p.tile_a, a.n_tiles);
        LBM_CUDA_TRY(c->moments_fn(a, s));
        LBM_CUDA_TRY(launch_reduce(a.partials, nb, c->d_result, s));
        LBM_CUDA_TRY(cudaMemcpyAsync(r, c->d_result, sizeof(r), cudaMemcpyDeviceToHost, s));
        LBM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    fill_stats(c, r, residual, c->u_saved_valid, stats);
    if (residual) c->u_saved_valid = true;
    if (!finite_stats(*stats))
        return fail(LBM_ERR_DIVERGED, "mass or momentum is not finite at step %lld", (long long)c->step);
    return LBM_OK;
}

extern "C" int lbm_num_samples(const lbm_ctx* c) { return c ? (int)c->samples.size() : 0; }

extern "C" int lbm_get_tiling(const lbm_ctx* c, lbm_tiling* out) {
    if (!c || !out) return fail(LBM_ERR_ARG, "NULL argument");
    *out = c->info;
    return LBM_OK;
}

extern "C" int lbm_free(lbm_ctx* c) {
    if (!c) return LBM_OK;
    cudaError_t e = cudaDeviceSynchronize();
    release(c);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize in lbm_free");
    return LBM_OK;
}

namespace lbm {
// Reduction launch data of a context, for entry points defined in other files.
int ctx_reduction_args(const lbm_ctx* c, NodeArgs* args, NodeLaunch* moments, int* nblocks, int* device) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
    *device = c->device;
    *args = c->na;
    args->pdf = c->pdf[c->cur];
    args->rho_out = nullptr;
    args->u_out = nullptr;
    args->residual = 0;
    args->u_saved = nullptr;
    *moments = c->moments_fn;
    *nblocks = c->nblocks;
    return LBM_OK;
}
}  // namespace lbm

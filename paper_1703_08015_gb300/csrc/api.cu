// api.cu -- the C ABI of include/lbm.h: context life cycle, stepping (with a
// captured CUDA graph of several steps), moments and PDF export/import.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"

namespace lbm {
StepLaunch select_step_f64(int lattice, int a, int model, int storage);
StepLaunch select_step_fixed(int lattice, int a, int model);
StepLaunch select_step_f32(int lattice, int a, int model, int storage);

StepLaunch select_step(int lattice, int a, int model, int storage, int arith) {
    if (storage == LBM_STORE_F64) {
        if (arith == LBM_ARITH_F64) return select_step_f64(lattice, a, model, storage);
        StepLaunch f = select_step_fixed(lattice, a, model);
        return f ? f : select_step_f64(lattice, a, model, storage);
    }
    return select_step_f32(lattice, a, model, storage);
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
    uint64_t* d_tmask = nullptr;
    int32_t* d_coords = nullptr;
    uint32_t* d_nodes = nullptr;
    WorkBlock* d_blocks = nullptr;
    long long* d_tile_off = nullptr;
    int32_t* d_tile_stride = nullptr;
    double* d_partials = nullptr;
    double* d_result = nullptr;
    double* d_u_saved = nullptr;
    int* d_err = nullptr;
    double* d_stage = nullptr;  // dense staging for host outputs
    size_t stage_bytes = 0;
    int nblocks = 0;            // blocks of the node kernels (= partial sums)
    bool u_saved_valid = false;
    StepArgs sa{};
    NodeArgs na{};
    StepLaunch step_fn = nullptr;
    NodeLaunch moments_fn = nullptr, export_fn = nullptr, import_fn = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_pairs = 8;  // each graph replays 2 * graph_pairs steps
    bool use_graph = true;
};

static cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

static int launch_one(lbm_ctx* c, cudaStream_t s) {
    StepArgs a = c->sa;
    a.src = c->pdf[c->cur];
    a.dst = c->pdf[1 - c->cur];
    cudaError_t e = c->step_fn(a, s);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    c->cur = 1 - c->cur;
    return LBM_OK;
}

static int build_graph(lbm_ctx* c, int start) {
    LBM_CUDA_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    const int saved = c->cur;
    c->cur = start;
    int rc = LBM_OK;
    for (int k = 0; k < 2 * c->graph_pairs && rc == LBM_OK; k++) rc = launch_one(c, c->cap);
    c->cur = saved;
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
    cudaFree(c->d_tmask);
    cudaFree(c->d_coords);
    cudaFree(c->d_nodes);
    cudaFree(c->d_blocks);
    cudaFree(c->d_tile_off);
    cudaFree(c->d_tile_stride);
    cudaFree(c->d_partials);
    cudaFree(c->d_result);
    cudaFree(c->d_u_saved);
    cudaFree(c->d_err);
    cudaFree(c->d_stage);
    delete c;
}

template <class T>
static int upload(T** dst, const std::vector<T>& v, cudaStream_t s) {
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

extern "C" int lbm_init(lbm_ctx** out, const lbm_params* p, const uint8_t* mask, void* pdf_a, void* pdf_b,
                        size_t pdf_bytes, const double* rho_init, const double* u_init, void* stream) {
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = validate_params(p);
    if (rc) return rc;
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return fail(LBM_ERR_ARG, "tau must be > 1/2");
    if (!pdf_a || !pdf_b || pdf_a == pdf_b) return fail(LBM_ERR_ARG, "two distinct PDF buffers are required");
    if ((reinterpret_cast<uintptr_t>(pdf_a) | reinterpret_cast<uintptr_t>(pdf_b)) & 255)
        return fail(LBM_ERR_ARG, "PDF buffers must be 256-byte aligned");
    HostTiling T;
    rc = build_tiling(p, mask, &T);
    if (rc) return rc;
    if (pdf_bytes < T.info.pdf_bytes)
        return fail(LBM_ERR_ARG, "PDF buffers hold %zu bytes, %zu needed", pdf_bytes, T.info.pdf_bytes);

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(LBM_ERR_OOM, "host allocation failed");
    c->p = *p;
    if (c->p.storage == LBM_STORE_F16S && !(c->p.f16_scale > 0.0)) c->p.f16_scale = 65536.0;
    c->info = T.info;
    c->q = lattice_q(p->lattice);
    c->nt = T.a * T.a * (T.d == 3 ? T.a : 1);
    c->pdf[0] = pdf_a;
    c->pdf[1] = pdf_b;
    c->pdf_bytes = pdf_bytes;
    const char* env = std::getenv("LBM_NO_GRAPH");
    c->use_graph = !(env && env[0] == '1');

    c->step_fn = select_step(p->lattice, p->tile_a, p->model, p->storage, p->arith);
    NodeLaunch init_fn = select_init(p->lattice, p->tile_a, p->model, p->storage);
    c->moments_fn = select_moments(p->lattice, p->tile_a, p->model, p->storage);
    c->export_fn = select_export(p->lattice, p->tile_a, p->storage);
    c->import_fn = select_import(p->lattice, p->tile_a, p->storage);
    if (!c->step_fn || !init_fn || !c->moments_fn || !c->export_fn || !c->import_fn) {
        release(c);
        return fail(LBM_ERR_ARG, "no kernel for lattice %d, tile %d, model %d, storage %d", p->lattice,
                    p->tile_a, p->model, p->storage);
    }

    cudaStream_t s = S(stream);
    const int nf = T.info.n_ftiles;
    c->nblocks = node_blocks(p->lattice, p->tile_a, nf);
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
    TRY(upload(&c->d_nbr, T.nbr, s));
    TRY(upload(&c->d_tmask, T.tmask, s));
    TRY(upload(&c->d_coords, T.coords, s));
    build_work_list(&T, work_threads_for(p->lattice, p->tile_a), 16);
    TRY(upload(&c->d_nodes, T.nodes, s));
    TRY(upload(&c->d_blocks, T.blocks, s));
    TRY(upload(&c->d_tile_off, T.tile_off, s));
    TRY(upload(&c->d_tile_stride, T.tile_stride, s));
    CTRY(cudaMalloc(&c->d_partials, (size_t)(c->nblocks > 0 ? c->nblocks : 1) * 8 * sizeof(double)));
    CTRY(cudaMalloc(&c->d_result, 8 * sizeof(double)));
    CTRY(cudaMalloc(&c->d_err, sizeof(int)));
    CTRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
    CTRY(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));

    StepArgs& sa = c->sa;
    sa.blocks = c->d_blocks;
    sa.nodes = c->d_nodes;
    sa.n_work_blocks = (int)T.blocks.size();
    sa.nbr = c->d_nbr;
    sa.tmask = c->d_tmask;
    sa.tile_off = c->d_tile_off;
    sa.tile_stride = c->d_tile_stride;
    sa.n_tiles = nf;
    sa.tau = p->tau;
    sa.omega = 1.0 / p->tau;
    for (int k = 0; k < 3; k++) sa.force[k] = (k < 2 || p->lattice == LBM_D3Q19) ? p->force[k] : 0.0;
    sa.f16_scale = c->p.f16_scale;
    sa.f16_inv_scale = c->p.f16_scale > 0 ? 1.0 / c->p.f16_scale : 0.0;
    sa.omega_f = (float)sa.omega;
    for (int k = 0; k < 3; k++) sa.force_f[k] = (float)sa.force[k];
    sa.f16_scale_f = (float)sa.f16_scale;
    sa.f16_inv_scale_f = (float)sa.f16_inv_scale;
    sa.err = c->d_err;
    fixed_consts(&c->p, &sa.fx);

    NodeArgs& na = c->na;
    na.nbr = c->d_nbr;
    na.tmask = c->d_tmask;
    na.coords = c->d_coords;
    na.tile_off = c->d_tile_off;
    na.tile_stride = c->d_tile_stride;
    na.n_tiles = nf;
    na.nx = p->nx;
    na.ny = p->ny;
    na.nz = p->nz;
    for (int k = 0; k < 3; k++) na.force[k] = sa.force[k];
    na.rho0 = p->rho0;
    na.f16_scale = sa.f16_scale;
    na.f16_inv_scale = sa.f16_inv_scale;
    na.partials = c->d_partials;

    // equilibrium start in copy 0; copy 1 is zeroed (its solid slots are never read)
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    double* d_rho = nullptr;
    double* d_u = nullptr;
    if (rho_init || u_init) {
        TRY(ensure_stage(c, N * 4 * sizeof(double)));
        if (rho_init) {
            d_rho = c->d_stage;
            CTRY(cudaMemcpyAsync(d_rho, rho_init, N * sizeof(double), cudaMemcpyHostToDevice, s));
        }
        if (u_init) {
            d_u = c->d_stage + N;
            const size_t nu = (size_t)(p->lattice == LBM_D3Q19 ? 3 : 2) * N;
            CTRY(cudaMemcpyAsync(d_u, u_init, nu * sizeof(double), cudaMemcpyHostToDevice, s));
        }
    }
    NodeArgs ia = na;
    ia.pdf = pdf_a;
    ia.rho_in = d_rho;
    ia.u_in = d_u;
    CTRY(init_fn(ia, s));
    CTRY(cudaMemsetAsync(pdf_b, 0, T.info.pdf_bytes, s));
    if (rho_init || u_init) CTRY(cudaStreamSynchronize(s));
#undef CTRY
#undef TRY
    c->cur = 0;
    *out = c;
    return LBM_OK;
}

extern "C" int lbm_step(lbm_ctx* c, int nsteps, void* stream) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps < 0");
    cudaStream_t s = S(stream);
    int left = nsteps;
    const int per_graph = 2 * c->graph_pairs;
    if (c->use_graph && left >= per_graph && c->info.n_ftiles > 0) {
        if (!c->graph[c->cur]) {
            int rc = build_graph(c, c->cur);
            if (rc) return rc;
        }
        while (left >= per_graph) {
            LBM_CUDA_TRY(cudaGraphLaunch(c->graph[c->cur], s));
            left -= per_graph;  // an even number of steps: the current copy is unchanged
        }
    }
    for (; left > 0; left--) {
        int rc = launch_one(c, s);
        if (rc) return rc;
    }
    c->step += nsteps;
    return LBM_OK;
}

extern "C" int lbm_moments(lbm_ctx* c, double* rho, double* u, lbm_stats* stats, int flags, void* stream) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
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
    if (residual && !c->d_u_saved)
        LBM_CUDA_TRY(cudaMalloc(&c->d_u_saved, (size_t)c->info.n_ftiles * 3 * c->nt * sizeof(double) + 8));
    NodeArgs a = c->na;
    a.pdf = c->pdf[c->cur];
    a.rho_out = d_rho;
    a.u_out = d_u;
    a.residual = residual ? 1 : 0;
    a.u_saved = residual ? c->d_u_saved : nullptr;
    LBM_CUDA_TRY(c->moments_fn(a, s));
    if (stats) LBM_CUDA_TRY(launch_reduce(c->d_partials, c->nblocks, c->d_result, s));
    if (!dev && rho) LBM_CUDA_TRY(cudaMemcpyAsync(rho, d_rho, N * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!dev && u) LBM_CUDA_TRY(cudaMemcpyAsync(u, d_u, d * N * sizeof(double), cudaMemcpyDeviceToHost, s));
    int rc = LBM_OK;
    if (stats) {
        double r[8];
        LBM_CUDA_TRY(cudaMemcpyAsync(r, c->d_result, sizeof r, cudaMemcpyDeviceToHost, s));
        LBM_CUDA_TRY(cudaStreamSynchronize(s));
        stats->mass = r[0];
        stats->momentum[0] = r[1];
        stats->momentum[1] = r[2];
        stats->momentum[2] = r[3];
        stats->u2 = r[4];
        stats->du2 = residual ? r[5] : 0.0;
        stats->residual = residual && c->u_saved_valid && r[4] > 0 ? std::sqrt(r[5] / r[4]) : INFINITY;
        stats->n_fluid = (int64_t)r[6];
        stats->step = c->step;
        if (residual) c->u_saved_valid = true;
        if (!std::isfinite(r[0]) || !std::isfinite(r[1]) || !std::isfinite(r[2]) || !std::isfinite(r[3]))
            rc = fail(LBM_ERR_DIVERGED, "mass or momentum is not finite at step %lld", (long long)c->step);
    } else if (!dev && (rho || u)) {
        LBM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return rc;
}

extern "C" int lbm_export_pdfs(lbm_ctx* c, double* pdfs, int flags, void* stream) {
    if (!c || !pdfs) return fail(LBM_ERR_ARG, "NULL argument");
    cudaStream_t s = S(stream);
    const size_t n = (size_t)c->q * c->p.nx * c->p.ny * c->p.nz;
    const bool dev = flags & LBM_OUT_DEVICE;
    double* d = pdfs;
    if (!dev) {
        int rc = ensure_stage(c, n * sizeof(double));
        if (rc) return rc;
        d = c->d_stage;
    }
    LBM_CUDA_TRY(launch_fill_nan(d, n, s));
    NodeArgs a = c->na;
    a.pdf = c->pdf[c->cur];
    a.dense_pdf = d;
    LBM_CUDA_TRY(c->export_fn(a, s));
    if (!dev) {
        LBM_CUDA_TRY(cudaMemcpyAsync(pdfs, d, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        LBM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return LBM_OK;
}

extern "C" int lbm_import_pdfs(lbm_ctx* c, const double* pdfs, int64_t step, int flags, void* stream) {
    if (!c || !pdfs) return fail(LBM_ERR_ARG, "NULL argument");
    cudaStream_t s = S(stream);
    const size_t n = (size_t)c->q * c->p.nx * c->p.ny * c->p.nz;
    const double* d = pdfs;
    if (!(flags & LBM_OUT_DEVICE)) {
        int rc = ensure_stage(c, n * sizeof(double));
        if (rc) return rc;
        LBM_CUDA_TRY(cudaMemcpyAsync(c->d_stage, pdfs, n * sizeof(double), cudaMemcpyHostToDevice, s));
        d = c->d_stage;
    }
    NodeArgs a = c->na;
    a.pdf = c->pdf[c->cur];
    a.dense_pdf_in = d;
    LBM_CUDA_TRY(c->import_fn(a, s));
    if (!(flags & LBM_OUT_DEVICE)) LBM_CUDA_TRY(cudaStreamSynchronize(s));
    c->step = step;
    c->u_saved_valid = false;
    return LBM_OK;
}

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
int ctx_reduction_args(const lbm_ctx* c, NodeArgs* args, NodeLaunch* moments, int* nblocks) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
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

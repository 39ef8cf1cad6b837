// noalloc.cu -- lbm_stats_noalloc: the FP64 mass / momentum reduction of
// lbm_moments for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc when they need the statistics: code
// that runs under a fixed device-memory budget handed out by another
// allocator, monitoring hooks that must not change the process's memory
// footprint between steps, or loops that cannot afford cudaMalloc's implicit
// device-wide synchronisation.  This entry point needs no allocation: its
// per-block partial sums live in a file-scope device array of fixed size that
// every GPU loading the library holds until the process exits, and the caller
// passes the output buffer.
#include <mutex>

#include "internal.h"

namespace lbm {

int ctx_reduction_args(const lbm_ctx* c, NodeArgs* args, NodeLaunch* moments, int* nblocks, int* device);

// Per-block partial sums of the moments kernel: 8 doubles per block.
static __device__ __align__(256) double g_stats_scratch[LBM_NOALLOC_MAX_BLOCKS * 8];

static std::mutex g_scratch_mutex;
static void* g_scratch_addr[256] = {};  // device address of g_stats_scratch, per device

// Device address of the scratch array on device `dev`, the current device
// (looked up once per device; a cudaDeviceReset of that device invalidates
// the cached address, and calls after one are not supported).
static int scratch_address(int dev, double** out) {
    if (dev < 0 || dev >= 256) return fail(LBM_ERR_CAPACITY, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_stats_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_stats_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<double*>(g_scratch_addr[dev]);
    return LBM_OK;
}

}  // namespace lbm

extern "C" int lbm_stats_noalloc(const lbm_ctx* ctx, double* stats_dev, void* stream) {
    using namespace lbm;
    if (!ctx || !stats_dev) return fail(LBM_ERR_ARG, "NULL argument");
    NodeArgs a;
    NodeLaunch moments = nullptr;
    int nblocks = 0, ctx_dev = 0, dev = 0;
    int rc = ctx_reduction_args(ctx, &a, &moments, &nblocks, &ctx_dev);
    if (rc) return rc;
    LBM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != ctx_dev)
        return fail(LBM_ERR_ARG, "lbm_stats_noalloc: device %d is current, the context was created on device %d",
                    dev, ctx_dev);
    if (nblocks > LBM_NOALLOC_MAX_BLOCKS)
        return fail(LBM_ERR_CAPACITY,
                    "lbm_stats_noalloc: the tiling needs %d partial-sum slots, the static scratch holds %d",
                    nblocks, LBM_NOALLOC_MAX_BLOCKS);
    double* scratch = nullptr;
    rc = scratch_address(dev, &scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    a.partials = scratch;  // every block writes all 8 of its slots before k_reduce reads them
    LBM_CUDA_TRY(moments(a, s));
    LBM_CUDA_TRY(launch_reduce(scratch, nblocks, stats_dev, s));
    return LBM_OK;
}

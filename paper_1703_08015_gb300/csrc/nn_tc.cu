// nn_tc.cu -- GEMMs of the learned warm start on the 5th-generation tensor
// cores (tcgen05): operands staged in shared memory by the block's threads,
// the FP32 accumulator in tensor memory (TMEM), one thread issuing the MMAs
// and an mbarrier reporting their completion.  A plain BF16 GEMM, the 3x3x3
// convolution (as an implicit GEMM, and reading a shared-memory halo tile)
// and its weight gradient (one GEMM per tap over packed operands).  See
// include/lbm_nn.h.
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"
#include "lbm_nn.h"
#include "tc.cuh"

namespace lbm {
namespace nn {

using bf16 = __nv_bfloat16;

__device__ unsigned g_tc_timeouts;  // blocks of the tensor-core kernels whose waits ran out

constexpr int TC_M = 128;                        // rows per block = accumulator lanes
constexpr int TC_BK = 64;                        // reduction depth of one stage: four K = 16 MMAs
constexpr uint32_t TC_KGAP = 128;                // core matrices adjacent along K (leading byte offset)
constexpr uint32_t TC_RGAP = (TC_BK / 8) * 128;  // 8-row groups (stride byte offset)
constexpr uint32_t TC_WAIT = 1u << 24;           // polls before a wait gives up

__host__ __device__ constexpr uint32_t tc_stage_bytes(int n) { return (uint32_t)(TC_M + n) * TC_BK * 2; }
constexpr int TC_STAGES = 3;  // operand stages in flight

// The pipeline of one block: `nk` stages of depth 64 in a ring of TC_STAGES
// shared-memory buffers.  fill(a, b, kc) stages A (128 x 64) and B (n x 64),
// K-major, 16-byte row segments at tc::tile_off, with cp.async or plain
// stores; the copies of the next TC_STAGES - 1 stages are in flight while the
// tensor cores work on the current one.  Thread 0 issues a stage's four MMAs
// into the TMEM accumulator and commits them to the stage's mbarrier; a
// buffer is refilled once the MMAs that read it have completed.  Then every
// thread reads its accumulator row, 16 columns at a time, into
// out(row_in_tile, first_column, values, ok).  `n` is a multiple of 16 in
// 16 .. 256.
template <class Fill, class Out>
__device__ __forceinline__ void tc_pipeline(unsigned char* smem, uint64_t* mbar, uint32_t* tmem_slot, int n, int nk,
                                            Fill fill, Out out) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t a_bytes = TC_M * TC_BK * 2;
    const uint32_t stage_bytes = tc_stage_bytes(n);
    uint32_t ncols = 32;
    while (ncols < (uint32_t)n) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(tmem_slot, ncols);
    if (tid == 0)
        for (int s = 0; s < TC_STAGES; s++) tc::mbar_init(&mbar[s], 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = tc::idesc_bf16_f32(TC_M, n);
    bool ok = true;
    // one cp.async group per stage, empty past the end, so that "all but the
    // newest TC_STAGES - 2 groups complete" always means "this stage landed"
    for (int p = 0; p < TC_STAGES - 1; p++) {
        if (p < nk) fill(smem + p * stage_bytes, smem + p * stage_bytes + a_bytes, p);
        tc::cp_async_commit();
    }
    for (int kc = 0; kc < nk; kc++) {
        const int s = kc % TC_STAGES;
        unsigned char* sa = smem + s * stage_bytes;
        tc::cp_async_wait<TC_STAGES - 2>();
        tc::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_u32(sa), b0 = a0 + a_bytes;
#pragma unroll
            for (int j = 0; j < TC_BK / 16; j++)
                tc::mma_bf16(tmem, tc::smem_desc(a0 + 2 * j * TC_KGAP, TC_KGAP, TC_RGAP),
                             tc::smem_desc(b0 + 2 * j * TC_KGAP, TC_KGAP, TC_RGAP), idesc, kc > 0 || j > 0);
            tc::mma_commit(&mbar[s]);
        }
        // refill the buffer of stage kc - 1 with stage kc + TC_STAGES - 1, once its MMAs are done
        const int nxt = kc + TC_STAGES - 1;
        if (nxt < nk) {
            const int r = nxt % TC_STAGES;
            if (kc >= 1) ok &= tc::mbar_wait(&mbar[r], ((kc - 1) / TC_STAGES) & 1, TC_WAIT);
            fill(smem + r * stage_bytes, smem + r * stage_bytes + a_bytes, nxt);
        }
        tc::cp_async_commit();
    }
    // the last commit arrives once every MMA of the block has completed
    const int last = nk - 1;
    bool done = tc::mbar_wait(&mbar[last % TC_STAGES], (last / TC_STAGES) & 1, TC_WAIT);
    if (!done) done = tc::mbar_wait(&mbar[last % TC_STAGES], (last / TC_STAGES) & 1, TC_WAIT);
    ok &= done;
    tc::cp_async_wait<0>();
    if (!ok && lane == 0) atomicAdd(&g_tc_timeouts, 1u);
    tc::fence_after_sync();
    for (int c0 = 0; c0 < n; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        out(warp * 32 + lane, c0, v, ok);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, ncols);
    }
}

// C[m][n] = sum_k A[m][k] B[n][k]: A, B BF16 with K contiguous, C FP32;
// M % 128 == 0, N % 16 == 0 (16 .. 256), K % 64 == 0.
__global__ void __launch_bounds__(128) k_gemm_tc(const bf16* __restrict__ A, const bf16* __restrict__ B,
                                                 float* __restrict__ C, int N, int K) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t mbar[TC_STAGES];
    __shared__ uint32_t tmem_slot;
    const int m0 = blockIdx.x * TC_M;
    auto fill = [&](unsigned char* sa, unsigned char* sb, int kc) {
        for (int e = threadIdx.x; e < TC_M * 8; e += 128) {
            const int r = e >> 3, g = e & 7;
            tc::cp_async16(sa + tc::tile_off(r, g, TC_KGAP, TC_RGAP), A + (size_t)(m0 + r) * K + kc * TC_BK + g * 8,
                           true);
        }
        for (int e = threadIdx.x; e < N * 8; e += 128) {
            const int r = e >> 3, g = e & 7;
            tc::cp_async16(sb + tc::tile_off(r, g, TC_KGAP, TC_RGAP), B + (size_t)r * K + kc * TC_BK + g * 8, true);
        }
    };
    auto out = [&](int r, int c0, const float (&v)[16], bool ok) {
#pragma unroll
        for (int k = 0; k < 16; k++) C[(size_t)(m0 + r) * N + c0 + k] = ok ? v[k] : __int_as_float(0x7fc00000);
    };
    tc_pipeline(smem, mbar, &tmem_slot, N, K / TC_BK, fill, out);
}

// Neighbour coordinate along one axis: zero padding (-1 outside) or periodic.
__device__ __forceinline__ int tc_nb(int c, int d, int n, bool wrap) {
    c += d;
    if (wrap) return c < 0 ? c + n : (c >= n ? c - n : c);
    return (c < 0 || c >= n) ? -1 : c;
}

// The 3x3x3 convolution of lbm_nn_conv3d as an implicit GEMM:
// y[p][co] = act(sum_k A[p][k] B[co][k] + bias[co]) with k = (tap, ci),
// A[p][(tap, ci)] = x[p + off(tap)][ci] (zero outside, or wrapped on the axes
// of `wrap`) and B[co][(tap, ci)] = wgt[tap][ci][co].  One block computes 128
// voxels x NT output channels from blockIdx.y * NT; Cin % 8 == 0 (each 16-byte
// row segment lies in one tap), NT % 16 == 0.  Rows k >= 27 Cin of the last
// stage are zero.
__global__ void __launch_bounds__(128) k_conv_tc(const bf16* __restrict__ x, int N, int D, int H, int W, int Cin,
                                                 const bf16* __restrict__ wgt, const float* __restrict__ bias,
                                                 int Cout, int NT, int relu, int wrap, bf16* __restrict__ y,
                                                 float* __restrict__ y32) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t mbar[TC_STAGES];
    __shared__ uint32_t tmem_slot;
    const long long M = (long long)N * D * H * W;
    const int K = 27 * Cin;
    const long long m0 = (long long)blockIdx.x * TC_M;
    const int n0 = blockIdx.y * NT;
    const bool wx = wrap & 1, wy = wrap & 2, wz = wrap & 4;
    // voxel (n, z, y, x) of each of the block's rows (n < 0: past the end)
    __shared__ int4 vox[TC_M];
    {
        const long long p = m0 + threadIdx.x;
        int4 c = make_int4(-1, 0, 0, 0);
        if (p < M) {
            long long t = p;
            c.w = (int)(t % W);
            t /= W;
            c.z = (int)(t % H);
            t /= H;
            c.y = (int)(t % D);
            c.x = (int)(t / D);
        }
        vox[threadIdx.x] = c;
    }
    __syncthreads();
    // a thread fills K group g = tid % 8 of rows tid / 8 + 16 j, j = 0 .. 7
    auto fill = [&](unsigned char* sa, unsigned char* sb, int kc) {
        const int g = threadIdx.x & 7;
        const int k = kc * TC_BK + g * 8;
        const bool kin = k < K;
        const int tap = kin ? k / Cin : 0, ci = k - tap * Cin;
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int r = (threadIdx.x >> 3) + 16 * j;
            const int4 c = vox[r];
            const bf16* src = x;  // a zero fill (padding, past the end) reads nothing
            bool full = false;
            if (kin && c.x >= 0) {
                const int zz = tc_nb(c.y, dz, D, wz), yy = tc_nb(c.z, dy, H, wy), xx = tc_nb(c.w, dx, W, wx);
                if ((zz | yy | xx) >= 0) {
                    src = x + ((((long long)c.x * D + zz) * H + yy) * W + xx) * Cin + ci;
                    full = true;
                }
            }
            tc::cp_async16(sa + tc::tile_off(r, g, TC_KGAP, TC_RGAP), src, full);
        }
        // B[co][k] from wgt[k][co]: 8 consecutive co of one k per 16-byte load,
        // stored down the 8 rows of one segment column
        for (int e = threadIdx.x; e < TC_BK * (NT / 8); e += 128) {
            const int kk = e / (NT / 8), c8 = (e - kk * (NT / 8)) * 8;
            const int k = kc * TC_BK + kk;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (k < K && n0 + c8 < Cout) v = *reinterpret_cast<const uint4*>(wgt + (size_t)k * Cout + n0 + c8);
            const bf16* h = reinterpret_cast<const bf16*>(&v);
            const int g = kk >> 3, col = kk & 7;
#pragma unroll
            for (int j = 0; j < 8; j++)
                *reinterpret_cast<bf16*>(sb + tc::tile_off(c8 + j, g, TC_KGAP, TC_RGAP) + col * 2) = h[j];
        }
    };
    // 16 columns of one row (Cout % 16 == 0: a chunk is wholly inside or outside)
    auto out = [&](int r, int c0, const float (&v)[16], bool ok) {
        const long long row = m0 + r;
        const int co0 = n0 + c0;
        if (row >= M || co0 >= Cout) return;
        float a[16];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            a[k] = ok ? v[k] + (bias ? bias[co0 + k] : 0.f) : __int_as_float(0x7fc00000);
            if (relu) a[k] = fmaxf(a[k], 0.f);
        }
        if (y) {
            uint32_t h[8];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const __nv_bfloat162 t = __floats2bfloat162_rn(a[2 * k], a[2 * k + 1]);
                h[k] = *reinterpret_cast<const uint32_t*>(&t);
            }
            uint4* dst = reinterpret_cast<uint4*>(y + row * Cout + co0);
            dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
            dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
        }
        if (y32) {
            float4* dst = reinterpret_cast<float4*>(y32 + row * Cout + co0);
#pragma unroll
            for (int k = 0; k < 4; k++) dst[k] = make_float4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
        }
    };
    tc_pipeline(smem, mbar, &tmem_slot, NT, (K + TC_BK - 1) / TC_BK, fill, out);
}

// The 3x3x3 convolution with the activations read by the tensor cores straight
// from a shared-memory halo tile (no im2col copy).  A block computes MB bricks
// of 8 (x) x 16 (y) x 1 (z) voxels stacked along z, each brick 128 accumulator
// rows (x fastest) of NT output channels in its own TMEM columns.  The halo
// tile holds (8 + 2) x (16 + 2) x (MB + 2) voxels of up to 64 input channels
// as 16-byte cells of 8 channels, laid out [channel group][z][y][x]: for one
// tap the 8 voxels of a brick line are 8 consecutive cells, i.e. one core
// matrix, the 16 lines of a brick are 10 cells (160 B) apart, consecutive
// bricks one tile plane (180 cells) apart and two channel groups one tile
// (180 (MB + 2) cells) apart, so an MMA's A operand is a descriptor into the
// tile at the tap's and the brick's offset.  B (the weights, K-major per
// output channel) streams through a three-stage ring as in k_conv_tc; each
// stage feeds the MMAs of all MB bricks.  Input channels beyond 64 are taken
// in chunks, the tile reloaded once the MMAs of the previous chunk have
// completed.  Cin % 16 == 0, NT % 16 == 0, MB * NT <= 512.
constexpr int HX = 10, HY = 18;          // halo tile extent in x and y (z: MB + 2)
constexpr int HPLANE = HX * HY;          // cells of one z plane of the tile
constexpr uint32_t HLINE = HX * 16;      // brick lines (stride byte offset)
constexpr int HCC = 64;                  // input channels per chunk
constexpr int HMB_MAX = 4;               // bricks per block, at most

// bytes between channel groups of the tile (the descriptors' leading byte offset)
__host__ __device__ constexpr uint32_t halo_gap(int mb) { return (uint32_t)(HPLANE * (mb + 2)) * 16; }
// shared memory of a block: the halo tile of min(Cin, 64) channels and the B ring
__host__ __device__ constexpr uint32_t halo_tile_bytes(int cin, int mb) {
    return (uint32_t)((cin < HCC ? cin : HCC) / 8) * halo_gap(mb);
}
__host__ __device__ constexpr uint32_t halo_smem_bytes(int cin, int nt, int mb) {
    return halo_tile_bytes(cin, mb) + TC_STAGES * (uint32_t)nt * TC_BK * 2;
}

// Halo-tile coordinate c (the box's coordinate, possibly -1 .. n) along an
// axis of n voxels: periodic or zero padding; -1 (a zero cell) as well beyond
// one voxel past either edge, where only rows outside the box would read it.
__device__ __forceinline__ int halo_nb(int c, int n, bool wrap) {
    if (c < -1 || c > n) return -1;
    if (wrap) return c < 0 ? c + n : (c >= n ? c - n : c);
    return (c < 0 || c >= n) ? -1 : c;
}

// The weights of the halo-tile convolution as the B stages it streams: for
// output-channel tile ty (NT channels from ty * NT) and global stage gs (the
// stages of input-channel chunk cb = 0, HCC, .. in order, 27 cc / TC_BK
// rounded up per chunk of cc channels), the stage's NT x TC_BK operand in its
// shared-memory layout (K-major core matrices, tile_off), element (co, kk) =
// wgt[tap][cb + ci][ty NT + co] for k = (stage within chunk) TC_BK + kk = tap
// cc + ci, zero past the chunk's 27 cc rows or past Cout.  One thread per
// 16-byte core-matrix row (8 consecutive kk of one co).
__global__ void k_pack_weights(const bf16* __restrict__ wgt, int Cin, int Cout, int NT, int G_total,
                               unsigned char* __restrict__ wpack) {
    const uint32_t bstage = (uint32_t)NT * TC_BK * 2;
    const long long units = (long long)bstage / 16;  // per stage
    const long long total = (long long)((Cout + NT - 1) / NT) * G_total * units;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long u = e % units, stage = e / units;
        const int gs = (int)(stage % G_total), ty = (int)(stage / G_total);
        // chunk and stage within it
        int cb = 0, kc = gs;
        for (;;) {
            const int cc = Cin - cb < HCC ? Cin - cb : HCC;
            const int nk = (27 * cc + TC_BK - 1) / TC_BK;
            if (kc < nk) break;
            kc -= nk;
            cb += HCC;
        }
        const int cc = Cin - cb < HCC ? Cin - cb : HCC;
        const int c8 = (int)(u / (TC_BK / 8)) , gk = (int)(u % (TC_BK / 8));  // row co = c8, k-group gk
        const int co = ty * NT + c8;
        uint4 out;
        bf16* h = reinterpret_cast<bf16*>(&out);
#pragma unroll
        for (int col = 0; col < 8; col++) {
            const int k = kc * TC_BK + gk * 8 + col;
            bf16 v = __float2bfloat16(0.f);
            if (k < 27 * cc && co < Cout) {
                const int tap = k / cc, ci = k - tap * cc;
                v = wgt[((size_t)tap * Cin + cb + ci) * Cout + co];
            }
            h[col] = v;
        }
        *reinterpret_cast<uint4*>(wpack + (size_t)stage * bstage + tc::tile_off(c8, gk, TC_KGAP, TC_RGAP)) = out;
    }
}

__global__ void __launch_bounds__(128) k_conv_halo(const bf16* __restrict__ x, int N, int D, int H, int W, int Cin,
                                                   const unsigned char* __restrict__ wpack, int G_total,
                                                   const float* __restrict__ bias,
                                                   int Cout, int NT, int MB, int relu, int wrap,
                                                   bf16* __restrict__ y, float* __restrict__ y32) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t mbar[TC_STAGES];
    __shared__ uint32_t tmem_slot;
    unsigned char* const tile = smem;
    unsigned char* const ring = smem + halo_tile_bytes(Cin, MB);
    const uint32_t bstage = (uint32_t)NT * TC_BK * 2;
    const uint32_t hgap = halo_gap(MB);
    const int hcells = HPLANE * (MB + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int BX = (W + 7) / 8, BY = (H + 15) / 16, BZ = (D + MB - 1) / MB;
    int b = blockIdx.x;
    const int xb = b % BX;
    b /= BX;
    const int yb = b % BY;
    b /= BY;
    const int z0 = (b % BZ) * MB, n0 = b / BZ;
    const int x0 = xb * 8, y0 = yb * 16;
    const int nb = D - z0 < MB ? D - z0 : MB;  // bricks inside the box
    const int c0 = blockIdx.y * NT;
    const bool wx = wrap & 1, wy = wrap & 2, wz = wrap & 4;

    uint32_t ncols = 32;
    while (ncols < (uint32_t)(MB * NT)) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(&tmem_slot, ncols);
    if (tid == 0)
        for (int s = 0; s < TC_STAGES; s++) tc::mbar_init(&mbar[s], 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = tc::idesc_bf16_f32(TC_M, NT);
    const uint32_t tile_a = tc::smem_u32(tile);
    bool ok = true;
    int g = 0;  // stages issued by the block so far (selects the ring buffer and mbarrier phase)

    // B stage number gs of this block's channel tile (k_pack_weights wrote it
    // in its shared-memory layout): one 16-byte copy per core-matrix row
    const unsigned char* const wtile = wpack + (size_t)blockIdx.y * G_total * bstage;
    auto fill_b = [&](unsigned char* sb, int gs) {
        const unsigned char* src = wtile + (size_t)gs * bstage;
        for (uint32_t e = tid; e < bstage / 16; e += 128) tc::cp_async16(sb + e * 16, src + e * 16, true);
    };

    for (int cb = 0; cb < Cin; cb += HCC) {
        const int cc = Cin - cb < HCC ? Cin - cb : HCC;
        const int nk = (27 * cc + TC_BK - 1) / TC_BK;
        if (cb > 0) {  // every MMA that reads the tile has completed
            const int last = g - 1;
            ok &= tc::mbar_wait(&mbar[last % TC_STAGES], (last / TC_STAGES) & 1, TC_WAIT);
        }
        // the halo tile of this chunk (zero outside the box, wrapped on periodic axes)
        for (int e = tid; e < (cc / 8) * hcells; e += 128) {
            const int cg = e / hcells, cell = e - cg * hcells;
            const int hx = cell % HX, hy = (cell / HX) % HY, hz = cell / HPLANE;
            const int zz = halo_nb(z0 + hz - 1, D, wz), yy = halo_nb(y0 + hy - 1, H, wy),
                      xx = halo_nb(x0 + hx - 1, W, wx);
            const bool full = (zz | yy | xx) >= 0;
            const bf16* src = full ? x + ((((long long)n0 * D + zz) * H + yy) * W + xx) * Cin + cb + cg * 8 : x;
            tc::cp_async16(tile + (size_t)e * 16, src, full);
        }
        // the ring's first stages join the tile's copies in the first group
        for (int p = 0; p < TC_STAGES - 1; p++) {
            if (p < nk) fill_b(ring + ((g + p) % TC_STAGES) * bstage, g + p);
            tc::cp_async_commit();
        }
        for (int kc = 0; kc < nk; kc++, g++) {
            const int s = g % TC_STAGES;
            tc::cp_async_wait<TC_STAGES - 2>();
            tc::fence_smem_to_async();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t b0 = tc::smem_u32(ring + s * bstage);
#pragma unroll
                for (int j = 0; j < TC_BK / 16; j++) {
                    const int k = kc * TC_BK + 16 * j;
                    if (k >= 27 * cc) break;
                    const int tap = k / cc, ci = k - tap * cc;
                    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;  // 0 .. 2: offsets -1 .. +1
                    const uint32_t a = tile_a + (uint32_t)(ci / 8) * hgap + (uint32_t)((dz * HY + dy) * HX + dx) * 16;
                    const uint64_t bdesc = tc::smem_desc(b0 + 2 * j * TC_KGAP, TC_KGAP, TC_RGAP);
                    for (int m = 0; m < nb; m++)  // brick m: one tile plane further along z
                        tc::mma_bf16(tmem + (uint32_t)(m * NT), tc::smem_desc(a + (uint32_t)(m * HPLANE) * 16, hgap, HLINE),
                                     bdesc, idesc, cb > 0 || kc > 0 || j > 0);
                }
                tc::mma_commit(&mbar[s]);
            }
            const int nxt = kc + TC_STAGES - 1;
            if (nxt < nk) {
                const int r = (g + TC_STAGES - 1) % TC_STAGES;
                if (kc >= 1) ok &= tc::mbar_wait(&mbar[r], ((g - 1) / TC_STAGES) & 1, TC_WAIT);
                fill_b(ring + r * bstage, g + TC_STAGES - 1);
            }
            tc::cp_async_commit();
        }
        tc::cp_async_wait<0>();
    }
    const int last = g - 1;
    bool done = tc::mbar_wait(&mbar[last % TC_STAGES], (last / TC_STAGES) & 1, TC_WAIT);
    if (!done) done = tc::mbar_wait(&mbar[last % TC_STAGES], (last / TC_STAGES) & 1, TC_WAIT);
    ok &= done;
    if (!ok && lane == 0) atomicAdd(&g_tc_timeouts, 1u);
    tc::fence_after_sync();
    // row r of brick m's accumulator = voxel (x0 + r % 8, y0 + r / 8, z0 + m) of sample n0
    const int r = warp * 32 + lane;
    const int vx = x0 + (r & 7), vy = y0 + (r >> 3);
    const bool inside = vx < W && vy < H;
    for (int q = 0; q < nb * NT; q += 16) {  // brick q / NT, its columns q % NT ..
        const int m = q / NT, cq = q - m * NT;
        const long long row = (((long long)n0 * D + z0 + m) * H + vy) * W + vx;
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)q, v);
        const int co0 = c0 + cq;
        if (!inside || co0 >= Cout) continue;
        float a[16];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            a[k] = ok ? v[k] + (bias ? bias[co0 + k] : 0.f) : __int_as_float(0x7fc00000);
            if (relu) a[k] = fmaxf(a[k], 0.f);
        }
        if (y) {
            uint32_t h[8];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const __nv_bfloat162 t = __floats2bfloat162_rn(a[2 * k], a[2 * k + 1]);
                h[k] = *reinterpret_cast<const uint32_t*>(&t);
            }
            uint4* dst = reinterpret_cast<uint4*>(y + row * Cout + co0);
            dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
            dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
        }
        if (y32) {
            float4* dst = reinterpret_cast<float4*>(y32 + row * Cout + co0);
#pragma unroll
            for (int k = 0; k < 4; k++) dst[k] = make_float4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, ncols);
    }
}

// ---- weight gradient on the tensor cores ------------------------------------
//
// dw[tap][ci][co] = sum_p x[p + off(tap)][ci] dy[p][co] as 27 K-major GEMMs
// over voxels.  x and dy are first packed channel-major over a padded grid
// (D + 2) x (H + 2) x Wp, Wp >= W + 2 a multiple of 8: padded voxel q holds x
// at q minus one voxel on each axis (wrapped on periodic axes, zero outside),
// dy only at interior voxels (zero on the padding).  With flat indices, the
// voxel p + off(tap) is q + dz Hp Wp + dy Wp + dx; the dz and dy parts are
// multiples of 8 values (16 bytes), and dx in {-1, 0, 1} is taken from one of
// three copies of packed x shifted by one value, so every operand row starts
// 16-byte aligned.  Rows are Lp values long, the data G values in, with zero
// guards of G values (G > Hp Wp + Wp) before and after.
//
//   xp[(dx + 1) Cp + ci][G + q] = xpad[ci][q + dx],   dyp[co][G + q] = dypad[co][q]
//
// with Cp the input channels rounded up to 16 (the rows past Cin zero).
constexpr int WG_STAGES = 3;
constexpr int WG_THREADS = 256;  // two warps per TMEM lane quadrant

// One block per padded row (sample, z, y): the row's values go through shared
// memory ([voxel][channel], an odd number of 32-bit words per voxel so that
// the channel-major reads do not collide in banks) and out channel-major,
// one warp per output row.  x has Cin channels, written as Cp >= Cin rows per
// copy (the rows past Cin zero).
__host__ __device__ constexpr int wg_pack_stride(int c) { return 2 * (((c + 1) / 2) | 1); }

__global__ void k_wgrad_pack(const bf16* __restrict__ x, const bf16* __restrict__ dy, int D, int H, int W, int Cin,
                             int Cp, int Cout, int wrap, int Hp, int Wp, long long G, long long Lp, bf16* __restrict__ xp,
                             bf16* __restrict__ dyp) {
    extern __shared__ __align__(16) unsigned char pack_smem[];
    const int sx = wg_pack_stride(Cp), sd = wg_pack_stride(Cout);
    bf16* xs = reinterpret_cast<bf16*>(pack_smem);
    bf16* ds = xs + (size_t)Wp * sx;
    const long long r = blockIdx.x;  // padded row
    const int Dp = D + 2;
    const int yp = (int)(r % Hp), zp = (int)((r / Hp) % Dp);
    const long long n = r / ((long long)Hp * Dp);
    const bool wx = wrap & 1, wy = wrap & 2, wz = wrap & 4;
    const int zs = halo_nb(zp - 1, D, wz), ys = halo_nb(yp - 1, H, wy);
    const bool interior = zp >= 1 && zp <= D && yp >= 1 && yp <= H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bf16 z0 = __float2bfloat16(0.f);
    // one 16-byte load per 8 channels where the channel count and alignment
    // allow (every load of the block in flight at once), else one per value
    auto load_row = [&](const bf16* base, int C, int Cw, bf16* dst, int sdst, bool vec, auto src_ok) {
        if (vec) {
            const int g8 = Cw / 8;
            for (int e = threadIdx.x; e < Wp * g8; e += blockDim.x) {
                const int v = e / g8, c8 = e - v * g8;
                uint4 val = make_uint4(0, 0, 0, 0);
                const long long off = src_ok(v);
                if (off >= 0 && c8 * 8 < C) val = *reinterpret_cast<const uint4*>(base + off * C + c8 * 8);
                const bf16* h8 = reinterpret_cast<const bf16*>(&val);
#pragma unroll
                for (int k = 0; k < 8; k++) dst[(size_t)v * sdst + c8 * 8 + k] = h8[k];
            }
        } else {
            for (int e = threadIdx.x; e < Wp * Cw; e += blockDim.x) {
                const int v = e / Cw, c = e - v * Cw;
                const long long off = src_ok(v);
                dst[(size_t)v * sdst + c] = (off >= 0 && c < C) ? base[off * C + c] : z0;
            }
        }
    };
    const long long xrow = ((n * D + zs) * H + ys) * W;  // voxel index of (zs, ys, 0)
    load_row(x, Cin, Cp, xs, sx, Cin % 8 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0, [&](int v) -> long long {
        const int xs_ = halo_nb(v - 1, W, wx);
        return (zs | ys | xs_) >= 0 ? xrow + xs_ : -1;
    });
    const long long drow = ((n * D + zp - 1) * H + yp - 1) * W;
    load_row(dy, Cout, Cout, ds, sd, Cout % 8 == 0 && (reinterpret_cast<uintptr_t>(dy) & 15) == 0,
             [&](int v) -> long long { return interior && v >= 1 && v <= W ? drow + v - 1 : -1; });
    __syncthreads();
    // two values per 32-bit store (rows start at even offsets: G, Lp, Wp even)
    const long long row0 = G + r * Wp;
    const int wh = Wp / 2;
    for (int rc = warp; rc < 3 * Cp; rc += nw) {  // rc = (dx + 1) Cp + ci
        const int sh = rc / Cp - 1, ci = rc - (sh + 1) * Cp;
        uint32_t* dst = reinterpret_cast<uint32_t*>(xp + (size_t)rc * Lp + row0);
        for (int vp = lane; vp < wh; vp += 32) {
            const int s0 = 2 * vp + sh, s1 = s0 + 1;
            __nv_bfloat162 pr;
            pr.x = (s0 >= 0 && s0 < Wp) ? xs[(size_t)s0 * sx + ci] : z0;
            pr.y = (s1 >= 0 && s1 < Wp) ? xs[(size_t)s1 * sx + ci] : z0;
            dst[vp] = *reinterpret_cast<const uint32_t*>(&pr);
        }
    }
    for (int co = warp; co < Cout; co += nw) {
        uint32_t* dst = reinterpret_cast<uint32_t*>(dyp + (size_t)co * Lp + row0);
        for (int vp = lane; vp < wh; vp += 32) {
            __nv_bfloat162 pr;
            pr.x = ds[(size_t)(2 * vp) * sd + co];
            pr.y = ds[(size_t)(2 * vp + 1) * sd + co];
            dst[vp] = *reinterpret_cast<const uint32_t*>(&pr);
        }
    }
}

// One block: 128 output channels (from blockIdx.z * 128; rows past Cout are
// zero) x the Cp columns of each of TG taps (from blockIdx.y * TG), summed
// over the voxel steps [blockIdx.x * spc, ..) of 64 values.  Each stage holds
// the dy tile (A, 128 x 64) and the TG shifted x tiles (B, Cp x 64 each),
// K-major; the x tiles lie back to back with one 8-row stride, so one MMA
// covers up to 256 / Cp taps, one TMEM accumulator column range per tap.  The
// two warps of each TMEM lane quadrant split the fills (taps of one parity
// each) and the epilogue's column chunks; the three-stage ring and the bounded
// waits are those of tc_pipeline.  The block's sums go to the partial sums of
// its voxel chunk, part[blockIdx.x][tap][ci][co] (plain stores, NaN when a
// wait ran out); k_sum_chunks adds the chunks to dw in a fixed order, so the
// gradient does not depend on the order in which blocks finish.
__global__ void __launch_bounds__(WG_THREADS) k_wgrad_tc(const bf16* __restrict__ xp, const bf16* __restrict__ dyp, int Cin,
                                                  int Cp, int Cout, int Hp, int Wp, long long G, long long Lp,
                                                  long long nsteps, long long spc, int TG, float* __restrict__ part) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t mbar[WG_STAGES];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t0 = blockIdx.y * TG, ntap = 27 - t0 < TG ? 27 - t0 : TG;
    const int m0 = blockIdx.z * TC_M;
    const long long s0 = (long long)blockIdx.x * spc, s1 = s0 + spc < nsteps ? s0 + spc : nsteps;
    const int nk = (int)(s1 - s0);
    const uint32_t a_bytes = TC_M * TC_BK * 2, b_bytes = (uint32_t)Cp * TC_BK * 2;
    const uint32_t stage_bytes = a_bytes + (uint32_t)TG * b_bytes;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(TG * Cp)) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(&tmem_slot, ncols);
    if (tid == 0)
        for (int s = 0; s < WG_STAGES; s++) tc::mbar_init(&mbar[s], 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int tpm = 256 / Cp;  // taps per MMA
    bool ok = true;
    // this thread's 16-byte segment g of rows r0, r0 + 16, .. (of the taps of
    // its parity): fixed bases, per tap one offset (the copy for dx and the
    // dz, dy shift)
    const int th = tid & 127, par = tid >> 7;
    const int g = th & 7, r0 = th >> 3;
    const uint32_t so = tc::tile_off(r0, g, TC_KGAP, TC_RGAP), so16 = 2 * TC_RGAP;  // + 16 rows
    const bf16* xb = xp + (size_t)r0 * Lp + g * 8;
    const bf16* ab = dyp + g * 8;
    const long long copy = (long long)Cp * Lp, plane = (long long)Hp * Wp;
    auto fill = [&](unsigned char* st, int kc) {
        const long long q = G + (s0 + kc) * TC_BK;
#pragma unroll
        for (int j = par; j < TC_M / 16; j += 2) {
            const int co = m0 + r0 + 16 * j;
            tc::cp_async16(st + so + j * so16, ab + (size_t)(co < Cout ? co : 0) * Lp + q, co < Cout);
        }
        unsigned char* sb = st + a_bytes + so + par * b_bytes;
#pragma unroll 1
        for (int t = par; t < ntap; t += 2, sb += 2 * b_bytes) {
            const int tap = t0 + t;
            const bf16* src = xb + (tap % 3) * copy + (tap / 9 - 1) * plane + (long long)((tap / 3) % 3 - 1) * Wp + q;
            for (int ci = r0, k = 0; ci < Cp; ci += 16, k++)
                tc::cp_async16(sb + k * so16, src + (size_t)(ci - r0) * Lp, true);
        }
    };
    for (int p = 0; p < WG_STAGES - 1; p++) {
        if (p < nk) fill(smem + p * stage_bytes, p);
        tc::cp_async_commit();
    }
    for (int kc = 0; kc < nk; kc++) {
        const int s = kc % WG_STAGES;
        unsigned char* st = smem + s * stage_bytes;
        tc::cp_async_wait<WG_STAGES - 2>();
        tc::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_u32(st);
            // the taps' x tiles follow each other with the same 8-row stride:
            // one MMA covers up to 256 / Cp taps (N = their Cp columns each)
            for (int t = 0; t < ntap; t += tpm) {
                const int nn = (ntap - t < tpm ? ntap - t : tpm) * Cp;
                const uint32_t id = tc::idesc_bf16_f32(TC_M, nn);
                const uint32_t b0 = a0 + a_bytes + (uint32_t)t * b_bytes;
#pragma unroll
                for (int j = 0; j < TC_BK / 16; j++)
                    tc::mma_bf16(tmem + (uint32_t)(t * Cp), tc::smem_desc(a0 + 2 * j * TC_KGAP, TC_KGAP, TC_RGAP),
                                 tc::smem_desc(b0 + 2 * j * TC_KGAP, TC_KGAP, TC_RGAP), id, kc > 0 || j > 0);
            }
            tc::mma_commit(&mbar[s]);
        }
        const int nxt = kc + WG_STAGES - 1;
        if (nxt < nk) {
            const int r = nxt % WG_STAGES;
            if (kc >= 1) ok &= tc::mbar_wait(&mbar[r], ((kc - 1) / WG_STAGES) & 1, TC_WAIT);
            fill(smem + r * stage_bytes, nxt);
        }
        tc::cp_async_commit();
    }
    if (nk > 0) {
        const int last = nk - 1;
        bool done = tc::mbar_wait(&mbar[last % WG_STAGES], (last / WG_STAGES) & 1, TC_WAIT);
        if (!done) done = tc::mbar_wait(&mbar[last % WG_STAGES], (last / WG_STAGES) & 1, TC_WAIT);
        ok &= done;
    }
    tc::cp_async_wait<0>();
    if (!ok && lane == 0) atomicAdd(&g_tc_timeouts, 1u);
    tc::fence_after_sync();
    // warps w and w + 4 read the same TMEM lanes (32 (w % 4) ..), alternate chunks
    const int quad = warp & 3;
    const int co = m0 + quad * 32 + lane;
    if (nk > 0)
        for (int c0 = 16 * par; c0 < ntap * Cp; c0 += 32) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
            if (co >= Cout) continue;
            const int t = c0 / Cp, ci0 = c0 - t * Cp;  // Cp % 16 == 0: one tap per 16 columns
            float* dst = part + (size_t)blockIdx.x * 27 * Cin * Cout + ((size_t)(t0 + t) * Cin + ci0) * Cout + co;
#pragma unroll
            for (int k = 0; k < 16; k++)
                if (ci0 + k < Cin) dst[(size_t)k * Cout] = ok ? v[k] : __int_as_float(0x7fc00000);
        }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, ncols);
    }
}

}  // namespace nn
}  // namespace lbm

using namespace lbm;
using namespace lbm::nn;

static int tc_launch_ok(const void* kernel, uint32_t smem, const char* what) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, what);
}

extern "C" int lbm_nn_gemm_bf16(const void* a, const void* b, float* c, int m, int n, int k, void* stream) {
    if (!a || !b || !c || m < 1 || n < 16 || n > 256 || k < 1 || m % TC_M || n % 16 || k % TC_BK)
        return fail(LBM_ERR_ARG, "lbm_nn_gemm_bf16: needs m %% 128 == 0, n %% 16 == 0 in 16..256, k %% 64 == 0");
    const uint32_t smem = TC_STAGES * tc_stage_bytes(n);
    int rc = tc_launch_ok((const void*)k_gemm_tc, smem, "cudaFuncSetAttribute(k_gemm_tc)");
    if (rc) return rc;
    k_gemm_tc<<<m / TC_M, 128, smem, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(a),
                                                                           static_cast<const bf16*>(b), c, n, k);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "k_gemm_tc launch");
}

namespace lbm {
namespace nn {
// The tensor-core convolution for the shapes it takes (cin % 8 == 0, cout %
// 16 == 0, 16-byte aligned operands); returns 1, launching nothing, for the
// others.
int conv3d_tc(const void* x, int n, int d, int h, int w, int cin, const void* wgt, const float* bias, int cout,
              int relu, int wrap, void* y, float* y32, cudaStream_t s) {
    if (cin % 8 || cout % 16 || ((uintptr_t)x | (uintptr_t)wgt | (uintptr_t)y | (uintptr_t)y32) & 15) return 1;
    const int tiles = (cout + 127) / 128;
    const int nt = ((cout / tiles + 15) / 16) * 16;
    const long long M = (long long)n * d * h * w;
    const long long gx = (M + TC_M - 1) / TC_M;
    if (gx > 0x7fffffff) return 1;
    const uint32_t smem = TC_STAGES * tc_stage_bytes(nt);
    int rc = tc_launch_ok((const void*)k_conv_tc, smem, "cudaFuncSetAttribute(k_conv_tc)");
    if (rc) return rc;
    k_conv_tc<<<dim3((unsigned)gx, (unsigned)((cout + nt - 1) / nt)), 128, smem, s>>>(
        static_cast<const bf16*>(x), n, d, h, w, cin, static_cast<const bf16*>(wgt), bias, cout, nt, relu, wrap,
        static_cast<bf16*>(y), y32);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "k_conv_tc launch");
}
}  // namespace nn
}  // namespace lbm

namespace lbm {
namespace nn {
static int g_halo_mb = 0, g_halo_nt = 0;  // fixed by lbm_nn_conv_tune; 0 = chosen per shape
// The halo-tile convolution's weights packed as B stages (k_pack_weights):
// kept for the process, grown on demand; calls on one stream reuse it in order.
static unsigned char* g_wpack = nullptr;
static size_t g_wpack_bytes = 0;

static int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            sms = 148;
        }
    }
    return sms;
}

// The halo-tile tensor-core convolution (cin % 16 == 0, cout % 16 == 0,
// 16-byte aligned operands); returns 1, launching nothing, for other shapes.
int conv3d_halo(const void* x, int n, int d, int h, int w, int cin, const void* wgt, const float* bias, int cout,
                int relu, int wrap, void* y, float* y32, cudaStream_t s) {
    if (cin % 16 || cout % 16 || ((uintptr_t)x | (uintptr_t)wgt | (uintptr_t)y | (uintptr_t)y32) & 15) return 1;
    const long long plane_bricks = (long long)n * ((h + 15) / 16) * ((w + 7) / 8);
    if (plane_bricks * d > 0x7fffffff) return 1;
    const int sms = sm_count();
    // Launch shape: mb bricks per block along z and nt output channels per
    // block (the default tile of at most 128 channels, or a half, quarter ..
    // of it).  Preferred: at least 1.5 blocks per SM in the grid and two
    // blocks per SM by shared memory (one block's halo copy overlaps another's
    // MMAs) within the SM's 512 TMEM columns; among those, the most work per
    // block (mb nt), then the deeper brick stack.  Measured on the U-Net's
    // layers, this picks the fastest shape or one within 5 % of it.
    const int tiles = (cout + 127) / 128;
    const int nt0 = ((cout / tiles + 15) / 16) * 16;
    int mb = 0, nt = 0;
    long long key = -1;
    for (int ntc = g_halo_nt ? g_halo_nt : nt0; ntc >= 16; ntc = (ntc % 32 == 0 && !g_halo_nt) ? ntc / 2 : 0) {
        for (int m = HMB_MAX; m >= 1; m--) {
            if ((g_halo_mb && m != g_halo_mb) || (!g_halo_mb && m == 3) || m * ntc > 512) continue;
            const long long nblk = plane_bricks * ((d + m - 1) / m) * ((cout + ntc - 1) / ntc);
            uint32_t cols = 32;
            while (cols < (uint32_t)(m * ntc)) cols <<= 1;
            uint32_t per_sm = (228u << 10) / (halo_smem_bytes(cin, ntc, m) + 1024u);
            per_sm = per_sm > 16 ? 16 : per_sm;
            const bool occ = per_sm >= 2 && cols * per_sm <= 512u, grid = 2 * nblk >= 3LL * sms;
            // lexicographic: both, occupancy, then work per block (or, short of
            // a full grid, the block count), then brick depth
            const long long k = ((long long)(occ && grid) << 62) | ((long long)occ << 61) |
                                ((grid ? (long long)(m * ntc) : (nblk < (1LL << 40) ? nblk : (1LL << 40) - 1)) << 3) | m;
            if (k > key) key = k, mb = m, nt = ntc;
        }
    }
    if (!mb) return 1;
    const int gy = (cout + nt - 1) / nt;
    const long long blocks = plane_bricks * ((d + mb - 1) / mb);
    const uint32_t smem = halo_smem_bytes(cin, nt, mb);
    int rc = tc_launch_ok((const void*)k_conv_halo, smem, "cudaFuncSetAttribute(k_conv_halo)");
    if (rc) return rc;
    // the weights as the blocks' B stages (a library-owned buffer, repacked per call)
    int G_total = 0;
    for (int cb = 0; cb < cin; cb += HCC) G_total += (27 * (cin - cb < HCC ? cin - cb : HCC) + TC_BK - 1) / TC_BK;
    const size_t pack_bytes = (size_t)gy * G_total * nt * TC_BK * 2;
    if (pack_bytes > g_wpack_bytes) {
        if (g_wpack) cudaFree(g_wpack);
        g_wpack = nullptr;
        g_wpack_bytes = 0;
        if (cudaMalloc(&g_wpack, pack_bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            g_wpack = nullptr;
            return 1;  // no room: the other kernels need no packed weights
        }
        g_wpack_bytes = pack_bytes;
    }
    const long long units = (long long)pack_bytes / 16;
    k_pack_weights<<<(unsigned)((units + 127) / 128 < 1216 ? (units + 127) / 128 : 1216), 128, 0, s>>>(
        static_cast<const bf16*>(wgt), cin, cout, nt, G_total, g_wpack);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_pack_weights launch");
    k_conv_halo<<<dim3((unsigned)blocks, (unsigned)gy), 128, smem, s>>>(
        static_cast<const bf16*>(x), n, d, h, w, cin, g_wpack, G_total, bias, cout, nt, mb, relu, wrap,
        static_cast<bf16*>(y), y32);
    e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "k_conv_halo launch");
}
}  // namespace nn
}  // namespace lbm

namespace lbm {
namespace nn {
// Packed operands of the tensor-core weight gradient: one buffer kept for the
// process and grown on demand (calls on one stream reuse it in order).
static unsigned char* g_wg_buf = nullptr;
static size_t g_wg_bytes = 0;
// Per-chunk partial sums of the weight gradients (k_wgrad_tc, k_wgrad,
// k_bias_grad), summed in chunk order by k_sum_chunks: kept for the process
// and grown on demand, like the packed operands.
static float* g_part_buf = nullptr;
static size_t g_part_floats = 0;

float* chunk_scratch(size_t floats) {
    if (floats > g_part_floats) {
        if (g_part_buf) cudaFree(g_part_buf);
        g_part_buf = nullptr;
        g_part_floats = 0;
        if (cudaMalloc(&g_part_buf, floats * sizeof(float)) != cudaSuccess) {
            (void)cudaGetLastError();
            g_part_buf = nullptr;
            return nullptr;
        }
        g_part_floats = floats;
    }
    return g_part_buf;
}

// dst[e] += sum over c = 0 .. chunks-1 of part[c][e], in that order.
__global__ void k_sum_chunks(const float* __restrict__ part, long long chunks, long long E, float* __restrict__ dst) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (long long c = 0; c < chunks; c++) s += part[c * E + e];
        dst[e] += s;
    }
}

int sum_chunks(const float* part, long long chunks, long long E, float* dst, cudaStream_t s) {
    const long long blocks = (E + 255) / 256;
    k_sum_chunks<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(part, chunks, E, dst);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "k_sum_chunks launch");
}

// dw += the weight gradient on the tensor cores (input channels padded to a
// multiple of 16, 8 <= cin <= 256: below 8 the padding would multiply the
// work); returns 1, launching nothing, for other shapes or when the packed
// operands do not fit.
int wgrad_tc(const void* x, const void* dy, int n, int d, int h, int w, int cin, int cout, int wrap, float* dw,
             cudaStream_t s) {
    const int cp = (cin + 15) / 16 * 16;
    if (cin < 8 || cp > 256) return 1;
    const int Dp = d + 2, Hp = h + 2, Wp = (w + 2 + 7) / 8 * 8;
    const long long plane = (long long)Hp * Wp;
    const long long G = (plane + Wp + 8 + 63) / 64 * 64;
    const long long L = (long long)n * Dp * plane;
    const long long nsteps = (L + TC_BK - 1) / TC_BK;
    const long long Lp = 2 * G + nsteps * TC_BK;
    const size_t rows = 3 * (size_t)cp + (size_t)cout;
    const size_t bytes = rows * (size_t)Lp * 2;
    const uint32_t pack_smem = (uint32_t)Wp * (uint32_t)(wg_pack_stride(cp) + wg_pack_stride(cout)) * 2;
    if (pack_smem > 200u * 1024u || (long long)n * Dp * Hp > 0x7fffffff) return 1;
    if (bytes > g_wg_bytes) {
        if (g_wg_buf) cudaFree(g_wg_buf);
        g_wg_buf = nullptr;
        g_wg_bytes = 0;
        if (cudaMalloc(&g_wg_buf, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            g_wg_buf = nullptr;
            return 1;  // no room: the gather kernel needs none
        }
        g_wg_bytes = bytes;
    }
    bf16* xpk = reinterpret_cast<bf16*>(g_wg_buf);
    bf16* dypk = xpk + (size_t)3 * cp * Lp;
    cudaError_t e = cudaMemset2DAsync(g_wg_buf, (size_t)Lp * 2, 0, (size_t)G * 2, rows, s);
    if (e == cudaSuccess)
        e = cudaMemset2DAsync(g_wg_buf + (size_t)(G + L) * 2, (size_t)Lp * 2, 0, (size_t)(Lp - G - L) * 2, rows, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset2DAsync (weight-gradient guards)");
    int rc = tc_launch_ok((const void*)k_wgrad_pack, pack_smem, "cudaFuncSetAttribute(k_wgrad_pack)");
    if (rc) return rc;
    k_wgrad_pack<<<(unsigned)(n * (long long)Dp * Hp), 256, pack_smem, s>>>(
        static_cast<const bf16*>(x), static_cast<const bf16*>(dy), d, h, w, cin, cp, cout, wrap, Hp, Wp, G, Lp, xpk, dypk);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_wgrad_pack launch");
    // taps per block: the stage (dy tile + TG x tiles) within 72 KB, TG Cin <= 448 TMEM columns
    const int TG = 448 / cp < 27 ? 448 / cp : 27;
    const int groups = (27 + TG - 1) / TG, mt = (cout + TC_M - 1) / TC_M;
    long long chunks = sm_count() / (groups * mt);
    if (chunks < 1) chunks = 1;
    if (chunks > nsteps) chunks = nsteps;
    const long long spc = (nsteps + chunks - 1) / chunks;
    chunks = (nsteps + spc - 1) / spc;
    const uint32_t smem = WG_STAGES * (uint32_t)(TC_M * TC_BK * 2 + TG * cp * TC_BK * 2);
    rc = tc_launch_ok((const void*)k_wgrad_tc, smem, "cudaFuncSetAttribute(k_wgrad_tc)");
    if (rc) return rc;
    const long long E = 27LL * cin * cout;
    float* part = chunk_scratch((size_t)(chunks * E));
    if (!part) return fail(LBM_ERR_OOM, "weight-gradient partial sums: %lld floats", chunks * E);
    k_wgrad_tc<<<dim3((unsigned)chunks, (unsigned)groups, (unsigned)mt), WG_THREADS, smem, s>>>(xpk, dypk, cin, cp, cout, Hp, Wp,
                                                                                       G, Lp, nsteps, spc, TG, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_wgrad_tc launch");
    return sum_chunks(part, chunks, E, dw, s);
}
}  // namespace nn
}  // namespace lbm

extern "C" int lbm_nn_conv3d_tc(const void* x, int n, int d, int h, int w, int cin, const void* wgt,
                                const float* bias, int cout, int relu, int wrap, void* y, float* y32, void* stream) {
    if (!x || !wgt || n < 1 || d < 1 || h < 1 || w < 1 || cin < 1 || cout < 1 || (!y && !y32) || (wrap & ~7))
        return fail(LBM_ERR_ARG, "lbm_nn_conv3d_tc: bad arguments");
    // the halo-tile kernel for cin % 16 == 0, else the im2col one (cin % 8 == 0)
    int rc = conv3d_halo(x, n, d, h, w, cin, wgt, bias, cout, relu, wrap, y, y32, static_cast<cudaStream_t>(stream));
    if (rc == 1) rc = conv3d_tc(x, n, d, h, w, cin, wgt, bias, cout, relu, wrap, y, y32, static_cast<cudaStream_t>(stream));
    if (rc == 1)
        return fail(LBM_ERR_ARG, "lbm_nn_conv3d_tc: needs cin %% 8 == 0, cout %% 16 == 0 and 16-byte aligned operands");
    return rc;
}

extern "C" int lbm_nn_conv_tune(int bricks_z, int cout_tile) {
    if (bricks_z < 0 || bricks_z > HMB_MAX || cout_tile < 0 || cout_tile > 128 || cout_tile % 16 ||
        (bricks_z && cout_tile && bricks_z * cout_tile > 512))
        return fail(LBM_ERR_ARG, "lbm_nn_conv_tune: bricks_z in 0..4, cout_tile a multiple of 16 in 0..128");
    g_halo_mb = bricks_z;
    g_halo_nt = cout_tile;
    return LBM_OK;
}

extern "C" int lbm_nn_tc_timeouts(unsigned* count) {
    if (!count) return fail(LBM_ERR_ARG, "lbm_nn_tc_timeouts: NULL argument");
    cudaError_t e = cudaMemcpyFromSymbol(count, g_tc_timeouts, sizeof(unsigned));
    if (e == cudaSuccess) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_tc_timeouts, &zero, sizeof(unsigned));
    }
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "lbm_nn_tc_timeouts");
}

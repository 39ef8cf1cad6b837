// nn.cu -- kernels of the learned warm start (not in the paper): 3x3x3
// convolutions as implicit GEMMs on tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation) for the shapes the tcgen05 kernels of
// nn_tc.cu do not take, their backward passes, the dispatch between the two,
// and the elementwise steps of training.  See include/lbm_nn.h.
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"
#include "lbm_nn.h"

namespace lbm {
namespace nn {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned lds32(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }

constexpr int BM = 64;  // GEMM rows per block
constexpr int BK = 32;  // reduction depth per shared-memory stage
constexpr int LD = BK + 8;

// Neighbour coordinate along one axis with zero padding (returns -1 outside)
// or periodic wrap.
__device__ __forceinline__ int nb_coord(int c, int d, int n, bool wrap) {
    c += d;
    if (wrap) return c < 0 ? c + n : (c >= n ? c - n : c);
    return (c < 0 || c >= n) ? -1 : c;
}

// C[p][co] = sum_k A[p][k] B[k][co], A[p][(tap,ci)] = x[p + off(tap)][ci] (0 outside,
// or wrapped on the axes set in `wrap`), B[(tap,ci)][co] = wgt[tap][ci][co]; one
// block computes 64 voxels x NF*8 outputs starting at channel blockIdx.y * NF*8.
// VEC: Cin % 16 == 0, so that a thread's 16 consecutive k share one tap and are
// read as two 16-byte vectors.
template <int NF, bool VEC>
__global__ void __launch_bounds__(128) k_conv(const bf16* __restrict__ x, int N, int D, int H, int W, int Cin,
                                              const bf16* __restrict__ wgt, const float* __restrict__ bias,
                                              int Cout, int relu, int wrap, bf16* __restrict__ y,
                                              float* __restrict__ y32) {
    constexpr int BN = NF * 8;
    __shared__ __align__(16) bf16 As[BM][LD];
    __shared__ __align__(16) bf16 Bs[BN][LD];
    const long long M = (long long)N * D * H * W;
    const int K = 27 * Cin;
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float acc[NF][4];
#pragma unroll
    for (int f = 0; f < NF; f++) acc[f][0] = acc[f][1] = acc[f][2] = acc[f][3] = 0.f;

    // this thread gathers row ar, columns ak .. ak+15 of every A stage
    const int ar = tid >> 1, ak = (tid & 1) * 16;
    const long long am = m0 + ar;
    const bool arow = am < M;
    int an = 0, az = 0, ay = 0, ax = 0;
    if (arow) {
        long long t = am;
        ax = (int)(t % W);
        t /= W;
        ay = (int)(t % H);
        t /= H;
        az = (int)(t % D);
        an = (int)(t / D);
    }
    const bool wx = wrap & 1, wy = wrap & 2, wz = wrap & 4;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += BK) {
        int k = k0 + ak;
        if (VEC) {
            uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
            if (arow && k < K) {
                const int tap = k / Cin, ci = k - tap * Cin;
                const int zz = nb_coord(az, tap / 9 - 1, D, wz), yy = nb_coord(ay, (tap / 3) % 3 - 1, H, wy),
                          xx = nb_coord(ax, tap % 3 - 1, W, wx);
                if ((zz | yy | xx) >= 0) {
                    const uint4* src =
                        reinterpret_cast<const uint4*>(x + ((((long long)an * D + zz) * H + yy) * W + xx) * Cin + ci);
                    v0 = src[0];
                    v1 = src[1];
                }
            }
            *reinterpret_cast<uint4*>(&As[ar][ak]) = v0;
            *reinterpret_cast<uint4*>(&As[ar][ak + 8]) = v1;
        } else {
            int tap = k / Cin, ci = k - tap * Cin;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                bf16 v = zero;
                if (arow && k < K) {
                    const int zz = nb_coord(az, tap / 9 - 1, D, wz), yy = nb_coord(ay, (tap / 3) % 3 - 1, H, wy),
                              xx = nb_coord(ax, tap % 3 - 1, W, wx);
                    if ((zz | yy | xx) >= 0) v = x[((((long long)an * D + zz) * H + yy) * W + xx) * Cin + ci];
                }
                As[ar][ak + j] = v;
                k++;
                if (++ci == Cin) {
                    ci = 0;
                    tap++;
                }
            }
        }
        for (int e = tid; e < BN * BK; e += 128) {
            const int kk = e / BN, nn = e - kk * BN;
            const int kg = k0 + kk;
            Bs[nn][kk] = (kg < K && n0 + nn < Cout) ? wgt[(long long)kg * Cout + n0 + nn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            const int r = warp * 16 + (lane >> 2), c = ks + (lane & 3) * 2;
            const unsigned a[4] = {lds32(&As[r][c]), lds32(&As[r + 8][c]), lds32(&As[r][c + 8]),
                                   lds32(&As[r + 8][c + 8])};
#pragma unroll
            for (int f = 0; f < NF; f++) {
                const int nn = f * 8 + (lane >> 2);
                const unsigned b[2] = {lds32(&Bs[nn][c]), lds32(&Bs[nn][c + 8])};
                mma_bf16(acc[f], a, b);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int f = 0; f < NF; f++)
#pragma unroll
        for (int h2 = 0; h2 < 2; h2++)
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const long long row = m0 + warp * 16 + (lane >> 2) + h2 * 8;
                const int co = n0 + f * 8 + (lane & 3) * 2 + j;
                if (row < M && co < Cout) {
                    float v = acc[f][h2 * 2 + j] + (bias ? bias[co] : 0.f);
                    if (relu) v = fmaxf(v, 0.f);
                    if (y) y[row * Cout + co] = __float2bfloat16(v);
                    if (y32) y32[row * Cout + co] = v;
                }
            }
}

// dW[(tap,ci)][co] = sum_p x[p + off(tap)][ci] dy[p][co]: GEMM with 64 rows of
// (tap, ci) per block, NF*8 output channels from blockIdx.z * NF*8, split over
// voxel chunks (blockIdx.y); each block stores its chunk's partial sums to
// part[blockIdx.y], added to dw in chunk order afterwards.  The gather form,
// for the shapes the tcgen05 weight gradient does not take (fewer than 8
// input channels, more than 256).
template <int NF>
__global__ void __launch_bounds__(128) k_wgrad(const bf16* __restrict__ x, const bf16* __restrict__ dy, int N,
                                               int D, int H, int W, int Cin, int Cout, int wrap,
                                               float* __restrict__ dw, long long vox_per_block) {
    constexpr int BN = NF * 8;
    __shared__ __align__(16) bf16 As[BM][LD];  // [k row][voxel]
    __shared__ __align__(16) bf16 Bs[BN][LD];  // [co][voxel]
    __shared__ int vpos[BK][4];                 // n, z, y, x of the stage's voxels (n < 0: none)
    const long long M = (long long)N * D * H * W;
    const int K = 27 * Cin;
    const int k0 = blockIdx.x * BM;
    const int n0 = blockIdx.z * BN;
    const long long v_begin = (long long)blockIdx.y * vox_per_block;
    const long long v_end = v_begin + vox_per_block < M ? v_begin + vox_per_block : M;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float acc[NF][4];
#pragma unroll
    for (int f = 0; f < NF; f++) acc[f][0] = acc[f][1] = acc[f][2] = acc[f][3] = 0.f;
    // this thread gathers row kr of every A stage, voxels vq, vq + 2, ...
    const int kr = tid & 63, vq = tid >> 6;
    const int kg = k0 + kr;
    const bool krow = kg < K;
    const int tap = krow ? kg / Cin : 0, ci = krow ? kg - tap * Cin : 0;
    const int dz = tap / 9 - 1, dyy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const bool wx = wrap & 1, wy = wrap & 2, wz = wrap & 4;
    const bf16 zero = __float2bfloat16(0.f);
    for (long long v0 = v_begin; v0 < v_end; v0 += BK) {
        if (tid < BK) {
            const long long v = v0 + tid;
            if (v < v_end) {
                long long t = v;
                vpos[tid][3] = (int)(t % W);
                t /= W;
                vpos[tid][2] = (int)(t % H);
                t /= H;
                vpos[tid][1] = (int)(t % D);
                vpos[tid][0] = (int)(t / D);
            } else {
                vpos[tid][0] = -1;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < BK / 2; j++) {
            const int vv = vq + 2 * j;
            bf16 val = zero;
            const int n = vpos[vv][0];
            if (krow && n >= 0) {
                const int zz = nb_coord(vpos[vv][1], dz, D, wz), yy = nb_coord(vpos[vv][2], dyy, H, wy),
                          xx = nb_coord(vpos[vv][3], dx, W, wx);
                if ((zz | yy | xx) >= 0) val = x[((((long long)n * D + zz) * H + yy) * W + xx) * Cin + ci];
            }
            As[kr][vv] = val;
        }
        for (int e = tid; e < BN * BK; e += 128) {
            const int vv = e / BN, nn = e - vv * BN;
            const long long v = v0 + vv;
            Bs[nn][vv] = (v < v_end && n0 + nn < Cout) ? dy[v * Cout + n0 + nn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            const int r = warp * 16 + (lane >> 2), c = ks + (lane & 3) * 2;
            const unsigned a[4] = {lds32(&As[r][c]), lds32(&As[r + 8][c]), lds32(&As[r][c + 8]),
                                   lds32(&As[r + 8][c + 8])};
#pragma unroll
            for (int f = 0; f < NF; f++) {
                const int nn = f * 8 + (lane >> 2);
                const unsigned b[2] = {lds32(&Bs[nn][c]), lds32(&Bs[nn][c + 8])};
                mma_bf16(acc[f], a, b);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int f = 0; f < NF; f++)
#pragma unroll
        for (int h2 = 0; h2 < 2; h2++)
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const int row = k0 + warp * 16 + (lane >> 2) + h2 * 8;
                const int co = n0 + f * 8 + (lane & 3) * 2 + j;
                if (row < K && co < Cout) dw[(long long)blockIdx.y * K * Cout + (long long)row * Cout + co] = acc[f][h2 * 2 + j];
            }
}

// Partial bias gradients of row blocks: part[blockIdx.x][c] = sum of dy over the block's rows.
__global__ void k_bias_grad(const bf16* __restrict__ dy, long long M, int C, float* __restrict__ part,
                            long long rows_per_block) {
    const long long r0 = (long long)blockIdx.x * rows_per_block;
    const long long r1 = r0 + rows_per_block < M ? r0 + rows_per_block : M;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.f;
        for (long long r = r0; r < r1; r++) s += __bfloat162float(dy[r * C + c]);
        part[(long long)blockIdx.x * C + c] = s;
    }
}

__global__ void k_weight_flip(const bf16* __restrict__ w, int Cin, int Cout, bf16* __restrict__ wt) {
    const long long n = 27ll * Cin * Cout;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(e % Cout);
        const long long t = e / Cout;
        const int ci = (int)(t % Cin), tap = (int)(t / Cin);
        wt[((long long)(26 - tap) * Cout + co) * Cin + ci] = w[e];
    }
}

__global__ void k_relu_mask(bf16* __restrict__ g, const bf16* __restrict__ act, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(act[e]) > 0.f)) g[e] = __float2bfloat16(0.f);
}

__global__ void k_pool2(const bf16* __restrict__ x, int N, int D, int H, int W, int C, bf16* __restrict__ y) {
    const int d = D / 2, h = H / 2, w = W / 2;
    const long long n = (long long)N * d * h * w * C;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long t = e / C;
        const int xx = (int)(t % w);
        t /= w;
        const int yy = (int)(t % h);
        t /= h;
        const int zz = (int)(t % d);
        const int nn = (int)(t / d);
        float s = 0.f;
        for (int k = 0; k < 8; k++) {
            const int z = 2 * zz + (k >> 2), y_ = 2 * yy + ((k >> 1) & 1), x_ = 2 * xx + (k & 1);
            s += __bfloat162float(x[((((long long)nn * D + z) * H + y_) * W + x_) * C + c]);
        }
        y[e] = __float2bfloat16(0.125f * s);
    }
}

__global__ void k_pool2_bwd(const bf16* __restrict__ dy, int N, int D, int H, int W, int C, bf16* __restrict__ dx) {
    const long long n = (long long)N * D * H * W * C;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long t = e / C;
        const int x_ = (int)(t % W);
        t /= W;
        const int y_ = (int)(t % H);
        t /= H;
        const int z = (int)(t % D);
        const int nn = (int)(t / D);
        const long long src = ((((long long)nn * (D / 2) + z / 2) * (H / 2) + y_ / 2) * (W / 2) + x_ / 2) * C + c;
        dx[e] = __float2bfloat16(0.125f * __bfloat162float(dy[src]));
    }
}

__global__ void k_up2(const bf16* __restrict__ x, int N, int D, int H, int W, int C, bf16* __restrict__ y) {
    const long long n = (long long)N * 8 * D * H * W * C;
    const int D2 = 2 * D, H2 = 2 * H, W2 = 2 * W;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long t = e / C;
        const int x_ = (int)(t % W2);
        t /= W2;
        const int y_ = (int)(t % H2);
        t /= H2;
        const int z = (int)(t % D2);
        const int nn = (int)(t / D2);
        y[e] = x[((((long long)nn * D + z / 2) * H + y_ / 2) * W + x_ / 2) * C + c];
    }
}

__global__ void k_up2_bwd(const bf16* __restrict__ dy, int N, int D, int H, int W, int C, bf16* __restrict__ dx) {
    const long long n = (long long)N * D * H * W * C;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long t = e / C;
        const int x_ = (int)(t % W);
        t /= W;
        const int y_ = (int)(t % H);
        t /= H;
        const int z = (int)(t % D);
        const int nn = (int)(t / D);
        float s = 0.f;
        for (int k = 0; k < 8; k++) {
            const int zz = 2 * z + (k >> 2), yy = 2 * y_ + ((k >> 1) & 1), xx = 2 * x_ + (k & 1);
            s += __bfloat162float(dy[((((long long)nn * 2 * D + zz) * 2 * H + yy) * 2 * W + xx) * C + c]);
        }
        dx[e] = __float2bfloat16(s);
    }
}

__global__ void k_concat(const bf16* __restrict__ a, int ca, const bf16* __restrict__ b, int cb, size_t vox,
                         bf16* __restrict__ y) {
    const int c = ca + cb;
    const size_t n = vox * c;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t v = e / c;
        const int k = (int)(e - v * c);
        y[e] = k < ca ? a[v * ca + k] : b[v * cb + (k - ca)];
    }
}

__global__ void k_split(const bf16* __restrict__ y, int ca, int cb, size_t vox, bf16* __restrict__ a,
                        bf16* __restrict__ b) {
    const int c = ca + cb;
    const size_t n = vox * c;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t v = e / c;
        const int k = (int)(e - v * c);
        if (k < ca) {
            if (a) a[v * ca + k] = y[e];
        } else if (b) {
            b[v * cb + (k - ca)] = y[e];
        }
    }
}

__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ tgt, const uint8_t* __restrict__ mask,
                      size_t vox, int c, float inv_count, double* __restrict__ loss, bf16* __restrict__ dpred) {
    double s = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < vox * c; e += (size_t)gridDim.x * blockDim.x) {
        const size_t v = e / c;
        float d = 0.f;
        if (mask[v]) d = pred[e] - tgt[e];
        s += (double)d * d;
        dpred[e] = __float2bfloat16(2.f * d * inv_count);
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv_count);
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ pb, size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float gr = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gr;
        const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
        m[e] = mm;
        v[e] = vv;
        const float q = p[e] - lr * (mm * c1) / (sqrtf(vv * c2) + eps);
        p[e] = q;
        g[e] = 0.f;
        if (pb) pb[e] = __float2bfloat16(q);
    }
}

__global__ void k_add(const bf16* __restrict__ a, const bf16* __restrict__ b, size_t n, bf16* __restrict__ y) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] = __float2bfloat16(__bfloat162float(a[e]) + __bfloat162float(b[e]));
}

__global__ void k_mask_input(const uint8_t* __restrict__ mask, size_t vox, float value, bf16* __restrict__ x) {
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < vox; v += (size_t)gridDim.x * blockDim.x) {
        x[2 * v] = __float2bfloat16(mask[v] ? 1.f : 0.f);
        x[2 * v + 1] = __float2bfloat16(value);
    }
}

__global__ void k_fields_to_target(const double* __restrict__ rho, const double* __restrict__ u, size_t vox,
                                   double rho0, double inv_s_rho, double inv_s_u, float* __restrict__ t) {
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < vox; v += (size_t)gridDim.x * blockDim.x) {
        double r = rho[v];
        const bool ok = isfinite(r);
        t[4 * v] = ok ? (float)((r - rho0) * inv_s_rho) : 0.f;
        for (int c = 0; c < 3; c++) {
            const double uc = u[c * vox + v];
            t[4 * v + 1 + c] = ok && isfinite(uc) ? (float)(uc * inv_s_u) : 0.f;
        }
    }
}

__global__ void k_target_to_fields(const float* __restrict__ t, size_t vox, double rho0, double s_rho, double s_u,
                                   double* __restrict__ rho, double* __restrict__ u) {
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < vox; v += (size_t)gridDim.x * blockDim.x) {
        rho[v] = rho0 + s_rho * (double)t[4 * v];
        for (int c = 0; c < 3; c++) u[c * vox + v] = s_u * (double)t[4 * v + 1 + c];
    }
}

__global__ void k_f2b(const float* __restrict__ x, size_t n, bf16* __restrict__ y) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] = __float2bfloat16(x[e]);
}

__global__ void k_b2f(const bf16* __restrict__ x, size_t n, float* __restrict__ y) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] = __bfloat162float(x[e]);
}

static unsigned grid_for(size_t n) {
    const size_t b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? (b ? b : 1) : 4096);
}

static cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

static int check(cudaError_t e, const char* what) { return e == cudaSuccess ? LBM_OK : cuda_fail(e, what); }

}  // namespace nn
}  // namespace lbm

using namespace lbm;
using namespace lbm::nn;

// Output-channel tiling shared by the forward and weight-gradient GEMMs: the
// channels are split into equal tiles of at most 128, each a multiple of 8.
static int pick_nf(int cout, int* n_tiles) {
    const int tiles = (cout + 127) / 128;
    const int per = (cout + tiles - 1) / tiles;
    const int need = (per + 7) / 8;
    static const int sizes[] = {1, 2, 4, 6, 8, 12, 16};
    int nf = 16;
    for (int s : sizes)
        if (s >= need) {
            nf = s;
            break;
        }
    *n_tiles = (cout + nf * 8 - 1) / (nf * 8);
    return nf;
}

namespace lbm {
namespace nn {
int conv3d_halo(const void* x, int n, int d, int h, int w, int cin, const void* wgt, const float* bias, int cout,
                int relu, int wrap, void* y, float* y32, cudaStream_t s);
float* chunk_scratch(size_t floats);
int sum_chunks(const float* part, long long chunks, long long E, float* dst, cudaStream_t s);
int wgrad_tc(const void* x, const void* dy, int n, int d, int h, int w, int cin, int cout, int wrap, float* dw,
             cudaStream_t s);
}  // namespace nn
}  // namespace lbm

extern "C" int lbm_nn_conv3d(const void* x, int n, int d, int h, int w, int cin, const void* wgt,
                             const float* bias, int cout, int relu, int wrap, void* y, float* y32, void* stream) {
    if (!x || !wgt || n < 1 || d < 1 || h < 1 || w < 1 || cin < 1 || cout < 1 || (!y && !y32) || (wrap & ~7))
        return fail(LBM_ERR_ARG, "lbm_nn_conv3d: bad arguments");
    // the tcgen05 halo-tile kernel where the shape allows (cin % 16 == 0,
    // cout % 16 == 0), else the mma.sync kernel below
    const int tc = conv3d_halo(x, n, d, h, w, cin, wgt, bias, cout, relu, wrap, y, y32, S(stream));
    if (tc != 1) return tc;
    const long long M = (long long)n * d * h * w;
    int ny = 0;
    const int nf = pick_nf(cout, &ny);
    const dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)ny);
    const bool vec = cin % 16 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    auto go = [&](auto kern) {
        kern<<<grid, 128, 0, S(stream)>>>(static_cast<const bf16*>(x), n, d, h, w, cin, static_cast<const bf16*>(wgt),
                                          bias, cout, relu, wrap, static_cast<bf16*>(y), y32);
    };
#define LBM_NN_CONV(NF_)                         \
    case NF_:                                   \
        if (vec) go(k_conv<NF_, true>);         \
        else go(k_conv<NF_, false>);            \
        break;
    switch (nf) {
        LBM_NN_CONV(1)
        LBM_NN_CONV(2)
        LBM_NN_CONV(4)
        LBM_NN_CONV(6)
        LBM_NN_CONV(8)
        LBM_NN_CONV(12)
        LBM_NN_CONV(16)
    }
#undef LBM_NN_CONV
    return check(cudaGetLastError(), "k_conv launch");
}

extern "C" int lbm_nn_weight_flip(const void* wgt, int cin, int cout, void* wt, void* stream) {
    if (!wgt || !wt || cin < 1 || cout < 1) return fail(LBM_ERR_ARG, "lbm_nn_weight_flip: bad arguments");
    k_weight_flip<<<grid_for(27ull * cin * cout), 256, 0, S(stream)>>>(static_cast<const bf16*>(wgt), cin, cout,
                                                                       static_cast<bf16*>(wt));
    return check(cudaGetLastError(), "k_weight_flip launch");
}

extern "C" int lbm_nn_conv3d_wgrad(const void* x, const void* dy, int n, int d, int h, int w, int cin, int cout,
                                   int wrap, float* dw, float* dbias, void* stream) {
    if (!x || !dy || !dw || n < 1 || d < 1 || h < 1 || w < 1 || cin < 1 || cout < 1 || (wrap & ~7))
        return fail(LBM_ERR_ARG, "lbm_nn_conv3d_wgrad: bad arguments");
    // the tcgen05 GEMMs over packed operands where the shape allows, else the
    // gather kernel below; both leave per-chunk partial sums that are added in
    // chunk order (the result does not depend on the order blocks finish in)
    int rc = wgrad_tc(x, dy, n, d, h, w, cin, cout, wrap, dw, S(stream));
    const long long M = (long long)n * d * h * w;
    if (rc == 1) {
        const int K = 27 * cin;
        const long long vpb = 8192;
        int nz = 0;
        const int nf = pick_nf(cout, &nz);
        const dim3 grid((unsigned)((K + BM - 1) / BM), (unsigned)((M + vpb - 1) / vpb), (unsigned)nz);
        float* part = chunk_scratch((size_t)grid.y * K * cout);
        if (!part) return fail(LBM_ERR_OOM, "weight-gradient partial sums");
        auto go = [&](auto kern) {
            kern<<<grid, 128, 0, S(stream)>>>(static_cast<const bf16*>(x), static_cast<const bf16*>(dy), n, d, h, w,
                                              cin, cout, wrap, part, vpb);
        };
        switch (nf) {
            case 1: go(k_wgrad<1>); break;
            case 2: go(k_wgrad<2>); break;
            case 4: go(k_wgrad<4>); break;
            case 6: go(k_wgrad<6>); break;
            case 8: go(k_wgrad<8>); break;
            case 12: go(k_wgrad<12>); break;
            default: go(k_wgrad<16>); break;
        }
        rc = check(cudaGetLastError(), "k_wgrad launch");
        if (!rc) rc = sum_chunks(part, grid.y, (long long)K * cout, dw, S(stream));
    }
    if (rc || !dbias) return rc;
    const long long rpb = 4096, nb = (M + rpb - 1) / rpb;
    float* part = chunk_scratch((size_t)nb * cout);  // the weight gradient's sums are already in dw
    if (!part) return fail(LBM_ERR_OOM, "bias-gradient partial sums");
    k_bias_grad<<<(unsigned)nb, 128, 0, S(stream)>>>(static_cast<const bf16*>(dy), M, cout, part, rpb);
    rc = check(cudaGetLastError(), "k_bias_grad launch");
    return rc ? rc : sum_chunks(part, nb, cout, dbias, S(stream));
}

extern "C" int lbm_nn_relu_mask(void* g, const void* act, size_t count, void* stream) {
    if (!g || !act) return fail(LBM_ERR_ARG, "lbm_nn_relu_mask: NULL");
    k_relu_mask<<<grid_for(count), 256, 0, S(stream)>>>(static_cast<bf16*>(g), static_cast<const bf16*>(act), count);
    return check(cudaGetLastError(), "k_relu_mask launch");
}

extern "C" int lbm_nn_pool2(const void* x, int n, int d, int h, int w, int c, void* y, void* stream) {
    if (!x || !y || (d | h | w) & 1) return fail(LBM_ERR_ARG, "lbm_nn_pool2: bad arguments");
    k_pool2<<<grid_for((size_t)n * d * h * w * c / 8), 256, 0, S(stream)>>>(static_cast<const bf16*>(x), n, d, h, w,
                                                                            c, static_cast<bf16*>(y));
    return check(cudaGetLastError(), "k_pool2 launch");
}

extern "C" int lbm_nn_pool2_bwd(const void* dy, int n, int d, int h, int w, int c, void* dx, void* stream) {
    if (!dy || !dx || (d | h | w) & 1) return fail(LBM_ERR_ARG, "lbm_nn_pool2_bwd: bad arguments");
    k_pool2_bwd<<<grid_for((size_t)n * d * h * w * c), 256, 0, S(stream)>>>(static_cast<const bf16*>(dy), n, d, h, w,
                                                                            c, static_cast<bf16*>(dx));
    return check(cudaGetLastError(), "k_pool2_bwd launch");
}

extern "C" int lbm_nn_up2(const void* x, int n, int d, int h, int w, int c, void* y, void* stream) {
    if (!x || !y) return fail(LBM_ERR_ARG, "lbm_nn_up2: NULL");
    k_up2<<<grid_for((size_t)n * 8 * d * h * w * c), 256, 0, S(stream)>>>(static_cast<const bf16*>(x), n, d, h, w, c,
                                                                           static_cast<bf16*>(y));
    return check(cudaGetLastError(), "k_up2 launch");
}

extern "C" int lbm_nn_up2_bwd(const void* dy, int n, int d, int h, int w, int c, void* dx, void* stream) {
    if (!dy || !dx) return fail(LBM_ERR_ARG, "lbm_nn_up2_bwd: NULL");
    k_up2_bwd<<<grid_for((size_t)n * d * h * w * c), 256, 0, S(stream)>>>(static_cast<const bf16*>(dy), n, d, h, w, c,
                                                                           static_cast<bf16*>(dx));
    return check(cudaGetLastError(), "k_up2_bwd launch");
}

extern "C" int lbm_nn_concat(const void* a, int ca, const void* b, int cb, size_t voxels, void* y, void* stream) {
    if (!a || !b || !y) return fail(LBM_ERR_ARG, "lbm_nn_concat: NULL");
    k_concat<<<grid_for(voxels * (ca + cb)), 256, 0, S(stream)>>>(static_cast<const bf16*>(a), ca,
                                                                 static_cast<const bf16*>(b), cb, voxels,
                                                                 static_cast<bf16*>(y));
    return check(cudaGetLastError(), "k_concat launch");
}

extern "C" int lbm_nn_split(const void* y, int ca, int cb, size_t voxels, void* a, void* b, void* stream) {
    if (!y) return fail(LBM_ERR_ARG, "lbm_nn_split: NULL");
    k_split<<<grid_for(voxels * (ca + cb)), 256, 0, S(stream)>>>(static_cast<const bf16*>(y), ca, cb, voxels,
                                                                static_cast<bf16*>(a), static_cast<bf16*>(b));
    return check(cudaGetLastError(), "k_split launch");
}

extern "C" int lbm_nn_mse(const float* pred, const float* target, const uint8_t* mask, size_t voxels, int c,
                          size_t count, double* loss, void* dpred, void* stream) {
    if (!pred || !target || !mask || !loss || !dpred || c < 1) return fail(LBM_ERR_ARG, "lbm_nn_mse: bad arguments");
    const float inv = count ? 1.f / ((float)count * c) : 0.f;
    LBM_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(double), S(stream)));
    k_mse<<<grid_for(voxels * c), 256, 0, S(stream)>>>(pred, target, mask, voxels, c, inv, loss,
                                                       static_cast<bf16*>(dpred));
    return check(cudaGetLastError(), "k_mse launch");
}

extern "C" int lbm_nn_adam(float* p, float* g, float* m, float* v, void* pb, size_t count, float lr, float beta1,
                           float beta2, float eps, int t, void* stream) {
    if (!p || !g || !m || !v || t < 1) return fail(LBM_ERR_ARG, "lbm_nn_adam: bad arguments");
    const float c1 = 1.f / (1.f - powf(beta1, (float)t)), c2 = 1.f / (1.f - powf(beta2, (float)t));
    k_adam<<<grid_for(count), 256, 0, S(stream)>>>(p, g, m, v, static_cast<bf16*>(pb), count, lr, beta1, beta2, eps,
                                                   c1, c2);
    return check(cudaGetLastError(), "k_adam launch");
}

extern "C" int lbm_nn_add(const void* a, const void* b, size_t count, void* y, void* stream) {
    if (!a || !b || !y) return fail(LBM_ERR_ARG, "lbm_nn_add: NULL");
    k_add<<<grid_for(count), 256, 0, S(stream)>>>(static_cast<const bf16*>(a), static_cast<const bf16*>(b), count,
                                                  static_cast<bf16*>(y));
    return check(cudaGetLastError(), "k_add launch");
}

extern "C" int lbm_nn_mask_input(const uint8_t* mask, size_t voxels, float value, void* x, void* stream) {
    if (!mask || !x) return fail(LBM_ERR_ARG, "lbm_nn_mask_input: NULL");
    k_mask_input<<<grid_for(voxels), 256, 0, S(stream)>>>(mask, voxels, value, static_cast<bf16*>(x));
    return check(cudaGetLastError(), "k_mask_input launch");
}

extern "C" int lbm_nn_fields_to_target(const double* rho, const double* u, size_t voxels, double rho0,
                                       double s_rho, double s_u, float* t, void* stream) {
    if (!rho || !u || !t || !(s_rho != 0.0) || !(s_u != 0.0))
        return fail(LBM_ERR_ARG, "lbm_nn_fields_to_target: bad arguments");
    k_fields_to_target<<<grid_for(voxels), 256, 0, S(stream)>>>(rho, u, voxels, rho0, 1.0 / s_rho, 1.0 / s_u, t);
    return check(cudaGetLastError(), "k_fields_to_target launch");
}

extern "C" int lbm_nn_target_to_fields(const float* t, size_t voxels, double rho0, double s_rho, double s_u,
                                       double* rho, double* u, void* stream) {
    if (!t || !rho || !u) return fail(LBM_ERR_ARG, "lbm_nn_target_to_fields: NULL");
    k_target_to_fields<<<grid_for(voxels), 256, 0, S(stream)>>>(t, voxels, rho0, s_rho, s_u, rho, u);
    return check(cudaGetLastError(), "k_target_to_fields launch");
}

extern "C" int lbm_nn_f32_to_bf16(const float* x, size_t count, void* y, void* stream) {
    if (!x || !y) return fail(LBM_ERR_ARG, "lbm_nn_f32_to_bf16: NULL");
    k_f2b<<<grid_for(count), 256, 0, S(stream)>>>(x, count, static_cast<bf16*>(y));
    return check(cudaGetLastError(), "k_f2b launch");
}

extern "C" int lbm_nn_bf16_to_f32(const void* x, size_t count, float* y, void* stream) {
    if (!x || !y) return fail(LBM_ERR_ARG, "lbm_nn_bf16_to_f32: NULL");
    k_b2f<<<grid_for(count), 256, 0, S(stream)>>>(static_cast<const bf16*>(x), count, y);
    return check(cudaGetLastError(), "k_b2f launch");
}

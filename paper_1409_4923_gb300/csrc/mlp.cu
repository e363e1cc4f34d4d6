// mlp.cu -- surrogate network: BF16 tensor-core GEMMs with fused epilogues,
// loss, Adam and the C ABI of include/sde_mlp.h.
//
// Every GEMM of the forward and backward pass is one templated kernel: a
// 64 x 64 output tile per 128-thread block, 32-deep K slices staged in shared
// memory, 2 x 2 warps of 32 x 32, mma.m16n8k16 BF16 x BF16 -> FP32 with
// fragments loaded by ldmatrix (transposed where the operand is stored the
// other way round).  Epilogues fuse the bias, SiLU and its derivative.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sde.h"
#include "sde_mlp.h"

cudaError_t sde_tc_forward(int M, const float* x, const float* maps, uint32_t log_mask,
                           const __nv_bfloat16* W1, const float* b1, const __nv_bfloat16* W2,
                           const float* b2, const __nv_bfloat16* W3, const float* b3,
                           const __nv_bfloat16* W4, const float* b4, __nv_bfloat16* h2, float* y,
                           int* error, int sm_count, cudaStream_t st);

namespace {

constexpr int kIn = SDE_MLP_IN, kInPad = 16, kH = SDE_MLP_HIDDEN, kOut = SDE_MLP_OUT, kOutPad = 8;
constexpr uint64_t kMaxBatch = 65536;
constexpr uint64_t kMaxForwardChunk = 1u << 20;
constexpr int kSplitRows = 256;        // batch rows per split of the weight-gradient GEMMs

// Offsets in the flat parameter vector.
constexpr size_t oW1 = 0, oB1 = oW1 + kH * kInPad, oW2 = oB1 + kH, oB2 = oW2 + kH * kH,
                 oW3 = oB2 + kH, oB3 = oW3 + kH * kH, oW4 = oB3 + kH, oB4 = oW4 + kOutPad * kH,
                 kNParams = oB4 + kOutPad;
static_assert(kNParams == SDE_MLP_NPARAMS, "parameter layout");

enum { EPI_F32 = 0, EPI_FWD_SILU = 1, EPI_FWD_LINEAR = 2, EPI_BWD_DSILU = 3 };

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16* A; int lda;
    const __nv_bfloat16* B; int ldb;
    float* C; int ldc;                  // EPI_F32 / EPI_FWD_LINEAR output, EPI_FWD_SILU pre-activation (may be null)
    __nv_bfloat16* O; int ldo;          // BF16 output (SiLU activation or back-propagated gradient)
    const float* bias;                  // EPI_FWD_*
    const float* H; int ldh;            // EPI_BWD_DSILU: pre-activation of the layer below
    int k_split;                        // rows of K per blockIdx.z (split-K), 0 = all
    size_t c_split_stride;              // elements between the outputs of consecutive splits
};

__device__ __forceinline__ float silu(float x) { return x / (1.0f + __expf(-x)); }
__device__ __forceinline__ float dsilu(float x)
{
    const float s = 1.0f / (1.0f + __expf(-x));
    return s * (1.0f + x * (1.0f - s));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int BM = 64, BN = 64, BK = 32;

// C tile (BM x BN) = op(A) op(B).  A_KM: A stored [K][M] (else [M][K]); B_KN:
// B stored [K][N] (else [N][K]).  Operands are loaded 8 BF16 at a time; rows
// or columns outside the matrix are zero-filled.
template <bool A_KM, bool B_KN, int EPI>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g)
{
    __shared__ __align__(16) __nv_bfloat16 sA[A_KM ? BK : BM][(A_KM ? BM : BK) + 8];
    __shared__ __align__(16) __nv_bfloat16 sB[B_KN ? BK : BN][(B_KN ? BN : BK) + 8];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    int kb = 0, ke = g.K;
    if (g.k_split > 0) {
        kb = blockIdx.z * g.k_split;
        ke = min(g.K, kb + g.k_split);
    }
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

    // ---- staging of A and B (2 x 16-byte chunks per thread each): the next
    // K tile is fetched into registers while the current one is multiplied
    uint4 va[2], ub[2];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int c = tid + 128 * j;
            va[j] = make_uint4(0u, 0u, 0u, 0u);
            ub[j] = make_uint4(0u, 0u, 0u, 0u);
            if (!A_KM) {
                const int r = c >> 2, col = (c & 3) * 8;
                const int gm = m0 + r, gk = k0 + col;
                if (gm < g.M && gk < ke) va[j] = *(const uint4*)(g.A + (size_t)gm * g.lda + gk);
            } else {
                const int r = c >> 3, col = (c & 7) * 8;
                const int gk = k0 + r, gm = m0 + col;
                if (gk < ke && gm < g.M) va[j] = *(const uint4*)(g.A + (size_t)gk * g.lda + gm);
            }
            if (!B_KN) {
                const int r = c >> 2, col = (c & 3) * 8;
                const int gn = n0 + r, gk = k0 + col;
                if (gn < g.N && gk < ke) ub[j] = *(const uint4*)(g.B + (size_t)gn * g.ldb + gk);
            } else {
                const int r = c >> 3, col = (c & 7) * 8;
                const int gk = k0 + r, gn = n0 + col;
                if (gk < ke && gn < g.N) ub[j] = *(const uint4*)(g.B + (size_t)gk * g.ldb + gn);
            }
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int c = tid + 128 * j;
            if (!A_KM) *(uint4*)&sA[c >> 2][(c & 3) * 8] = va[j];
            else *(uint4*)&sA[c >> 3][(c & 7) * 8] = va[j];
            if (!B_KN) *(uint4*)&sB[c >> 2][(c & 3) * 8] = ub[j];
            else *(uint4*)&sB[c >> 3][(c & 7) * 8] = ub[j];
        }
    };
    if (kb < ke) fetch(kb);
    for (int k0 = kb; k0 < ke; k0 += BK) {
        stash();
        __syncthreads();
        if (k0 + BK < ke) fetch(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int mb = wm + mt * 16;
                if (!A_KM) {
                    const int r = mb + (lane & 15), col = kk + (lane >> 4) * 8;
                    ldsm_x4(smem_u32(&sA[r][col]), af[mt][0], af[mt][1], af[mt][2], af[mt][3]);
                } else {
                    const int r = kk + (lane >> 4) * 8 + (lane & 7), col = mb + ((lane >> 3) & 1) * 8;
                    ldsm_x4_t(smem_u32(&sA[r][col]), af[mt][0], af[mt][1], af[mt][2], af[mt][3]);
                }
            }
            uint32_t bf[4][2];
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                const int nb = wn + np * 16;
                uint32_t r0, r1, r2, r3;
                if (!B_KN) {
                    const int r = nb + (lane >> 4) * 8 + (lane & 7), col = kk + ((lane >> 3) & 1) * 8;
                    ldsm_x4(smem_u32(&sB[r][col]), r0, r1, r2, r3);
                } else {
                    const int r = kk + ((lane >> 3) & 1) * 8 + (lane & 7), col = nb + (lane >> 4) * 8;
                    ldsm_x4_t(smem_u32(&sB[r][col]), r0, r1, r2, r3);
                }
                bf[np * 2][0] = r0; bf[np * 2][1] = r1;
                bf[np * 2 + 1][0] = r2; bf[np * 2 + 1][1] = r3;
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
        }
        __syncthreads();
    }

    // ---- epilogue: thread holds rows g, g+8 and columns 2t, 2t+1 of each 16 x 8 tile
    const int gi = lane >> 2, ti = lane & 3;
    float* C = g.C;
    if (EPI == EPI_F32 && g.k_split > 0) C += (size_t)blockIdx.z * g.c_split_stride;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm + mt * 16 + gi + h * 8;
                if (m >= g.M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int n = n0 + wn + nt * 8 + ti * 2 + e;
                    if (n >= g.N) continue;
                    float v = acc[mt][nt][h * 2 + e];
                    if (EPI == EPI_F32) {
                        C[(size_t)m * g.ldc + n] = v;
                    } else if (EPI == EPI_FWD_LINEAR) {
                        C[(size_t)m * g.ldc + n] = v + g.bias[n];
                    } else if (EPI == EPI_FWD_SILU) {
                        v += g.bias[n];
                        if (C) C[(size_t)m * g.ldc + n] = v;
                        g.O[(size_t)m * g.ldo + n] = __float2bfloat16_rn(silu(v));
                    } else {
                        v *= dsilu(g.H[(size_t)m * g.ldh + n]);
                        g.O[(size_t)m * g.ldo + n] = __float2bfloat16_rn(v);
                    }
                }
            }
}

template <bool A_KM, bool B_KN, int EPI>
cudaError_t gemm(const GemmArgs& a, int splits, cudaStream_t st)
{
    dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, splits > 0 ? splits : 1);
    gemm_bf16_kernel<A_KM, B_KN, EPI><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

// Raw inputs -> mapped BF16 inputs [Mp][16] (rows >= M and columns >= 7 zero).
__global__ void input_map_kernel(const float* __restrict__ x, uint64_t M, uint64_t Mp,
                                 const float* __restrict__ maps, uint32_t log_mask,
                                 __nv_bfloat16* __restrict__ X)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Mp * kInPad) return;
    const uint64_t m = i / kInPad;
    const int c = (int)(i % kInPad);
    float v = 0.0f;
    if (m < M && c < kIn) {
        float r = x[m * kIn + c];
        if (log_mask & (1u << c)) r = log10f(r);
        v = (r - maps[c]) * maps[kIn + c];
    }
    X[i] = __float2bfloat16_rn(v);
}

// Standardised outputs y' [Mp][8] -> y [M][2] in raw units.
__global__ void output_map_kernel(const float* __restrict__ yp, uint64_t M,
                                  const float* __restrict__ maps, float* __restrict__ y)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * kOut) return;
    const uint64_t m = i / kOut;
    const int o = (int)(i % kOut);
    y[i] = yp[m * kOutPad + o] * maps[2 * kIn + kOut + o] + maps[2 * kIn + o];
}

// Residual of the standardised outputs r = y' - t' for element i of the
// padded [Mp][kOutPad] output block (zero in the padding).
__device__ __forceinline__ float loss_residual(const float* __restrict__ yp, const float* __restrict__ t, uint64_t M,
                                               const float* __restrict__ maps, uint64_t i, bool& real)
{
    const uint64_t m = i / kOutPad;
    const int o = (int)(i % kOutPad);
    real = m < M && o < kOut;
    if (!real) return 0.0f;
    const float tp = (t[m * kOut + o] - maps[2 * kIn + o]) / maps[2 * kIn + kOut + o];
    return yp[m * kOutPad + o] - tp;
}

// The loss's gradient dY' = (y' - t') / M (BF16, padded columns zero), one
// thread per element: the start of back-propagation.
__global__ void dy_kernel(const float* __restrict__ yp, const float* __restrict__ t, uint64_t M, uint64_t Mp,
                          const float* __restrict__ maps, __nv_bfloat16* __restrict__ dY)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Mp * kOutPad) return;
    bool real;
    const float r = loss_residual(yp, t, M, maps, i, real);
    dY[i] = __float2bfloat16_rn(real ? r * (1.0f / (float)M) : 0.0f);
}

// Loss of the standardised outputs, sum over rows of 0.5 |y' - t'|^2 / M, in
// FP64.  One block; fixed-order reduction.  It runs beside back-propagation.
__global__ void __launch_bounds__(1024) loss_kernel(const float* __restrict__ yp, const float* __restrict__ t,
                                                    uint64_t M, uint64_t Mp, const float* __restrict__ maps,
                                                    float* __restrict__ loss_out, double* __restrict__ loss64)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (uint64_t i = threadIdx.x; i < Mp * kOutPad; i += blockDim.x) {
        bool real;
        const float r = loss_residual(yp, t, M, maps, i, real);
        if (real) s += 0.5 * (double)r * (double)r;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double L = red[0] / (double)M;
        if (loss_out) *loss_out = (float)L;
        if (loss64) *loss64 = L;
    }
}

// Sum of split-K partials (fixed order) into the gradient vector.
__global__ void split_reduce_kernel(const float* __restrict__ part, int splits, size_t n, float* __restrict__ out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * n + i];
    out[i] = s;
}

// Column sums of a BF16 [Mp][N] matrix (bias gradients).  A block of 32 x 8
// threads takes 32 columns: thread (c, r) sums rows r, r + 8, ... of column c
// in order, then the eight partials of each column are added in order of r.
constexpr int kColsumRows = 8;

__global__ void __launch_bounds__(32 * kColsumRows) colsum_kernel(const __nv_bfloat16* __restrict__ G, uint64_t Mp,
                                                                  int N, int ld, float* __restrict__ out)
{
    __shared__ float part[kColsumRows][32];
    const int c = threadIdx.x & 31, r = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + c;
    float s = 0.0f;
    if (n < N) {
#pragma unroll 8
        for (uint64_t m = (uint64_t)r; m < Mp; m += kColsumRows) s += __bfloat162float(G[m * ld + n]);
    }
    part[r][c] = s;
    __syncthreads();
    if (r == 0 && n < N) {
        float t = part[0][c];
#pragma unroll
        for (int q = 1; q < kColsumRows; ++q) t += part[q][c];
        out[n] = t;
    }
}

// Adam on the flat FP32 parameters; refreshes the BF16 copies.
__global__ void adam_kernel(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                            float* __restrict__ m1, float* __restrict__ m2, size_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float wi = w[i] - lr * (a * c1) / (sqrtf(b * c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
}

// ---- training loop on the device (sde_mlp_fit): one step is captured once as
// a CUDA graph and replayed; everything that changes between steps is read
// from FitState in device memory.

struct FitState {
    unsigned long long k;   // steps done
};

__device__ __forceinline__ uint32_t mix32(uint32_t h)
{
    h ^= h >> 16; h *= 0x7FEB352Du;
    h ^= h >> 15; h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h;
}

// Row of position `pos` in the shuffled order of an epoch: a four-round
// Feistel network keyed by (seed, epoch) permutes [0, 2^bits) (bits even,
// 2^bits >= N), and positions that land at or above N walk on along their
// cycle until they fall below N.  The walk ends because the cycle through pos
// returns to pos < N; 2^bits < 4N makes it short on average.  The result is a
// bijection of [0, N).
__device__ __forceinline__ uint32_t shuffle_row(uint32_t pos, uint32_t N, uint32_t bits,
                                                unsigned long long seed, unsigned long long epoch)
{
    const uint32_t half = bits >> 1, mask = (1u << half) - 1u;
    uint32_t key[4];
    unsigned long long z = seed * 0x9E3779B97F4A7C15ull + epoch * 0xD1B54A32D192ED03ull;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        z += 0x9E3779B97F4A7C15ull;
        unsigned long long y = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        y = (y ^ (y >> 27)) * 0x94D049BB133111EBull;
        key[r] = (uint32_t)(y ^ (y >> 31));
    }
    uint32_t x = pos;
    for (uint32_t it = 0; it <= (1u << bits); ++it) {
        uint32_t L = x >> half, R = x & mask;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t F = mix32(R ^ key[r]) & mask;
            const uint32_t nL = R;
            R = L ^ F;
            L = nL;
        }
        x = (L << half) | R;
        if (x < N) break;
    }
    return x;
}

// The step's minibatch: rows of positions [s batch, (s + 1) batch) of epoch
// k / per_epoch's order (s = k mod per_epoch), copied into xb, tb.
__global__ void fit_gather_kernel(const FitState* __restrict__ fs, const float* __restrict__ X,
                                  const float* __restrict__ T, uint32_t N, uint32_t batch, uint32_t per_epoch,
                                  uint32_t bits, unsigned long long seed, float* __restrict__ xb,
                                  float* __restrict__ tb)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    const unsigned long long k = fs->k;
    const uint32_t pos = (uint32_t)(k % per_epoch) * batch + i;
    const uint32_t row = shuffle_row(pos, N, bits, seed, k / per_epoch);
#pragma unroll
    for (int c = 0; c < kIn; ++c) xb[(size_t)i * kIn + c] = X[(size_t)row * kIn + c];
#pragma unroll
    for (int o = 0; o < kOut; ++o) tb[(size_t)i * kOut + o] = T[(size_t)row * kOut + o];
}

// Adam as adam_kernel with step k's learning rate and bias corrections from
// the table sched (lr, c1, c2 per step).
__global__ void adam_fit_kernel(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                                float* __restrict__ m1, float* __restrict__ m2, size_t n,
                                const FitState* __restrict__ fs, const float* __restrict__ sched, float b1,
                                float b2, float eps)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* sk = sched + 3ull * fs->k;
    const float lr = sk[0], c1 = sk[1], c2 = sk[2];
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float wi = w[i] - lr * (a * c1) / (sqrtf(b * c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
}

// Record the step's loss and advance the step counter.
__global__ void fit_end_kernel(FitState* fs, const float* __restrict__ loss, float* __restrict__ losses)
{
    if (losses) losses[fs->k] = *loss;
    fs->k += 1ull;
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

unsigned nblk(size_t n, unsigned t = 256) { return (unsigned)((n + t - 1) / t); }

// Flags of the surrogate-guided scan: predicted model error above tol,
// predicted Monte Carlo stderr above se_tol, or a sign change of the
// predicted <v> against a 4-neighbour.
__global__ void guided_flags_kernel(const float* __restrict__ v1, const float* __restrict__ v2,
                                    const float* __restrict__ lse, uint32_t nx, uint32_t ny, float kappa,
                                    float r0, float se_scale, float tol, float se_tol,
                                    uint8_t* __restrict__ flags, uint32_t* __restrict__ count)
{
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (uint64_t)nx * ny) return;
    const uint32_t i = (uint32_t)(p / ny), j = (uint32_t)(p % ny);
    const float v = 0.5f * (v1[p] + v2[p]);
    const float model_err = kappa * fabsf(v1[p] - v2[p]) + r0;
    const float se = se_scale * exp10f(lse[p]);
    bool f = !(model_err <= tol) || !(se <= se_tol);
    const bool neg = v < 0.0f;
    auto differs = [&](uint64_t q) { return ((0.5f * (v1[q] + v2[q])) < 0.0f) != neg; };
    if (i > 0 && differs(p - ny)) f = true;
    if (i + 1 < nx && differs(p + ny)) f = true;
    if (j > 0 && differs(p - 1)) f = true;
    if (j + 1 < ny && differs(p + 1)) f = true;
    flags[p] = f ? 1 : 0;
    const unsigned ballot = __ballot_sync(__activemask(), f);
    if (f && (threadIdx.x & 31u) == (uint32_t)(__ffs(ballot) - 1)) atomicAdd(count, (uint32_t)__popc(ballot));
}

}  // namespace

struct sde_mlp {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // back-propagation side branches: weight gradients (side[0]) and bias
    // gradients (side[1]) run beside the chain of back-propagation GEMMs
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t fork_ev = nullptr, join_ev[2] = {nullptr, nullptr};
    std::string err;
    float* w = nullptr;              // FP32 master parameters
    __nv_bfloat16* wb = nullptr;     // BF16 copies
    float* grad = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    float* maps = nullptr;           // shift[7], scale[7], out_shift[2], out_scale[2]
    uint32_t log_mask = 0;
    uint64_t step = 0;
    // activation workspace for up to cap rows
    uint64_t cap = 0;
    __nv_bfloat16* X = nullptr;      // [cap][16]
    float* H[3] = {nullptr, nullptr, nullptr};                 // [cap][256] pre-activations
    __nv_bfloat16* A[3] = {nullptr, nullptr, nullptr};         // [cap][256] activations
    float* Yp = nullptr;             // [cap][8]
    __nv_bfloat16* dY = nullptr;     // [cap][8]
    __nv_bfloat16* dH[3] = {nullptr, nullptr, nullptr};        // [cap][256]
    float* part = nullptr;           // split-K partials
    size_t part_elems = 0;
    double* loss64 = nullptr;
    double* host_loss = nullptr;
    int use_tc = 1;                  // forward pass on the fused tcgen05 kernels
    int sm_count = 0;
    int* tc_error = nullptr;         // device word set by a timed-out tensor-core wait
};

static std::string g_mlp_error;

static int mfail(sde_mlp* n, int code, const std::string& msg)
{
    if (n) n->err = msg; else g_mlp_error = msg;
    return code;
}

#define MLP_CUDA(n, call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) \
    return mfail((n), e_ == cudaErrorMemoryAllocation ? SDE_ENOMEM : SDE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); } while (0)

static void free_acts(sde_mlp* n)
{
    cudaFree(n->X); n->X = nullptr;
    for (int i = 0; i < 3; ++i) {
        cudaFree(n->H[i]); cudaFree(n->A[i]); cudaFree(n->dH[i]);
        n->H[i] = nullptr; n->A[i] = nullptr; n->dH[i] = nullptr;
    }
    cudaFree(n->Yp); cudaFree(n->dY); cudaFree(n->part);
    n->Yp = nullptr; n->dY = nullptr; n->part = nullptr;
    n->cap = 0;
    n->part_elems = 0;
}

static uint64_t pad64(uint64_t m) { return (m + 63u) & ~(uint64_t)63u; }

static int ensure_acts(sde_mlp* n, uint64_t Mp, bool train)
{
    if (Mp <= n->cap && (!train || n->dY)) return SDE_OK;
    cudaStreamSynchronize(n->stream);
    free_acts(n);
    const uint64_t c = Mp;
    MLP_CUDA(n, cudaMalloc(&n->X, c * kInPad * sizeof(__nv_bfloat16)));
    for (int i = 0; i < 3; ++i) {
        MLP_CUDA(n, cudaMalloc(&n->A[i], c * kH * sizeof(__nv_bfloat16)));
        if (train) {
            MLP_CUDA(n, cudaMalloc(&n->H[i], c * kH * sizeof(float)));
            MLP_CUDA(n, cudaMalloc(&n->dH[i], c * kH * sizeof(__nv_bfloat16)));
        }
    }
    MLP_CUDA(n, cudaMalloc(&n->Yp, c * kOutPad * sizeof(float)));
    if (train) {
        MLP_CUDA(n, cudaMalloc(&n->dY, c * kOutPad * sizeof(__nv_bfloat16)));
        const size_t splits = (c + kSplitRows - 1) / kSplitRows;
        n->part_elems = splits * (size_t)kH * kH;
        MLP_CUDA(n, cudaMalloc(&n->part, n->part_elems * sizeof(float)));
    }
    n->cap = c;
    return SDE_OK;
}

// Forward pass on Mp (padded) rows already mapped into n->X; standardised
// outputs into n->Yp.  store_pre: keep the pre-activations for the backward.
static cudaError_t forward_rows(sde_mlp* n, uint64_t Mp, bool store_pre)
{
    const int M = (int)Mp;
    GemmArgs a{};
    a.M = M; a.N = kH; a.K = kInPad; a.A = n->X; a.lda = kInPad; a.B = n->wb + oW1; a.ldb = kInPad;
    a.C = store_pre ? n->H[0] : nullptr; a.ldc = kH; a.O = n->A[0]; a.ldo = kH; a.bias = n->w + oB1;
    cudaError_t e = gemm<false, false, EPI_FWD_SILU>(a, 0, n->stream);
    for (int l = 1; l < 3 && e == cudaSuccess; ++l) {
        GemmArgs b{};
        b.M = M; b.N = kH; b.K = kH; b.A = n->A[l - 1]; b.lda = kH;
        b.B = n->wb + (l == 1 ? oW2 : oW3); b.ldb = kH;
        b.C = store_pre ? n->H[l] : nullptr; b.ldc = kH; b.O = n->A[l]; b.ldo = kH;
        b.bias = n->w + (l == 1 ? oB2 : oB3);
        e = gemm<false, false, EPI_FWD_SILU>(b, 0, n->stream);
    }
    if (e == cudaSuccess) {
        GemmArgs c{};
        c.M = M; c.N = kOutPad; c.K = kH; c.A = n->A[2]; c.lda = kH; c.B = n->wb + oW4; c.ldb = kH;
        c.C = n->Yp; c.ldc = kOutPad; c.bias = n->w + oB4;
        e = gemm<false, false, EPI_FWD_LINEAR>(c, 0, n->stream);
    }
    return e;
}

// Weight gradient dW[N][K] = dH^T X over Mp batch rows (split-K, fixed-order sum).
static cudaError_t weight_grad(sde_mlp* n, const __nv_bfloat16* dH, int ldh, int N,
                               const __nv_bfloat16* X, int ldx, int K, uint64_t Mp, float* out)
{
    const int splits = (int)((Mp + kSplitRows - 1) / kSplitRows);
    GemmArgs a{};
    a.M = N; a.N = K; a.K = (int)Mp; a.A = dH; a.lda = ldh; a.B = X; a.ldb = ldx;
    a.C = n->part; a.ldc = K; a.k_split = kSplitRows; a.c_split_stride = (size_t)N * K;
    cudaError_t e = gemm<true, true, EPI_F32>(a, splits, n->stream);
    if (e != cudaSuccess) return e;
    split_reduce_kernel<<<nblk((size_t)N * K), 256, 0, n->stream>>>(n->part, splits, (size_t)N * K, out);
    return cudaGetLastError();
}

// Loss and gradients (into n->grad) for a batch already in n->X (Mp rows).
// The side streams start after the work enqueued so far on the network's stream.
static cudaError_t fork_sides(sde_mlp* n)
{
    cudaError_t e = cudaEventRecord(n->fork_ev, n->stream);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(n->side[k], n->fork_ev, 0);
    return e;
}

static cudaError_t join_sides(sde_mlp* n)
{
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventRecord(n->join_ev[k], n->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(n->stream, n->join_ev[k], 0);
    }
    return e;
}

// dY, then per layer from the top: the gradient of the layer's output dH
// feeds three independent products: the weight gradient (split-K GEMM and
// its fixed-order reduction, in order on side[0], which owns the split-K
// buffer), the bias gradient (column sums, side[1]) and the back-propagation
// GEMM to the layer below (the critical path, on the network's stream).  The
// side streams join the network's stream before it returns; every product
// is the same as in one stream.
static cudaError_t backward_rows(sde_mlp* n, const float* t, uint64_t M, uint64_t Mp, float* loss_dev)
{
    dy_kernel<<<nblk(Mp * kOutPad), 256, 0, n->stream>>>(n->Yp, t, M, Mp, n->maps, n->dY);
    cudaError_t e = cudaGetLastError();
    // layer 4; the loss value itself on side[1], before the bias gradients
    if (e == cudaSuccess) e = fork_sides(n);
    if (e == cudaSuccess) {
        loss_kernel<<<1, 1024, 0, n->side[1]>>>(n->Yp, t, M, Mp, n->maps, loss_dev, n->loss64);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        cudaStream_t main = n->stream;
        n->stream = n->side[0];
        e = weight_grad(n, n->dY, kOutPad, kOutPad, n->A[2], kH, kH, Mp, n->grad + oW4);
        n->stream = main;
    }
    if (e == cudaSuccess) {
        colsum_kernel<<<1, 32 * kColsumRows, 0, n->side[1]>>>(n->dY, Mp, kOutPad, kOutPad, n->grad + oB4);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        GemmArgs a{};
        a.M = (int)Mp; a.N = kH; a.K = kOutPad; a.A = n->dY; a.lda = kOutPad; a.B = n->wb + oW4; a.ldb = kH;
        a.O = n->dH[2]; a.ldo = kH; a.H = n->H[2]; a.ldh = kH;
        e = gemm<false, true, EPI_BWD_DSILU>(a, 0, n->stream);
    }
    // layers 3, 2 (weights W3, W2) and the input layer
    const size_t oW[3] = {oW1, oW2, oW3}, oB[3] = {oB1, oB2, oB3};
    for (int l = 2; l >= 0 && e == cudaSuccess; --l) {
        const __nv_bfloat16* below = l == 0 ? n->X : n->A[l - 1];
        const int kin = l == 0 ? kInPad : kH;
        e = fork_sides(n);                      // dH[l] is complete
        if (e == cudaSuccess) {
            cudaStream_t main = n->stream;
            n->stream = n->side[0];
            e = weight_grad(n, n->dH[l], kH, kH, below, kin, kin, Mp, n->grad + oW[l]);
            n->stream = main;
        }
        if (e == cudaSuccess) {
            colsum_kernel<<<kH / 32, 32 * kColsumRows, 0, n->side[1]>>>(n->dH[l], Mp, kH, kH, n->grad + oB[l]);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && l > 0) {
            GemmArgs a{};
            a.M = (int)Mp; a.N = kH; a.K = kH; a.A = n->dH[l]; a.lda = kH; a.B = n->wb + oW[l]; a.ldb = kH;
            a.O = n->dH[l - 1]; a.ldo = kH; a.H = n->H[l - 1]; a.ldh = kH;
            e = gemm<false, true, EPI_BWD_DSILU>(a, 0, n->stream);
        }
    }
    const cudaError_t ej = join_sides(n);     // always: a capture needs its branches joined
    return e != cudaSuccess ? e : ej;
}

extern "C" {

const char* sde_mlp_last_error(const sde_mlp* n) { return n ? n->err.c_str() : g_mlp_error.c_str(); }

int sde_mlp_create(sde_mlp** out, uint64_t seed, void* cuda_stream)
{
    if (!out) return mfail(nullptr, SDE_EINVAL, "out is NULL");
    *out = nullptr;
    sde_mlp* n = new (std::nothrow) sde_mlp();
    if (!n) return mfail(nullptr, SDE_ENOMEM, "host allocation failed");
    cudaError_t e = cudaSuccess;
    if (cuda_stream == nullptr) {
        e = cudaStreamCreate(&n->stream);
        n->own_stream = e == cudaSuccess;
    } else {
        n->stream = (cudaStream_t)cuda_stream;
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&n->side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&n->fork_ev, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&n->join_ev[k], cudaEventDisableTiming);
    const size_t P = kNParams;
    if (e == cudaSuccess) e = cudaMalloc(&n->w, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->wb, P * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&n->grad, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->m1, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->m2, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->maps, 32 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->loss64, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&n->tc_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(n->tc_error, 0, sizeof(int));
    if (e == cudaSuccess) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->sm_count, cudaDevAttrMultiProcessorCount, dev);
    }
    if (e == cudaSuccess) e = cudaMallocHost(&n->host_loss, sizeof(double));
    if (e != cudaSuccess) {
        mfail(nullptr, SDE_ECUDA, std::string("sde_mlp_create: ") + cudaGetErrorString(e));
        sde_mlp_destroy(n);
        return SDE_ECUDA;
    }
    // Glorot-uniform weights from a splitmix64 stream, zero biases and padding
    std::vector<float> h(P, 0.0f);
    uint64_t s = seed ^ 0x5DEECE66DULL;
    auto next_u = [&s]() {
        s += 0x9E3779B97F4A7C15ULL;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](size_t off, int rows, int cols, int live_rows, int live_cols) {
        const double lim = std::sqrt(6.0 / (double)(live_rows + live_cols));
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c)
                h[off + (size_t)r * cols + c] =
                    (r < live_rows && c < live_cols) ? (float)((2.0 * next_u() - 1.0) * lim) : 0.0f;
    };
    fill(oW1, kH, kInPad, kH, kIn);
    fill(oW2, kH, kH, kH, kH);
    fill(oW3, kH, kH, kH, kH);
    fill(oW4, kOutPad, kH, kOut, kH);
    float maps[32] = {0};
    for (int i = 0; i < kIn; ++i) maps[kIn + i] = 1.0f;
    maps[2 * kIn + kOut] = maps[2 * kIn + kOut + 1] = 1.0f;
    e = cudaMemcpyAsync(n->maps, maps, sizeof(maps), cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    *out = n;
    if (e != cudaSuccess) return mfail(n, SDE_ECUDA, cudaGetErrorString(e));
    return sde_mlp_set_params(n, h.data());
}

int sde_mlp_set_maps(sde_mlp* n, const float* shift, const float* scale, uint32_t log_mask,
                     const float* out_shift, const float* out_scale)
{
    if (!n || !shift || !scale || !out_shift || !out_scale) return SDE_EINVAL;
    float maps[32] = {0};
    for (int i = 0; i < kIn; ++i) {
        if (!std::isfinite(shift[i]) || !std::isfinite(scale[i])) return mfail(n, SDE_EINVAL, "non-finite input map");
        maps[i] = shift[i];
        maps[kIn + i] = scale[i];
    }
    for (int o = 0; o < kOut; ++o) {
        if (!std::isfinite(out_shift[o]) || !(out_scale[o] != 0.0f) || !std::isfinite(out_scale[o]))
            return mfail(n, SDE_EINVAL, "bad output map");
        maps[2 * kIn + o] = out_shift[o];
        maps[2 * kIn + kOut + o] = out_scale[o];
    }
    if (log_mask >> kIn) return mfail(n, SDE_EINVAL, "log mask has bits beyond the 7 inputs");
    n->log_mask = log_mask;
    MLP_CUDA(n, cudaMemcpyAsync(n->maps, maps, sizeof(maps), cudaMemcpyHostToDevice, n->stream));
    MLP_CUDA(n, cudaStreamSynchronize(n->stream));
    return SDE_OK;
}

int sde_mlp_set_params(sde_mlp* n, const float* host)
{
    if (!n || !host) return SDE_EINVAL;
    const size_t P = kNParams;
    MLP_CUDA(n, cudaMemcpyAsync(n->w, host, P * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    to_bf16_kernel<<<nblk(P), 256, 0, n->stream>>>(n->w, n->wb, P);
    MLP_CUDA(n, cudaGetLastError());
    MLP_CUDA(n, cudaMemsetAsync(n->m1, 0, P * sizeof(float), n->stream));
    MLP_CUDA(n, cudaMemsetAsync(n->m2, 0, P * sizeof(float), n->stream));
    MLP_CUDA(n, cudaStreamSynchronize(n->stream));
    n->step = 0;
    return SDE_OK;
}

int sde_mlp_get_params(sde_mlp* n, float* host)
{
    if (!n || !host) return SDE_EINVAL;
    MLP_CUDA(n, cudaMemcpyAsync(host, n->w, kNParams * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    MLP_CUDA(n, cudaStreamSynchronize(n->stream));
    return SDE_OK;
}

int sde_mlp_forward(sde_mlp* n, const float* x, uint64_t M, float* y)
{
    if (!n || !x || !y || M == 0) return n ? mfail(n, SDE_EINVAL, "bad forward arguments") : SDE_EINVAL;
    // the tensor-core layers keep their weights resident per CTA: large chunks
    // amortise the weight loads
    const uint64_t chunk = n->use_tc ? kMaxForwardChunk : kMaxBatch;
    int rc = ensure_acts(n, pad64(M < chunk ? M : chunk), false);
    if (rc) return rc;
    for (uint64_t r0 = 0; r0 < M; r0 += chunk) {
        const uint64_t m = (M - r0) < chunk ? (M - r0) : chunk;
        const uint64_t Mp = pad64(m);
        if (n->use_tc) {
            // two fused tcgen05 kernels: maps and layers 1-2, layers 3-4 and the output map
            MLP_CUDA(n, sde_tc_forward((int)m, x + r0 * kIn, n->maps, n->log_mask, n->wb + oW1, n->w + oB1,
                                       n->wb + oW2, n->w + oB2, n->wb + oW3, n->w + oB3, n->wb + oW4,
                                       n->w + oB4, n->A[1], y + r0 * kOut, n->tc_error, n->sm_count,
                                       n->stream));
            continue;
        }
        input_map_kernel<<<nblk(Mp * kInPad), 256, 0, n->stream>>>(x + r0 * kIn, m, Mp, n->maps, n->log_mask, n->X);
        MLP_CUDA(n, cudaGetLastError());
        MLP_CUDA(n, forward_rows(n, Mp, false));
        output_map_kernel<<<nblk(m * kOut), 256, 0, n->stream>>>(n->Yp, m, n->maps, y + r0 * kOut);
        MLP_CUDA(n, cudaGetLastError());
    }
    return SDE_OK;
}

int sde_mlp_gradients(sde_mlp* n, const float* x, const float* t, uint64_t M, float* host_grad,
                      double* host_loss)
{
    if (!n || !x || !t || !host_grad || M == 0 || M > kMaxBatch)
        return n ? mfail(n, SDE_EINVAL, "bad gradient arguments (1 <= M <= 65536)") : SDE_EINVAL;
    const uint64_t Mp = pad64(M);
    int rc = ensure_acts(n, Mp, true);
    if (rc) return rc;
    MLP_CUDA(n, cudaMemsetAsync(n->grad, 0, kNParams * sizeof(float), n->stream));
    input_map_kernel<<<nblk(Mp * kInPad), 256, 0, n->stream>>>(x, M, Mp, n->maps, n->log_mask, n->X);
    MLP_CUDA(n, cudaGetLastError());
    MLP_CUDA(n, forward_rows(n, Mp, true));
    MLP_CUDA(n, backward_rows(n, t, M, Mp, nullptr));
    MLP_CUDA(n, cudaMemcpyAsync(host_grad, n->grad, kNParams * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    MLP_CUDA(n, cudaMemcpyAsync(n->host_loss, n->loss64, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    MLP_CUDA(n, cudaStreamSynchronize(n->stream));
    if (host_loss) *host_loss = *n->host_loss;
    return SDE_OK;
}

int sde_mlp_train_step(sde_mlp* n, const float* x, const float* t, uint64_t M, float lr, float beta1,
                       float beta2, float eps, float* loss_dev)
{
    if (!n || !x || !t || M == 0 || M > kMaxBatch)
        return n ? mfail(n, SDE_EINVAL, "bad train arguments (1 <= M <= 65536)") : SDE_EINVAL;
    if (!(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return mfail(n, SDE_EINVAL, "bad Adam hyper-parameters");
    const uint64_t Mp = pad64(M);
    int rc = ensure_acts(n, Mp, true);
    if (rc) return rc;
    input_map_kernel<<<nblk(Mp * kInPad), 256, 0, n->stream>>>(x, M, Mp, n->maps, n->log_mask, n->X);
    MLP_CUDA(n, cudaGetLastError());
    MLP_CUDA(n, forward_rows(n, Mp, true));
    MLP_CUDA(n, backward_rows(n, t, M, Mp, loss_dev));
    n->step += 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)n->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)n->step)));
    adam_kernel<<<nblk(kNParams), 256, 0, n->stream>>>(n->w, n->wb, n->grad, n->m1, n->m2, kNParams, lr, beta1,
                                                        beta2, eps, c1, c2);
    MLP_CUDA(n, cudaGetLastError());
    return SDE_OK;
}

// One training step on the device (gathered minibatch, forward, loss and
// gradients, Adam with step k's entry of sched), enqueued on n->stream.
static cudaError_t fit_step(sde_mlp* n, FitState* fs, const float* sched, const float* X, const float* T,
                            uint32_t N, uint32_t batch, uint32_t per_epoch, uint32_t bits, unsigned long long seed,
                            float beta1, float beta2, float eps, float* xb, float* tb, float* loss, float* losses)
{
    const uint64_t Mp = pad64(batch);
    fit_gather_kernel<<<nblk(batch), 256, 0, n->stream>>>(fs, X, T, N, batch, per_epoch, bits, seed, xb, tb);
    input_map_kernel<<<nblk(Mp * kInPad), 256, 0, n->stream>>>(xb, batch, Mp, n->maps, n->log_mask, n->X);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = forward_rows(n, Mp, true);
    if (e == cudaSuccess) e = backward_rows(n, tb, batch, Mp, loss);
    if (e != cudaSuccess) return e;
    adam_fit_kernel<<<nblk(kNParams), 256, 0, n->stream>>>(n->w, n->wb, n->grad, n->m1, n->m2, kNParams, fs, sched,
                                                            beta1, beta2, eps);
    fit_end_kernel<<<1, 1, 0, n->stream>>>(fs, loss, losses);
    return cudaGetLastError();
}

int sde_mlp_fit(sde_mlp* n, const float* X, const float* T, uint64_t N, uint64_t steps, uint32_t batch,
                float lr, float lr_final, float beta1, float beta2, float eps, uint64_t seed, float* losses)
{
    if (!n) return SDE_EINVAL;
    // the schedule table takes 12 bytes per step on the host and the device
    if (!X || !T || N == 0 || N > (1ull << 30) || steps == 0 || steps > (1ull << 22) || batch == 0 ||
        batch > kMaxBatch || batch > N)
        return mfail(n, SDE_EINVAL,
                     "bad fit arguments (1 <= batch <= min(N, 65536), N <= 2^30, 1 <= steps <= 2^22)");
    if (!(lr > 0.0f) || !(lr_final > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
        !(eps > 0.0f))
        return mfail(n, SDE_EINVAL, "bad Adam hyper-parameters");
    int rc = ensure_acts(n, pad64(batch), true);
    if (rc) return rc;
    uint32_t bits = 2;
    while ((1ull << bits) < N) bits += 2;
    const uint32_t per_epoch = (uint32_t)(N / batch);
    // per-step learning rate (half-cosine decay) and Adam's bias corrections,
    // in the arithmetic of sde_mlp_train_step
    std::vector<float> sched(3 * steps);
    const double pi = 3.14159265358979323846;
    for (uint64_t k = 0; k < steps; ++k) {
        const double frac = steps > 1 ? (double)k / (double)(steps - 1) : 0.0;
        sched[3 * k] = (float)((double)lr_final + 0.5 * ((double)lr - (double)lr_final) * (1.0 + std::cos(pi * frac)));
        const double t = (double)(n->step + k + 1);
        sched[3 * k + 1] = (float)(1.0 / (1.0 - std::pow((double)beta1, t)));
        sched[3 * k + 2] = (float)(1.0 / (1.0 - std::pow((double)beta2, t)));
    }
    // scratch: FitState, the step's loss, the gathered minibatch, the schedule
    const size_t off_x = 64, off_t = off_x + ((size_t)batch * kIn * 4 + 255) / 256 * 256;
    const size_t off_s = off_t + ((size_t)batch * kOut * 4 + 255) / 256 * 256;
    const size_t bytes = off_s + sched.size() * 4;
    char* scratch = nullptr;
    MLP_CUDA(n, cudaMalloc(&scratch, bytes));
    FitState* fs = (FitState*)scratch;
    float* loss = (float*)(scratch + 32);
    float* xb = (float*)(scratch + off_x);
    float* tb = (float*)(scratch + off_t);
    float* dsched = (float*)(scratch + off_s);
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const cudaStream_t user = n->stream;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, 64, user);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dsched, sched.data(), sched.size() * 4, cudaMemcpyHostToDevice, user);
    if (e == cudaSuccess) e = cudaEventRecord(ev, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        n->stream = cs;
        cudaError_t ec = fit_step(n, fs, dsched, X, T, (uint32_t)N, batch, per_epoch, bits, seed, beta1, beta2,
                                  eps, xb, tb, loss, losses);
        n->stream = user;
        e = cudaStreamEndCapture(cs, &graph);
        if (ec != cudaSuccess) e = ec;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    for (uint64_t k = 0; k < steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, cs);
    if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, ev, 0);
    const cudaError_t es = cs ? cudaStreamSynchronize(cs) : cudaSuccess;
    if (e == cudaSuccess) e = es;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
    const cudaError_t eu = cudaStreamSynchronize(user);     // the schedule upload used `sched`
    if (e == cudaSuccess) e = eu;
    cudaFree(scratch);
    MLP_CUDA(n, e);
    n->step += steps;
    return SDE_OK;
}

int sde_mlp_gemm_bf16(sde_mlp* n, int a_layout, int b_layout, uint32_t M, uint32_t N, uint32_t K,
                      const void* A, uint32_t lda, const void* B, uint32_t ldb, float* C, uint32_t ldc)
{
    if (!n || !A || !B || !C || M == 0 || N == 0 || K == 0) return SDE_EINVAL;
    if ((lda | ldb) & 7u || ((uintptr_t)A | (uintptr_t)B) & 15u)
        return mfail(n, SDE_EINVAL, "operands need 16-byte aligned rows (leading dimensions % 8 == 0)");
    if ((a_layout == 0 && K % 8) || (a_layout == 1 && M % 8) || (b_layout == 0 && K % 8) || (b_layout == 1 && N % 8))
        return mfail(n, SDE_EINVAL, "the contiguous dimension of each operand must be a multiple of 8");
    GemmArgs g{};
    g.M = (int)M; g.N = (int)N; g.K = (int)K;
    g.A = (const __nv_bfloat16*)A; g.lda = (int)lda; g.B = (const __nv_bfloat16*)B; g.ldb = (int)ldb;
    g.C = C; g.ldc = (int)ldc;
    cudaError_t e;
    if (a_layout == 0 && b_layout == 0) e = gemm<false, false, EPI_F32>(g, 0, n->stream);
    else if (a_layout == 0 && b_layout == 1) e = gemm<false, true, EPI_F32>(g, 0, n->stream);
    else if (a_layout == 1 && b_layout == 1) e = gemm<true, true, EPI_F32>(g, 0, n->stream);
    else if (a_layout == 1 && b_layout == 0) e = gemm<true, false, EPI_F32>(g, 0, n->stream);
    else return mfail(n, SDE_EINVAL, "layout must be 0 or 1");
    MLP_CUDA(n, e);
    MLP_CUDA(n, cudaStreamSynchronize(n->stream));
    return SDE_OK;
}

int sde_mlp_set_tensor_path(sde_mlp* n, int use_tcgen05)
{
    if (!n || (use_tcgen05 != 0 && use_tcgen05 != 1)) return SDE_EINVAL;
    n->use_tc = use_tcgen05;
    return SDE_OK;
}

int sde_mlp_sync(sde_mlp* n)
{
    if (!n) return SDE_EINVAL;
    MLP_CUDA(n, cudaStreamSynchronize(n->stream));
    int err = 0;
    MLP_CUDA(n, cudaMemcpy(&err, n->tc_error, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) return mfail(n, SDE_ETIMEDOUT, "a tensor-core completion wait ran out (mbarrier not signalled)");
    return SDE_OK;
}

int sde_guided_flags(sde_mlp* n, const float* v1, const float* v2, const float* lse, uint32_t nx,
                     uint32_t ny, float kappa, float r0, float se_scale, float tol, float se_tol, uint8_t* flags,
                     uint32_t* count)
{
    if (!n || !v1 || !v2 || !lse || !flags || !count || nx == 0 || ny == 0) return SDE_EINVAL;
    const uint64_t total = (uint64_t)nx * ny;
    guided_flags_kernel<<<nblk(total), 256, 0, n->stream>>>(v1, v2, lse, nx, ny, kappa, r0, se_scale, tol,
                                                            se_tol, flags, count);
    MLP_CUDA(n, cudaGetLastError());
    return SDE_OK;
}

void sde_mlp_destroy(sde_mlp* n)
{
    if (!n) return;
    if (n->stream || n->own_stream) cudaStreamSynchronize(n->stream);
    free_acts(n);
    cudaFree(n->w); cudaFree(n->wb); cudaFree(n->grad); cudaFree(n->m1); cudaFree(n->m2);
    cudaFree(n->maps); cudaFree(n->loss64); cudaFree(n->tc_error);
    if (n->host_loss) cudaFreeHost(n->host_loss);
    for (int k = 0; k < 2; ++k) {
        if (n->side[k]) cudaStreamDestroy(n->side[k]);
        if (n->join_ev[k]) cudaEventDestroy(n->join_ev[k]);
    }
    if (n->fork_ev) cudaEventDestroy(n->fork_ev);
    if (n->own_stream) cudaStreamDestroy(n->stream);
    delete n;
}

}  // extern "C"

// mlp_tc.cu -- 256 x 256 layers of the surrogate network on the fifth-generation
// tensor cores (tcgen05): out[M][256] = SiLU(A[M][256] W^T + b) in BF16.
//
// One persistent CTA of 256 threads per SM.  The CTA copies W (256 x 256 BF16,
// 128 KB) into shared memory once, in the 128-byte-swizzled K-major layout the
// tensor core reads, and then walks 128-row tiles of A: the tile is staged in
// the same layout (64 KB, cp.async), one elected thread issues the 16 MMAs of
// K = 256 (tcgen05.mma kind::f16, M = 128, N = 256, FP32 accumulator in TMEM)
// and commits them to an mbarrier, and each warp reads 32 TMEM lanes (32 rows)
// of one half of the columns back with tcgen05.ld for the bias + SiLU
// epilogue (a warp may read the lane quarter of its index modulo 4).  As soon as the
// MMAs of a tile complete, the copy of the next tile starts, so it overlaps
// the epilogue.
//
// Every wait is bounded: if an mbarrier phase does not complete within the
// iteration limit the kernel records an error word, stops, releases its TMEM
// and returns.
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sde_tc {

constexpr int kRows = 128;            // MMA M: rows of A per tile
constexpr int kN = 256;               // MMA N: output features
constexpr int kK = 256;               // reduction length
constexpr int kKBlock = 64;           // BF16 elements per 128-byte swizzle row
constexpr int kKBlocks = kK / kKBlock;
constexpr int kBRegion = kN * 128;    // bytes of one K-block of W   (32 KB)
constexpr int kARegion = kRows * 128; // bytes of one K-block of A   (16 KB)
constexpr int kBBytes = kKBlocks * kBRegion;   // 128 KB
constexpr int kABytes = kKBlocks * kARegion;   //  64 KB
constexpr int kThreads = 256;        // 8 warps: warp w reads TMEM lanes 32 (w % 4) .., column half w / 4
constexpr int kSmemBytes = kBBytes + kABytes + 64 + kN * 4 + 1024;   // + barrier, TMEM slot, bias, alignment
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of the 16-byte chunk c (elements 8c .. 8c+7 of a 64-element
// K-block) of row r in a 128-byte-swizzled K-major region.
__device__ __forceinline__ uint32_t sw128(uint32_t r, uint32_t c) { return r * 128u + ((c ^ (r & 7u)) << 4); }

// Shared-memory matrix descriptor: 128-byte swizzle, K-major, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

// Instruction descriptor: BF16 x BF16 -> FP32, A and B K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ float silu(float x) { return __fdividef(x, 1.0f + __expf(-x)); }

// Asynchronous copy of the 128-row A tile starting at row r0 into the swizzled
// layout (rows past M are zero-filled by a zero source size).
__device__ __forceinline__ void load_tile_async(const __nv_bfloat16* __restrict__ A, int M, int r0,
                                                uint32_t sA_a, uint32_t tid)
{
    for (uint32_t i = tid; i < (uint32_t)kRows * (kK / 8); i += (uint32_t)kThreads) {
        const uint32_t r = i / (kK / 8), c = i % (kK / 8);
        const bool in = r0 + (int)r < M;
        const __nv_bfloat16* src = A + (in ? (size_t)(r0 + r) * kK + c * 8u : 0);
        const uint32_t dst = sA_a + (c >> 3) * kARegion + sw128(r, c & 7u);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                     :: "r"(dst), "l"(src), "r"(in ? 16u : 0u) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t phase)
{
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(kThreads, 1) silu_layer_tc_kernel(const __nv_bfloat16* __restrict__ A, int M,
                                                               const __nv_bfloat16* __restrict__ W,
                                                               const float* __restrict__ bias,
                                                               __nv_bfloat16* __restrict__ out,
                                                               int* __restrict__ error)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t* base = smem_raw + pad;
    uint8_t* sB = base;
    uint8_t* sA = base + kBBytes;
    uint64_t* mbar = (uint64_t*)(base + kBBytes + kABytes);
    uint32_t* tslot = (uint32_t*)(base + kBBytes + kABytes + 16);
    float* sbias = (float*)(base + kBBytes + kABytes + 64);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t mbar_a = smem_addr(mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(tslot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar_a) : "memory");
    for (uint32_t i = tid; i < (uint32_t)kN; i += (uint32_t)kThreads) sbias[i] = bias[i];
    // W -> shared memory (256 rows x 32 chunks of 16 bytes)
    for (uint32_t i = tid; i < (uint32_t)kN * (kK / 8); i += (uint32_t)kThreads) {
        const uint32_t n = i / (kK / 8), c = i % (kK / 8);
        const uint4 v = *(const uint4*)(W + (size_t)n * kK + c * 8u);
        *(uint4*)(sB + (c >> 3) * kBRegion + sw128(n, c & 7u)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t sA_a = smem_addr(sA), sB_a = smem_addr(sB);

    uint32_t phase = 0;
    bool ok = true;
    const int tiles = (M + kRows - 1) / kRows;
    int t = blockIdx.x;
    if (t < tiles) load_tile_async(A, M, t * kRows, sA_a, tid);
    for (; t < tiles && ok; t += gridDim.x) {
        const int r0 = t * kRows;
        // the tile is in shared memory: make it visible to the tensor core
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
#pragma unroll
            for (uint32_t ks = 0; ks < (uint32_t)(kK / 16); ++ks) {
                const uint32_t kb = ks >> 2, off = (ks & 3u) * 32u;
                const uint64_t ad = sdesc(sA_a + kb * kARegion + off);
                const uint64_t bd = sdesc(sB_a + kb * kBRegion + off);
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             :: "r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(ks) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mbar_a) : "memory");
        }
        __syncwarp();
        const bool mine = wait_phase(mbar_a, phase);
        ok = __syncthreads_and(mine) != 0;          // one decision for the whole block
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the MMAs have read the tile: fetch the next one during the epilogue
        if (ok && t + (int)gridDim.x < tiles) load_tile_async(A, M, (t + gridDim.x) * kRows, sA_a, tid);
        if (ok) {
            const uint32_t quarter = warp & 3u, half = warp >> 2;
            const int row = r0 + (int)(quarter * 32u + lane);
            const uint32_t taddr = tmem + ((quarter * 32u) << 16);
#pragma unroll 1
            for (uint32_t cb = half * (kN / 2); cb < (half + 1u) * (kN / 2); cb += 32u) {
                uint32_t v[32];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                             "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                             "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                               "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                               "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                               "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                               "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                               "=r"(v[30]), "=r"(v[31])
                             : "r"(taddr + cb));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < M) {
                    uint32_t packed[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float a = silu(__uint_as_float(v[2 * j]) + sbias[cb + 2 * j]);
                        const float b = silu(__uint_as_float(v[2 * j + 1]) + sbias[cb + 2 * j + 1]);
                        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                        packed[j] = *(const uint32_t*)&h;
                    }
                    uint4* dst = (uint4*)(out + (size_t)row * kN + cb);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
                }
            }
        } else if (tid == 0) {
            atomicExch(error, 1);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace sde_tc

// Host launcher (used by mlp.cu): grid = min(tiles, SMs).
cudaError_t sde_tc_silu_layer(const __nv_bfloat16* A, int M, const __nv_bfloat16* W, const float* bias,
                              __nv_bfloat16* out, int* error, int sm_count, cudaStream_t st)
{
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(sde_tc::silu_layer_tc_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, sde_tc::kSmemBytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int tiles = (M + sde_tc::kRows - 1) / sde_tc::kRows;
    const int grid = tiles < sm_count ? tiles : sm_count;
    sde_tc::silu_layer_tc_kernel<<<grid, sde_tc::kThreads, sde_tc::kSmemBytes, st>>>(A, M, W, bias, out, error);
    return cudaGetLastError();
}

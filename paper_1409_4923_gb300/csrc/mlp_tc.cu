// mlp_tc.cu -- the surrogate network's forward pass on the fifth-generation
// tensor cores (tcgen05), in two fused kernels over 128-row tiles:
//
//   layers 1-2:  raw inputs -> input map -> layer 1 (7 -> 256, K = 16) ->
//                SiLU -> BF16 A tile in shared memory -> layer 2 (256 x 256) ->
//                SiLU -> BF16 activations h2 in global memory;
//   layers 3-4:  h2 tile (cp.async) -> layer 3 (256 x 256) -> SiLU -> BF16 ->
//                layer 4 (256 -> 2) -> output map -> outputs in raw units.
//
// The activations between layers 1 and 2 and between layers 3 and 4 never
// reach global memory: per row, the pass reads 28 bytes of inputs and
// writes and reads 512 bytes of h2 and writes 8 bytes of outputs, instead of
// the four layers' 3 KB.
//
// One persistent CTA of 512 threads (16 warps) per SM.  It copies its 256 x 256 layer's
// weights W (BF16, 128 KB) into shared memory once, in the 128-byte-swizzled
// K-major layout the tensor core reads.  Per tile, the A operand is staged in
// the same layout (64 KB) and one elected thread issues the 16 MMAs of K = 256
// (tcgen05.mma kind::f16, M = 128, N = 256, FP32 accumulator in tensor memory)
// and commits them to an mbarrier.  The accumulator alternates between two
// 256-column halves of tensor memory, so the MMAs of tile t + 1 run while
// the 16 warps drain tile t: warp w reads 32 TMEM lanes (32 rows, the lane
// quarter w mod 4 that it may access) of one quarter of the columns (w / 4)
// with tcgen05.ld.  Sixteen warps (four per scheduler) give the SFU-bound
// SiLU chains of the producer and the drain enough warps to hide latency.  Layer 1 (K = 16) runs in the A tile's producer on the legacy
// tensor-core path (mma.sync m16n8k16, one K step); layer 4 is a dot product
// in the epilogue.  Arithmetic is that of the layer-by-layer path (BF16
// weights and activations, FP32 accumulation and biases) except for the SiLU,
// evaluated through tanh (see silu below).
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
constexpr int kThreads = 512;        // 16 warps: warp w drains TMEM lanes 32 (w % 4) .., column quarter w / 4
constexpr int kColGroups = kThreads / 128;   // column groups of the epilogue (4 x 64 columns)
constexpr int kIn = 7, kOut = 2;
constexpr int kXStride = 24;          // BF16 per staged input / layer-1 weight row (48 bytes: no ldmatrix conflicts)
constexpr uint32_t kTmemCols = 512;   // two 256-column accumulators
constexpr uint32_t kWaitLimit = 1u << 26;

// Shared-memory map (offsets from the 1024-aligned base).
constexpr int kOffB = 0;
constexpr int kOffA = kOffB + kBBytes;
constexpr int kOffBar = kOffA + kABytes;                 // mbarrier (8 B) and TMEM slot (4 B)
constexpr int kOffBias = kOffBar + 64;                   // 256 FP32
constexpr int kOffX = kOffBias + kN * 4;                 // 128 x 24 BF16 inputs
constexpr int kOffW1 = kOffX + kRows * kXStride * 2;     // 256 x 24 BF16 layer-1 weights
constexpr int kOffB1 = kOffW1 + kN * kXStride * 2;       // 256 FP32
constexpr int kOffW4 = kOffB1 + kN * 4;                  // 2 x 256 FP32 layer-4 weights
constexpr int kOffPart = kOffW4 + kOut * kN * 4;         // 4 x 128 x 2 FP32 partial outputs per column group
constexpr int kOffMaps = kOffPart + kColGroups * kRows * kOut * 4;   // 32 FP32 maps, then b4
constexpr int kSmemBytes = kOffMaps + 64 * 4 + 1024;     // + alignment slack
static_assert(kSmemBytes <= 227 * 1024, "shared memory");

enum { kProLoad = 0, kProLayer1 = 1 };    // A tile: copied from global, or computed from raw inputs
enum { kEpiStore = 0, kEpiOutput = 1 };   // drain: BF16 activations, or layer 4 and the output map

struct TcArgs {
    int M;
    const float* x;                  // kProLayer1: raw inputs [M][7]
    const float* maps;               // input shift[7], scale[7], output shift[2], scale[2]
    uint32_t log_mask;               // inputs mapped through log10
    const __nv_bfloat16* W1;         // kProLayer1: [256][16] BF16
    const float* b1;
    const __nv_bfloat16* A;          // kProLoad: activations [M][256] BF16
    const __nv_bfloat16* W;          // this layer: [256 out][256 in] BF16
    const float* b;
    __nv_bfloat16* out;              // kEpiStore: activations [M][256] BF16
    const __nv_bfloat16* W4;         // kEpiOutput: [8][256] BF16 (rows 0, 1 used)
    const float* b4;
    float* y;                        // kEpiOutput: outputs [M][2] in raw units
    int* error;
};

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

// SiLU(x) = x sigma(x) = h + h tanh(h) with h = x / 2: one SFU operation
// (tanh.approx, relative error below 2^-10, under the BF16 rounding that
// follows) instead of an exponential and a reciprocal.  The epilogues are
// bound by the SFU: 32768 activations per tile.
__device__ __forceinline__ float silu(float x)
{
    const float h = 0.5f * x;
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *(const uint32_t*)&h;
}

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

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Input map and layer 1 of the 128 rows from r0, written as SiLU(x W1^T + b1)
// in BF16 into the swizzled A tile.  Threads 0..127 map one row each into
// sX; then warp w computes rows 16 (w mod 8) .. + 15 of 128 columns (w / 8
// selects the half) with mma.sync (K = 16: the 7 inputs and zero padding),
// 64 columns (one K-block of the A tile) at a time.  The accumulator fragment holds rows g, g + 8
// and columns 2 t, 2 t + 1 of each 8-column tile: as a BF16 pair it is one
// 4-byte store, and the swizzle spreads the warp's 32 stores over all banks.
// Raw inputs of row r0 + tid (threads 0..127), loaded a tile ahead of their
// use so that the global-load latency overlaps the MMA wait and the epilogue.
__device__ __forceinline__ void prefetch_inputs(const TcArgs& g, int r0, uint32_t tid, float (&xr)[kIn])
{
#pragma unroll
    for (int c = 0; c < kIn; ++c) xr[c] = 0.0f;
    const int row = r0 + (int)tid;
    if (tid < (uint32_t)kRows && row < g.M) {
#pragma unroll
        for (int c = 0; c < kIn; ++c) xr[c] = g.x[(size_t)row * kIn + c];
    }
}

__device__ __forceinline__ void layer1_tile(const TcArgs& g, int r0, uint8_t* base, uint32_t tid,
                                            const float (&xr)[kIn])
{
    __nv_bfloat16* sX = (__nv_bfloat16*)(base + kOffX);
    const float* smaps = (const float*)(base + kOffMaps);
    if (tid < (uint32_t)kRows) {
        const int row = r0 + (int)tid;
        float v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = 0.0f;
        if (row < g.M) {
#pragma unroll
            for (int c = 0; c < kIn; ++c) {
                float r = xr[c];
                if ((g.log_mask >> c) & 1u) r = log10f(r);
                v[c] = __fmul_rn(r - smaps[c], smaps[kIn + c]);
            }
        }
        uint4* dst = (uint4*)(sX + tid * kXStride);
        dst[0] = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                            pack_bf16x2(v[6], v[7]));
        dst[1] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    const uint32_t warp = tid >> 5, lane = tid & 31u;
    const uint32_t wrow = (warp & 7u) * 16u;          // 16 rows
    const uint32_t kb0 = (warp >> 3) * 2u;            // and two K-blocks (128 columns) per warp
    uint32_t af[4];
    ldsm_x4(smem_addr(sX + (wrow + (lane & 15u)) * kXStride + (lane >> 4) * 8u), af[0], af[1], af[2], af[3]);
    const __nv_bfloat16* sW1 = (const __nv_bfloat16*)(base + kOffW1);
    const float* sb1 = (const float*)(base + kOffB1);
    uint8_t* sA = base + kOffA;
    const uint32_t gi = lane >> 2, ti = lane & 3u;
#pragma unroll 1
    for (uint32_t kb = kb0; kb < kb0 + 2u; ++kb) {
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
#pragma unroll
        for (uint32_t np = 0; np < 4u; ++np) {
            const uint32_t nb = kb * 64u + np * 16u;
            uint32_t q0, q1, q2, q3;
            ldsm_x4(smem_addr(sW1 + (nb + (lane >> 4) * 8u + (lane & 7u)) * kXStride + ((lane >> 3) & 1u) * 8u),
                    q0, q1, q2, q3);
            mma_bf16(acc[2 * np], af, q0, q1);
            mma_bf16(acc[2 * np + 1], af, q2, q3);
        }
#pragma unroll
        for (uint32_t nt = 0; nt < 8u; ++nt) {
            const uint32_t col = kb * 64u + nt * 8u + 2u * ti;
#pragma unroll
            for (uint32_t h = 0; h < 2u; ++h) {
                const uint32_t rr = wrow + gi + 8u * h;
                const uint32_t word = pack_bf16x2(silu(acc[nt][2 * h] + sb1[col]),
                                                  silu(acc[nt][2 * h + 1] + sb1[col + 1]));
                *(uint32_t*)(sA + kb * kARegion + sw128(rr, nt) + 4u * ti) = word;
            }
        }
    }
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

template <int PRO, int EPI>
__global__ void __launch_bounds__(kThreads, 1) mlp_tc_kernel(const __grid_constant__ TcArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t* base = smem_raw + pad;
    uint8_t* sB = base + kOffB;
    uint64_t* mbar = (uint64_t*)(base + kOffBar);
    uint32_t* tslot = (uint32_t*)(base + kOffBar + 16);
    float* sbias = (float*)(base + kOffBias);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t mbar_a = smem_addr(mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(tslot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar_a) : "memory");
    for (uint32_t i = tid; i < (uint32_t)kN; i += (uint32_t)kThreads) sbias[i] = g.b[i];
    float* smaps = (float*)(base + kOffMaps);
    if (tid < 18u) smaps[tid] = g.maps[tid];
    if (PRO == kProLayer1) {
        __nv_bfloat16* sW1 = (__nv_bfloat16*)(base + kOffW1);
        float* sb1 = (float*)(base + kOffB1);
        for (uint32_t i = tid; i < (uint32_t)kN * 2u; i += (uint32_t)kThreads)   // 2 x 16 bytes per row
            *(uint4*)(sW1 + (i >> 1) * kXStride + (i & 1u) * 8u) = *(const uint4*)(g.W1 + (size_t)(i >> 1) * 16u + (i & 1u) * 8u);
        for (uint32_t i = tid; i < (uint32_t)kN; i += (uint32_t)kThreads) sb1[i] = g.b1[i];
    }
    if (EPI == kEpiOutput) {
        float* sW4 = (float*)(base + kOffW4);
        for (uint32_t i = tid; i < (uint32_t)(kOut * kN); i += (uint32_t)kThreads)
            sW4[i] = __bfloat162float(g.W4[i]);
        if (tid < (uint32_t)kOut) smaps[32 + tid] = g.b4[tid];
    }
    // W -> shared memory (256 rows x 32 chunks of 16 bytes)
    for (uint32_t i = tid; i < (uint32_t)kN * (kK / 8); i += (uint32_t)kThreads) {
        const uint32_t n = i / (kK / 8), c = i % (kK / 8);
        const uint4 v = *(const uint4*)(g.W + (size_t)n * kK + c * 8u);
        *(uint4*)(sB + (c >> 3) * kBRegion + sw128(n, c & 7u)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t sA_a = smem_addr(base + kOffA), sB_a = smem_addr(sB);

    // Stage the A tile of tile t (all threads) and issue its MMAs into the
    // accumulator half acc (one thread), committed to the mbarrier.
    float xr[kIn];                                   // kProLayer1: the next tile's raw inputs
    auto produce_and_issue = [&](int t, uint32_t acc) {
        if (PRO == kProLoad) {
            load_tile_async(g.A, g.M, t * kRows, sA_a, tid);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        } else {
            layer1_tile(g, t * kRows, base, tid, xr);
            prefetch_inputs(g, (t + (int)gridDim.x) * kRows, tid, xr);
        }
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
                             :: "r"(acc), "l"(ad), "l"(bd), "r"(kIdesc), "r"(ks) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mbar_a) : "memory");
        }
        __syncwarp();
    };

    const int tiles = (g.M + kRows - 1) / kRows;
    int t = blockIdx.x;
    uint32_t phase = 0, it = 0;
    if (PRO == kProLayer1) prefetch_inputs(g, t * kRows, tid, xr);
    if (t < tiles) produce_and_issue(t, tmem);
    for (; t < tiles; t += gridDim.x, ++it) {
        const bool mine = wait_phase(mbar_a, phase);
        const bool ok = __syncthreads_and(mine) != 0;          // one decision for the whole block
        if (!ok) {
            // record the failure, give the MMAs in flight one more bounded
            // wait, then release the tensor memory below
            if (tid == 0) atomicExch(g.error, 1);
            wait_phase(mbar_a, phase);
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the MMAs of tile t are complete and have read the A tile: stage the
        // next tile and start its MMAs in the other accumulator half, then drain t
        const int tn = t + (int)gridDim.x;
        if (tn < tiles) produce_and_issue(tn, tmem + 256u * ((it + 1u) & 1u));
        const uint32_t acc = tmem + 256u * (it & 1u);
        const uint32_t quarter = warp & 3u, group = warp >> 2;
        const uint32_t trow = quarter * 32u + lane;             // row within the tile
        const int row = t * kRows + (int)trow;
        const uint32_t taddr = acc + ((quarter * 32u) << 16);
        float p0 = 0.0f, p1 = 0.0f;
        const float* sW4 = (const float*)(base + kOffW4);
#pragma unroll 1
        for (uint32_t cb = group * (kN / kColGroups); cb < (group + 1u) * (kN / kColGroups); cb += 32u) {
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
            uint32_t packed[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
                packed[j] = pack_bf16x2(silu(__uint_as_float(v[2 * j]) + sbias[cb + 2 * j]),
                                        silu(__uint_as_float(v[2 * j + 1]) + sbias[cb + 2 * j + 1]));
            if (EPI == kEpiStore) {
                if (row < g.M) {
                    uint4* dst = (uint4*)(g.out + (size_t)row * kN + cb);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
                }
            } else {
                // layer 4 on the BF16 activations, FP32 accumulation
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const __nv_bfloat162 h = *(const __nv_bfloat162*)&packed[j];
                    const float h0 = __low2float(h), h1 = __high2float(h);
                    const uint32_t c = cb + 2u * (uint32_t)j;
                    p0 = fmaf(h1, sW4[c + 1], fmaf(h0, sW4[c], p0));
                    p1 = fmaf(h1, sW4[kN + c + 1], fmaf(h0, sW4[kN + c], p1));
                }
            }
        }
        if (EPI == kEpiOutput) {
            float* spart = (float*)(base + kOffPart);
            if (group != 0u) {
                spart[(group * kRows + trow) * 2u] = p0;
                spart[(group * kRows + trow) * 2u + 1u] = p1;
            }
            __syncthreads();
            if (group == 0u && row < g.M) {
                float y0 = p0, y1 = p1;
#pragma unroll
                for (uint32_t q = 1; q < (uint32_t)kColGroups; ++q) {   // fixed order
                    y0 += spart[(q * kRows + trow) * 2u];
                    y1 += spart[(q * kRows + trow) * 2u + 1u];
                }
                y0 += smaps[32];
                y1 += smaps[33];
                g.y[(size_t)row * kOut] = fmaf(y0, smaps[2 * kIn + kOut], smaps[2 * kIn]);
                g.y[(size_t)row * kOut + 1] = fmaf(y1, smaps[2 * kIn + kOut + 1], smaps[2 * kIn + 1]);
            }
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

template <int PRO, int EPI>
static cudaError_t launch_tc(const sde_tc::TcArgs& a, int sm_count, cudaStream_t st)
{
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(sde_tc::mlp_tc_kernel<PRO, EPI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, sde_tc::kSmemBytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int tiles = (a.M + sde_tc::kRows - 1) / sde_tc::kRows;
    const int grid = tiles < sm_count ? tiles : sm_count;
    sde_tc::mlp_tc_kernel<PRO, EPI><<<grid, sde_tc::kThreads, sde_tc::kSmemBytes, st>>>(a);
    return cudaGetLastError();
}

// Host launcher (used by mlp.cu): the forward pass of M rows of raw inputs x
// [M][7] to raw outputs y [M][2], with h2 [M][256] (BF16) as the one
// intermediate in global memory.  Weight pointers are the BF16 copies of the
// parameter vector; biases and maps are FP32.
cudaError_t sde_tc_forward(int M, const float* x, const float* maps, uint32_t log_mask,
                           const __nv_bfloat16* W1, const float* b1, const __nv_bfloat16* W2,
                           const float* b2, const __nv_bfloat16* W3, const float* b3,
                           const __nv_bfloat16* W4, const float* b4, __nv_bfloat16* h2, float* y,
                           int* error, int sm_count, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    sde_tc::TcArgs a{};
    a.M = M; a.x = x; a.maps = maps; a.log_mask = log_mask; a.W1 = W1; a.b1 = b1;
    a.W = W2; a.b = b2; a.out = h2; a.error = error;
    cudaError_t e = launch_tc<sde_tc::kProLayer1, sde_tc::kEpiStore>(a, sm_count, st);
    if (e != cudaSuccess) return e;
    sde_tc::TcArgs c{};
    c.M = M; c.maps = maps; c.A = h2; c.W = W3; c.b = b3; c.W4 = W4; c.b4 = b4; c.y = y; c.error = error;
    return launch_tc<sde_tc::kProLoad, sde_tc::kEpiOutput>(c, sm_count, st);
}

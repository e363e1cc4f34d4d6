// mlp_tc.cu -- the surrogate network's forward pass on the fifth-generation
// tensor cores (tcgen05), in two persistent, warp-specialised kernels over
// 128-row tiles:
//
//   layers 1-2:  raw inputs -> input map -> layer 1 (7 -> 256, K = 16) ->
//                SiLU -> BF16 A tile in shared memory -> layer 2 (256 x 256) ->
//                SiLU -> BF16 activations h2 in global memory;
//   layers 3-4:  h2 tile (TMA) -> layer 3 (256 x 256) -> SiLU -> BF16 ->
//                layer 4 (256 -> 2) -> output map -> outputs in raw units.
//
// Per row the pass reads 28 bytes of inputs, writes and reads 512 bytes of
// h2 and writes 8 bytes of outputs, instead of the four layers' 3 KB.
//
// Each CTA (one per SM) copies its 256 x 256 layer's weights W (BF16, 128 KB)
// into shared memory once, in the 128-byte-swizzled K-major layout the tensor
// core reads.  The A operand of a tile moves through a ring of 16 KB slots,
// one 64-column K-block per slot, so that the A tile of tile t + 1 is written
// while the tensor core still reads the last blocks of tile t:
//
//   producers  write K-block c of a tile into the next free slot (layers 1-2:
//              sixteen warps compute layer 1 with mma.sync and SiLU; layers
//              3-4: one thread loads the block of h2 by TMA), then arrive on
//              the slot's "full" mbarrier;
//   issuer     one thread waits for each block, issues its four MMAs (K = 16
//              each; kind::f16, M = 128, N = 256, FP32 accumulator in tensor
//              memory) and commits them to the slot's "empty" mbarrier; after
//              a tile's last block it commits to the accumulator's mbarrier;
//   drain      warps read the accumulator with tcgen05.ld (warp w reads the
//              TMEM lanes 32 (w mod 4) .. + 31 that it may access), add the
//              bias, apply SiLU and either store BF16 h2 (layers 1-2, through
//              a per-warp staging block and a TMA tensor store) or form layer
//              4's dot products and the outputs (layers 3-4).
//
// The accumulator alternates between two 256-column halves of tensor memory,
// so the MMAs of tile t + 1 run while tile t is drained.  The layers 3-4 grid
// is a programmatic dependent launch of the layers 1-2 grid: its CTAs load
// their weights as SMs free up and wait (griddepcontrol.wait) for the first
// grid before they read h2.  The arithmetic is
// that of the layer-by-layer path (BF16 weights and activations, FP32
// accumulation and biases) except for the SiLU, evaluated through tanh (see
// silu_hb).
//
// Every wait is bounded: if an mbarrier phase does not complete within the
// iteration limit the kernel records an error word, stops, waits for its
// copies and MMAs in flight, releases its tensor memory and returns.  A group
// of warps agrees on each wait's outcome with bar.red.and before it uses a
// named barrier, so that a timeout leaves no warp at a barrier.
#include <cstdint>

#include <cuda.h>
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
constexpr int kColGroups = 4;         // column groups of the layers 3-4 drain (4 x 64 columns)
constexpr int kIn = 7, kOut = 2;
constexpr int kXStride = 24;          // BF16 per staged input / layer-1 weight row (48 bytes: no ldmatrix conflicts)
constexpr uint32_t kTmemCols = 512;   // two 256-column accumulators
constexpr uint32_t kWaitLimit = 1u << 26;

struct TcArgs {
    int M;
    const float* x;                  // layers 1-2: raw inputs [M][7]
    const float* maps;               // input shift[7], scale[7], output shift[2], scale[2]
    uint32_t log_mask;               // inputs mapped through log10
    const __nv_bfloat16* W1;         // layers 1-2: [256][16] BF16
    const float* b1;
    const __nv_bfloat16* A;          // layers 3-4: activations h2 [M][256] BF16
    const __nv_bfloat16* W;          // this kernel's 256 x 256 layer: [256 out][256 in] BF16
    const float* b;
    __nv_bfloat16* out;              // layers 1-2: activations h2 [M][256] BF16
    const __nv_bfloat16* W4;         // layers 3-4: [8][256] BF16 (rows 0, 1 used)
    const float* b4;
    float* y;                        // layers 3-4: outputs [M][2] in raw units
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
// follows) instead of an exponential and a reciprocal.  With x = acc + b and
// the half bias hb = b / 2 held in shared memory, h = fma(acc, 1/2, hb) is
// one rounding of (acc + b) / 2, which equals the rounded sum halved
// (halving is exact away from subnormals).
__device__ __forceinline__ float silu_hb(float acc, float hb)
{
    const float h = fmaf(acc, 0.5f, hb);
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

// Four 8 x 8 BF16 matrices to shared memory: lane l gives the address of row
// l mod 8 of matrix l / 8, and register m holds the element pair (row l / 4,
// columns 2 (l mod 4), + 1) of matrix m, as in an mma.sync accumulator.
__device__ __forceinline__ void stsm_x4(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3)
{
    asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1, %2, %3, %4};"
                 :: "r"(addr), "r"(r0), "r"(r1), "r"(r2), "r"(r3) : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *(const uint32_t*)&h;
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

// Raw inputs of row r0 + lane (lanes 0..15), loaded a tile ahead of their
// use so that the global-load latency overlaps the tile's work.
__device__ __forceinline__ void prefetch_inputs(const TcArgs& g, int r0, uint32_t lane, float (&xr)[kIn])
{
#pragma unroll
    for (int c = 0; c < kIn; ++c) xr[c] = 0.0f;
    const int row = r0 + (int)lane;
    if (lane < 16u && row < g.M) {
#pragma unroll
        for (int c = 0; c < kIn; ++c) xr[c] = g.x[(size_t)row * kIn + c];
    }
}

// 32 TMEM lanes x 16 columns (32-bit) from taddr into v; complete after
// tmem_wait16 on the same registers.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr));
}

// Waits for this thread's tensor-memory loads; the registers of the last one
// are operands, so that no use of them moves above the wait.
__device__ __forceinline__ void tmem_wait16(uint32_t (&v)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
                 :: "memory");
}

// Waits for the completion of the mbarrier phase with parity `phase`, for at
// most kWaitLimit polls; false on timeout.
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

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}

// Arrives on the mbarrier when every MMA this thread issued so far is complete.
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}

// Named barrier `id` over `count` threads that returns the AND of their `ok`.
__device__ __forceinline__ bool group_agree(bool ok, uint32_t id, uint32_t count)
{
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n"
                 " selp.u32 %0, 1, 0, q;\n}" : "=r"(r) : "r"((uint32_t)ok), "r"(id), "r"(count) : "memory");
    return r != 0u;
}

__device__ __forceinline__ void group_sync(uint32_t id, uint32_t count)
{
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(count) : "memory");
}

// mbarriers of both kernels: full[slot], empty[slot], accumulator full[b],
// accumulator empty[b], and the issuer's last commit.
enum { kBarFull = 0, kBarEmpty = 6, kBarAccFull = 12, kBarAccEmpty = 14, kBarDone = 16 };

constexpr int kL12Threads = 800;      // warps 0-7 drain, 8-23 produce, 24 issues the MMAs
constexpr int kL12Drain = 256;
constexpr int kL12ChunkArrivals = 256;   // the 8 producer warps of one K-block
constexpr int kL12Slots = 3;          // A ring: three 16 KB K-block slots, cycled across tiles
constexpr int kL12OffB = 0;
constexpr int kL12OffA = kBBytes;
constexpr int kL12OffStage = kL12OffA + kL12Slots * kARegion;    // 8 drain warps x 2 KB (32 rows x 32 columns)
constexpr int kL12OffBar = kL12OffStage + (kL12Drain / 32) * 2048;
constexpr int kL12OffTslot = kL12OffBar + 192;             // after the 17 mbarriers
constexpr int kL12OffBias = kL12OffBar + 256;
constexpr int kL12OffX = kL12OffBias + kN * 4;                   // 16 producer warps x 16 x 24 BF16
constexpr int kL12OffW1 = kL12OffX + 16 * 16 * kXStride * 2;      // 256 x 24 BF16
constexpr int kL12OffB1 = kL12OffW1 + kN * kXStride * 2;
constexpr int kL12OffMaps = kL12OffB1 + kN * 4;
constexpr int kL12SmemBytes = kL12OffMaps + 64 * 4 + 1024;
static_assert(kL12SmemBytes <= 227 * 1024, "shared memory");

// ---------------------------------------------------------------------------
// Input map and layers 1-2.  Warps 8-23 produce the A tile: warp w computes
// rows 16 ((w - 8) mod 8) .. + 15 of the K-blocks 2 ((w - 8) / 8) and that
// plus one (layer 1 on mma.sync, one K step over the 7 inputs and zero
// padding; each warp maps its own 16 input rows), SiLU, BF16, written by
// stmatrix into the block's slot of a ring of three slots cycled across
// tiles.  Warp 24 issues the MMAs.  Warps 0-7 drain (warp w: lane quarter
// w mod 4, column half w / 4; each 16-column load issued before the previous
// step's arithmetic) and write h2 32 x 32 at a time through a 2 KB staging
// block in the 64-byte swizzle, which a TMA tensor store copies to global
// memory (one 16-byte store per lane and row would touch 32 cache lines per
// instruction).
__global__ void __launch_bounds__(kL12Threads, 1) mlp_tc_layers12_kernel(const __grid_constant__ TcArgs g,
                                                                       const __grid_constant__ CUtensorMap tmH)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t* base = smem_raw + pad;
    uint8_t* sB = base + kL12OffB;
    uint8_t* sA = base + kL12OffA;
    const uint32_t bar0 = smem_addr(base + kL12OffBar);
    uint32_t* tslot = (uint32_t*)(base + kL12OffTslot);
    float* sbias = (float*)(base + kL12OffBias);
    __nv_bfloat16* sW1 = (__nv_bfloat16*)(base + kL12OffW1);
    float* sb1 = (float*)(base + kL12OffB1);
    float* smaps = (float*)(base + kL12OffMaps);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(tslot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (uint32_t c = 0; c < (uint32_t)kL12Slots; ++c) {
            mbar_init(bar0 + 8u * (kBarFull + c), (uint32_t)kL12ChunkArrivals);
            mbar_init(bar0 + 8u * (kBarEmpty + c), 1u);
        }
        for (uint32_t b = 0; b < 2u; ++b) {
            mbar_init(bar0 + 8u * (kBarAccFull + b), 1u);
            mbar_init(bar0 + 8u * (kBarAccEmpty + b), (uint32_t)(kL12Drain / 32));
        }
        mbar_init(bar0 + 8u * kBarDone, 1u);
    }
    for (uint32_t i = tid; i < (uint32_t)kN; i += (uint32_t)kL12Threads) sbias[i] = 0.5f * g.b[i];   // half biases
    if (tid < 18u) smaps[tid] = g.maps[tid];
    for (uint32_t i = tid; i < (uint32_t)kN * 2u; i += (uint32_t)kL12Threads)   // 2 x 16 bytes per row
        *(uint4*)(sW1 + (i >> 1) * kXStride + (i & 1u) * 8u) = *(const uint4*)(g.W1 + (size_t)(i >> 1) * 16u + (i & 1u) * 8u);
    for (uint32_t i = tid; i < (uint32_t)kN; i += (uint32_t)kL12Threads) sb1[i] = 0.5f * g.b1[i];
    for (uint32_t i = tid; i < (uint32_t)kN * (kK / 8); i += (uint32_t)kL12Threads) {
        const uint32_t n = i / (kK / 8), c = i % (kK / 8);
        const uint4 v = *(const uint4*)(g.W + (size_t)n * kK + c * 8u);
        *(uint4*)(sB + (c >> 3) * kBRegion + sw128(n, c & 7u)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // the layers 3-4 grid may start its prologue as SMs free up
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint32_t sA_a = smem_addr(sA), sB_a = smem_addr(sB);
    const int tiles = (g.M + kRows - 1) / kRows;
    const int ntile = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    bool ok = true;

    if (warp >= 8u && warp < 24u) {
        // producers: input map, then layer 1 one K-block at a time; warp pw
        // computes rows 16 (pw mod 8) .. + 15 of K-blocks 2 (pw / 8) and 2 (pw / 8) + 1,
        // mapping its own 16 input rows (lanes 0-15) into its own 16-row block
        // of sX, so that the producers need no barrier among themselves
        const uint32_t pw = warp - 8u;
        const uint32_t wrow = (pw & 7u) * 16u, kb0 = (pw >> 3) * 2u;
        const uint32_t ti = lane & 3u;
        __nv_bfloat16* sX = (__nv_bfloat16*)(base + kL12OffX) + pw * (16u * kXStride);
        float xr[kIn];
        prefetch_inputs(g, (int)blockIdx.x * kRows + (int)wrow, lane, xr);
        for (int i = 0; i < ntile && ok; ++i) {
            const int r0 = ((int)blockIdx.x + i * (int)gridDim.x) * kRows;
            if (lane < 16u) {
                const int row = r0 + (int)wrow + (int)lane;
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
                uint4* dst = (uint4*)(sX + lane * kXStride);
                dst[0] = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                                    pack_bf16x2(v[6], v[7]));
                dst[1] = make_uint4(0u, 0u, 0u, 0u);
            }
            __syncwarp();
            uint32_t af[4];
            ldsm_x4(smem_addr(sX + (lane & 15u) * kXStride + (lane >> 4) * 8u), af[0], af[1], af[2], af[3]);
            __syncwarp();
            prefetch_inputs(g, r0 + (int)gridDim.x * kRows + (int)wrow, lane, xr);
#pragma unroll 1
            for (uint32_t kb = kb0; kb < kb0 + 2u; ++kb) {
                if (!ok) break;
                const uint32_t k = (uint32_t)i * (uint32_t)kKBlocks + kb;   // chunk index in this block's stream
                const uint32_t slot = k % (uint32_t)kL12Slots, use = k / (uint32_t)kL12Slots;
                if (use > 0u && !wait_phase(bar0 + 8u * (kBarEmpty + slot), (use - 1u) & 1u)) {
                    ok = false;
                    break;
                }
                float acc[8][4];
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[a][j] = 0.0f;
#pragma unroll
                for (uint32_t np = 0; np < 4u; ++np) {
                    const uint32_t nb = kb * 64u + np * 16u;
                    uint32_t q0, q1, q2, q3;
                    ldsm_x4(smem_addr(sW1 + (nb + (lane >> 4) * 8u + (lane & 7u)) * kXStride + ((lane >> 3) & 1u) * 8u),
                            q0, q1, q2, q3);
                    mma_bf16(acc[2 * np], af, q0, q1);
                    mma_bf16(acc[2 * np + 1], af, q2, q3);
                }
                // SiLU, BF16, and four stmatrix of two 8-column tiles each: matrix m
                // of an instruction is rows 8 (m & 1) .. + 7 of tile 2 p + (m >> 1),
                // and lane l gives the swizzled address of row l mod 8 of matrix l / 8
                const uint32_t srow = wrow + (lane & 7u) + 8u * ((lane >> 3) & 1u);
#pragma unroll
                for (uint32_t pp = 0; pp < 4u; ++pp) {
                    uint32_t wv[4];
#pragma unroll
                    for (uint32_t m = 0; m < 4u; ++m) {
                        const uint32_t nt = 2u * pp + (m >> 1), h = m & 1u;
                        const uint32_t col = kb * 64u + nt * 8u + 2u * ti;
                        wv[m] = pack_bf16x2(silu_hb(acc[nt][2 * h], sb1[col]), silu_hb(acc[nt][2 * h + 1], sb1[col + 1]));
                    }
                    stsm_x4(sA_a + slot * (uint32_t)kARegion + sw128(srow, 2u * pp + (lane >> 4)), wv[0], wv[1], wv[2], wv[3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar0 + 8u * (kBarFull + slot)) : "memory");
            }
        }
    } else if (warp == 24u) {
        // MMA issuer: block c of tile i once its 256 producer threads have arrived
        if (lane == 0) {
            for (int i = 0; i < ntile && ok; ++i) {
                const uint32_t b = (uint32_t)i & 1u;
                if (i >= 2 && !wait_phase(bar0 + 8u * (kBarAccEmpty + b), (uint32_t)((i >> 1) - 1) & 1u)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + 256u * b;
                for (uint32_t c = 0; c < (uint32_t)kKBlocks; ++c) {
                    const uint32_t k = (uint32_t)i * (uint32_t)kKBlocks + c;
                    const uint32_t slot = k % (uint32_t)kL12Slots, use = k / (uint32_t)kL12Slots;
                    if (!wait_phase(bar0 + 8u * (kBarFull + slot), use & 1u)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (uint32_t q = 0; q < 4u; ++q) {
                        const uint32_t ks = c * 4u + q;
                        const uint64_t ad = sdesc(sA_a + slot * (uint32_t)kARegion + q * 32u);
                        const uint64_t bd = sdesc(sB_a + c * (uint32_t)kBRegion + q * 32u);
                        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                     :: "r"(acc), "l"(ad), "l"(bd), "r"(kIdesc), "r"(ks) : "memory");
                    }
                    mma_commit(bar0 + 8u * (kBarEmpty + slot));
                }
                if (!ok) break;
                mma_commit(bar0 + 8u * (kBarAccFull + b));
            }
            mma_commit(bar0 + 8u * kBarDone);
            wait_phase(bar0 + 8u * kBarDone, 0u);
        }
        __syncwarp();
    } else if (warp < 8u) {
        // drain: warp w reads TMEM lanes 32 (w mod 4) .. and column half w / 4
        const uint32_t quarter = warp & 3u, half = warp >> 2;
        const uint32_t trow = quarter * 32u + lane;
        // this warp's staging block: 32 rows x 64 bytes in the 64-byte swizzle
        // (16-byte chunk j of row r at chunk j ^ ((r >> 1) & 3)), which the
        // tensor store reads back into rows of h2
        uint8_t* stage = base + kL12OffStage + warp * 2048u;
        const uint32_t stage_a = smem_addr(stage);
        for (int i = 0; i < ntile; ++i) {
            const uint32_t b = (uint32_t)i & 1u;
            // each drain warp decides alone: no named barrier follows
            if (!wait_phase(bar0 + 8u * (kBarAccFull + b), (uint32_t)(i >> 1) & 1u)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = ((int)blockIdx.x + i * (int)gridDim.x) * kRows + (int)trow;
            const uint32_t taddr = tmem + 256u * b + ((quarter * 32u) << 16);
            // the half's 128 columns in steps of 16, each step's load issued
            // before the previous step's arithmetic; a 32-column box per two steps
            const uint32_t c0 = half * (kN / 2);
            uint32_t va[16], vb[16];
            tmem_ld16(taddr + c0, va);
            tmem_wait16(va);
#pragma unroll
            for (uint32_t j = 0; j < 8u; ++j) {
                uint32_t (&cur)[16] = (j & 1u) ? vb : va;
                uint32_t (&nxt)[16] = (j & 1u) ? va : vb;
                if (j < 7u) tmem_ld16(taddr + c0 + 16u * (j + 1u), nxt);
                const uint32_t cb = c0 + 16u * j;
                uint32_t packed[8];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    packed[k] = pack_bf16x2(silu_hb(__uint_as_float(cur[2 * k]), sbias[cb + 2 * k]),
                                            silu_hb(__uint_as_float(cur[2 * k + 1]), sbias[cb + 2 * k + 1]));
                if ((j & 1u) == 0u) {
                    // the previous tensor store has read the staging block
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    __syncwarp();
                }
#pragma unroll
                for (uint32_t qq = 0; qq < 2u; ++qq) {
                    const uint32_t q = 2u * (j & 1u) + qq;
                    *(uint4*)(stage + lane * 64u + ((q ^ ((lane >> 1) & 3u)) << 4)) =
                        make_uint4(packed[4 * qq], packed[4 * qq + 1], packed[4 * qq + 2], packed[4 * qq + 3]);
                }
                if (j & 1u) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    // the box's first row; rows past M are not written, and a box wholly
                    // past M is not issued
                    const int y0 = row - (int)lane;
                    if (lane == 0 && y0 < g.M) {
                        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                                     :: "l"((uint64_t)&tmH), "r"((int)(cb - 16u)), "r"(y0), "r"(stage_a) : "memory");
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                }
                if (j < 7u) tmem_wait16(nxt);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];"
                             :: "r"(bar0 + 8u * (kBarAccEmpty + b)) : "memory");
        }
    }
    if (warp < 8u && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // h2 written
    if (!ok) atomicExch(g.error, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// Layers 3-4 and the output map.  Warp 16 loads K-block c of each h2 tile by
// TMA (128-byte swizzle, rows past M zero-filled) into slot c as soon as the
// MMAs of the previous tile that read slot c are complete; warp 17 issues a
// block's four MMAs as soon as its copy has landed; warps 0-15 drain (warp w:
// lane quarter w mod 4, column quarter w / 4), form layer 4's partial dot
// products and combine the four column groups in a fixed order.
constexpr int kL34Threads = 576;      // warps 0-15 drain, 16 loads, 17 issues the MMAs
constexpr int kL34Drain = 512;
constexpr int kL34Slots = 4;          // one tile's four K-blocks (a fifth slot measured no faster)
constexpr int kL34OffB = 0;
constexpr int kL34OffA = kBBytes;
constexpr int kL34OffBar = kL34OffA + kL34Slots * kARegion;       // 17 mbarriers
constexpr int kL34OffTslot = kL34OffBar + 192;
constexpr int kL34OffBias = kL34OffBar + 256;
constexpr int kL34OffW4 = kL34OffBias + kN * 4;
constexpr int kL34OffPart = kL34OffW4 + kOut * kN * 4;  // 2 tiles x 4 column groups x 128 rows x 2
constexpr int kL34OffMaps = kL34OffPart + 2 * kColGroups * kRows * kOut * 4;
constexpr int kL34SmemBytes = kL34OffMaps + 64 * 4 + 1024;
static_assert(kL34SmemBytes <= 227 * 1024, "shared memory");

__global__ void __launch_bounds__(kL34Threads, 1) mlp_tc_layers34_kernel(const __grid_constant__ TcArgs g,
                                                                      const __grid_constant__ CUtensorMap tmA)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t* base = smem_raw + pad;
    uint8_t* sB = base + kL34OffB;
    const uint32_t bar0 = smem_addr(base + kL34OffBar);
    uint32_t* tslot = (uint32_t*)(base + kL34OffTslot);
    float* sbias = (float*)(base + kL34OffBias);
    float* sW4 = (float*)(base + kL34OffW4);
    float* smaps = (float*)(base + kL34OffMaps);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(tslot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (uint32_t c = 0; c < (uint32_t)kKBlocks; ++c) {
            mbar_init(bar0 + 8u * (kBarFull + c), 1u);
            mbar_init(bar0 + 8u * (kBarEmpty + c), 1u);
        }
        for (uint32_t b = 0; b < 2u; ++b) {
            mbar_init(bar0 + 8u * (kBarAccFull + b), 1u);
            mbar_init(bar0 + 8u * (kBarAccEmpty + b), (uint32_t)(kL34Drain / 32));
        }
        mbar_init(bar0 + 8u * kBarDone, 1u);
    }
    for (uint32_t i = tid; i < (uint32_t)kN; i += (uint32_t)kL34Threads) sbias[i] = 0.5f * g.b[i];   // half biases
    if (tid < 18u) smaps[tid] = g.maps[tid];
    for (uint32_t i = tid; i < (uint32_t)(kOut * kN); i += (uint32_t)kL34Threads) sW4[i] = __bfloat162float(g.W4[i]);
    if (tid < (uint32_t)kOut) smaps[32 + tid] = g.b4[tid];
    for (uint32_t i = tid; i < (uint32_t)kN * (kK / 8); i += (uint32_t)kL34Threads) {
        const uint32_t n = i / (kK / 8), c = i % (kK / 8);
        const uint4 v = *(const uint4*)(g.W + (size_t)n * kK + c * 8u);
        *(uint4*)(sB + (c >> 3) * kBRegion + sw128(n, c & 7u)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // h2 is read only after the layers 1-2 grid has completed (programmatic
    // dependent launch: this prologue may overlap that grid's last tiles)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const uint32_t sA_a = smem_addr(base + kL34OffA), sB_a = smem_addr(sB);
    const int tiles = (g.M + kRows - 1) / kRows;
    const int ntile = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    bool ok = true;

    if (warp == 16) {
        // TMA producer: block c of each tile into slot c
        if (lane == 0) {
            uint32_t nreq[kKBlocks] = {0u, 0u, 0u, 0u};   // copies requested per slot
            for (int i = 0; i < ntile && ok; ++i) {
                const int r0 = ((int)blockIdx.x + i * (int)gridDim.x) * kRows;
                for (uint32_t c = 0; c < (uint32_t)kKBlocks; ++c) {
                    const uint32_t fb = bar0 + 8u * (kBarFull + c);
                    if (i > 0 && !wait_phase(bar0 + 8u * (kBarEmpty + c), (uint32_t)(i - 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                                 :: "r"(fb), "r"((uint32_t)kARegion) : "memory");
                    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3}], [%4];"
                                 :: "r"(sA_a + c * (uint32_t)kARegion), "l"((uint64_t)&tmA),
                                    "r"((int)c * kKBlock), "r"(r0), "r"(fb) : "memory");
                    ++nreq[c];
                }
            }
            // no copy may still be in flight when the block exits
            for (uint32_t c = 0; c < (uint32_t)kKBlocks; ++c)
                if (nreq[c] > 0u) wait_phase(bar0 + 8u * (kBarFull + c), (nreq[c] - 1u) & 1u);
        }
        __syncwarp();
    } else if (warp == 17) {
        // MMA issuer: block c of tile i as soon as it has landed
        if (lane == 0) {
            for (int i = 0; i < ntile && ok; ++i) {
                const uint32_t b = (uint32_t)i & 1u;
                if (i >= 2 && !wait_phase(bar0 + 8u * (kBarAccEmpty + b), (uint32_t)((i >> 1) - 1) & 1u)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + 256u * b;
                for (uint32_t c = 0; c < (uint32_t)kKBlocks; ++c) {
                    if (!wait_phase(bar0 + 8u * (kBarFull + c), (uint32_t)i & 1u)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (uint32_t q = 0; q < 4u; ++q) {
                        const uint32_t ks = c * 4u + q;
                        const uint64_t ad = sdesc(sA_a + c * (uint32_t)kARegion + q * 32u);
                        const uint64_t bd = sdesc(sB_a + c * (uint32_t)kBRegion + q * 32u);
                        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                     :: "r"(acc), "l"(ad), "l"(bd), "r"(kIdesc), "r"(ks) : "memory");
                    }
                    mma_commit(bar0 + 8u * (kBarEmpty + c));
                }
                if (!ok) break;
                mma_commit(bar0 + 8u * (kBarAccFull + b));
            }
            // every MMA of this thread completes before the tensor memory is released
            mma_commit(bar0 + 8u * kBarDone);
            wait_phase(bar0 + 8u * kBarDone, 0u);
        }
        __syncwarp();
    } else if (warp < 16u) {
        // drain: warp w reads TMEM lanes 32 (w mod 4) .. and column quarter w / 4
        const uint32_t quarter = warp & 3u, group = warp >> 2;
        const uint32_t trow = quarter * 32u + lane;
        float* spart = (float*)(base + kL34OffPart);
        for (int i = 0; i < ntile; ++i) {
            const uint32_t b = (uint32_t)i & 1u;
            const bool mine = wait_phase(bar0 + 8u * (kBarAccFull + b), (uint32_t)(i >> 1) & 1u);
            if (!group_agree(mine, 1u, (uint32_t)kL34Drain)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = ((int)blockIdx.x + i * (int)gridDim.x) * kRows + (int)trow;
            const uint32_t taddr = tmem + 256u * b + ((quarter * 32u) << 16);
            float p0 = 0.0f, p1 = 0.0f;
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
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const uint32_t w = pack_bf16x2(silu_hb(__uint_as_float(v[2 * j]), sbias[cb + 2 * j]),
                                                   silu_hb(__uint_as_float(v[2 * j + 1]), sbias[cb + 2 * j + 1]));
                    const __nv_bfloat162 h = *(const __nv_bfloat162*)&w;
                    const float h0 = __low2float(h), h1 = __high2float(h);
                    const uint32_t c = cb + 2u * (uint32_t)j;
                    p0 = fmaf(h1, sW4[c + 1], fmaf(h0, sW4[c], p0));
                    p1 = fmaf(h1, sW4[kN + c + 1], fmaf(h0, sW4[kN + c], p1));
                }
            }
            // this warp is done with the accumulator half
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];"
                             :: "r"(bar0 + 8u * (kBarAccEmpty + b)) : "memory");
            // layer-4 partials of column groups 1-3 to group 0, in a buffer per tile parity
            float* sp = spart + b * (uint32_t)(kColGroups * kRows * kOut);
            if (group != 0u) {
                sp[(group * kRows + trow) * 2u] = p0;
                sp[(group * kRows + trow) * 2u + 1u] = p1;
            }
            group_sync(1u, (uint32_t)kL34Drain);
            if (group == 0u && row < g.M) {
                float y0 = p0, y1 = p1;
#pragma unroll
                for (uint32_t q = 1; q < (uint32_t)kColGroups; ++q) {   // fixed order
                    y0 += sp[(q * kRows + trow) * 2u];
                    y1 += sp[(q * kRows + trow) * 2u + 1u];
                }
                y0 += smaps[32];
                y1 += smaps[33];
                g.y[(size_t)row * kOut] = fmaf(y0, smaps[2 * kIn + kOut], smaps[2 * kIn]);
                g.y[(size_t)row * kOut + 1] = fmaf(y1, smaps[2 * kIn + kOut + 1], smaps[2 * kIn + 1]);
            }
        }
    }
    if (!ok) atomicExch(g.error, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace sde_tc

// cuTensorMapEncodeTiled, looked up once through the runtime (no link to the
// driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn lookup_encode_tiled()
{
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return (EncodeTiledFn)p;
}

// Layers 3-4 over h2 [M][256] (BF16): the tensor map describes h2 as a
// 2-D tensor of M rows and 256 columns whose 128-row x 64-column boxes land
// in the 128-byte-swizzled K-major layout of the tensor core's A operand.
static cudaError_t launch_layers34(const sde_tc::TcArgs& a, int sm_count, cudaStream_t st)
{
    static const EncodeTiledFn encode = lookup_encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    // the attribute belongs to the current device: set it on every launch
    cudaError_t e = cudaFuncSetAttribute(sde_tc::mlp_tc_layers34_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sde_tc::kL34SmemBytes);
    if (e != cudaSuccess) return e;
    alignas(64) CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)sde_tc::kK, (cuuint64_t)a.M};
    const cuuint64_t strides[1] = {(cuuint64_t)sde_tc::kK * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)sde_tc::kKBlock, (cuuint32_t)sde_tc::kRows};
    const cuuint32_t estr[2] = {1u, 1u};
    if (encode(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)a.A, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const int tiles = (a.M + sde_tc::kRows - 1) / sde_tc::kRows;
    const int grid = tiles < sm_count ? tiles : sm_count;
    // programmatic dependent launch: the kernel waits for the layers 1-2 grid
    // (griddepcontrol.wait) before it reads h2
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)sde_tc::kL34Threads);
    cfg.dynamicSmemBytes = (size_t)sde_tc::kL34SmemBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sde_tc::mlp_tc_layers34_kernel, a, tm);
}

static cudaError_t launch_layers12(const sde_tc::TcArgs& a, int sm_count, cudaStream_t st)
{
    static const EncodeTiledFn encode = lookup_encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    // the attribute belongs to the current device: set it on every launch
    cudaError_t e = cudaFuncSetAttribute(sde_tc::mlp_tc_layers12_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sde_tc::kL12SmemBytes);
    if (e != cudaSuccess) return e;
    // h2 [M][256] BF16 written in 32 x 32 boxes from 64-byte-swizzled staging blocks
    alignas(64) CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)sde_tc::kN, (cuuint64_t)a.M};
    const cuuint64_t strides[1] = {(cuuint64_t)sde_tc::kN * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {32u, 32u};
    const cuuint32_t estr[2] = {1u, 1u};
    if (encode(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)a.out, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const int tiles = (a.M + sde_tc::kRows - 1) / sde_tc::kRows;
    const int grid = tiles < sm_count ? tiles : sm_count;
    sde_tc::mlp_tc_layers12_kernel<<<grid, sde_tc::kL12Threads, sde_tc::kL12SmemBytes, st>>>(a, tm);
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
    cudaError_t e = launch_layers12(a, sm_count, st);
    if (e != cudaSuccess) return e;
    sde_tc::TcArgs c{};
    c.M = M; c.maps = maps; c.A = h2; c.W = W3; c.b = b3; c.W4 = W4; c.b4 = b4; c.y = y; c.error = error;
    return launch_layers34(c, sm_count, st);
}

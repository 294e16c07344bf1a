// The per-voxel network of Sec. 2 (81 -> 50 -> 30 -> 1, ReLU, softplus) and
// its input gradient on the 5th-generation tensor cores (tcgen05).
//
// A tile is 128 voxels = the MMA M dimension = the 128 TMEM lanes. Operands are
// staged in shared memory in the canonical K-major, no-swizzle layout (8-row x
// 16-byte core matrices); accumulators live in TMEM and are read back with
// tcgen05.ld, one voxel per TMEM lane. Float32 accuracy comes from splitting
// every operand into a TF32 head and a TF32 tail (x = hi + lo) and issuing
// hi*hi + hi*lo + lo*hi per product (error ~2^-21 relative); nsplit = 1 uses
// hi*hi only (plain TF32).
//
// Forward per tile:   A1[128 x 88] (stencil inputs) x W1^T -> D1[128 x 64]
//                     relu(D1 + b1) -> A2[128 x 64] x W2^T -> D2[128 x 32]
//                     y = b3 + w3 . relu(D2 + b2), M = M_scale softplus(y)  (CUDA cores)
// Backward per tile (after the forward): g_a2 = w3 g_y [a2 > 0]
//                     A3 = g_a2[128 x 32] x W2 -> D3 = g_a1 (pre-mask) [128 x 64]
//                     A4 = g_a1 [a1 > 0] [128 x 64] x W1 -> D4 = g_v[128 x 96]
// The forward saves, per voxel, y and the ReLU masks of both hidden layers
// (16 bytes); the backward starts from them at layer 3 instead of recomputing
// layers 1-2 (halo, operand build, two MMA layers and their epilogues).
// The backward folds g_v (81 columns) over the stencil's z offset in
// registers, stages the 27 folded images in shared memory and sums them per
// target cell of the tile's box (the tile grown by one cell, 3 fields x 4 x 6 x
// 18), so a tile writes 1296 floats instead of 81 x 128; k_stencil_tiles adds
// the overlapping boxes of up to 8 tiles per cell in a fixed order.
//
// Both kernels are persistent (one CTA of 17 warps per SM) and warp-
// specialised: 16 warps build operands and read accumulators, lane 0 of the
// 17th issues the MMAs. The first layer's operand and accumulator (forward)
// and the backward's A3, D3 and D4 are double-buffered, so the tensor cores
// run the next tile's first MMA layer while the compute warps read this tile's
// accumulators.
//
// Every mbarrier wait is bounded; on timeout the block records an error flag,
// waits (bounded) for its MMAs, frees its TMEM and returns. The host reports
// the flag as PMR_ETIMEOUT and clears it.
#include <algorithm>
#include <climits>
#include <cstring>

#include "common.cuh"

namespace pmr {
namespace {

constexpr int NI = 81, H1 = 50, H2 = 30;
constexpr int OFF_B1 = H1 * NI, OFF_W2 = OFF_B1 + H1, OFF_B2 = OFF_W2 + H2 * H1, OFF_W3 = OFF_B2 + H2,
              OFF_B3 = OFF_W3 + H2;

constexpr int TM = 128;           // voxels per tile = MMA M = TMEM lanes
constexpr int N1 = 64;            // layer 1 (81 -> 50, padded)
constexpr int K2 = 64, N2 = 32;   // layer 2 (50 -> 30, padded)
constexpr int K3 = 32, NB3 = 64;  // backward layer 2: g_a2 -> g_a1 (B = W2)
constexpr int K4 = 64, NB4 = 96;  // backward layer 1: g_a1 -> g_v  (B = W1)
constexpr int NT = 512;           // threads per block (16 warps; 4 per TMEM lane quadrant)

// voxel tile 2 (x) x 4 (y) x 16 (z); row = (lx * 4 + ly) * 16 + lz
constexpr int TX = 2, TY = 4, TZ = 16, HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int HALO = 3 * HX * HY * HZ;

// TMEM columns of the forward: D1 buffers at COL_D1 and COL_D1 + 64, D2 at COL_D2
constexpr uint32_t COL_D1 = 0, COL_D2 = 128;

constexpr uint32_t VEC_MASS = 160;  // float offset of the mass-network weights in the vector block
constexpr uint32_t SZ_VEC = 1920;    // b1[64], b2[32], w3[32], b3[4], mass network[301]: 4 * 461 rounded to 128 B

// Layer 1 of the forward runs on z-line tiles: 128 voxels (x, y, z0 .. z0+127)
// of one line along z. Its operand image holds, for rows i = 0 .. ZR-1 (the
// voxel at z0 + i - 1, periodic), the K1Z = 32 columns k = c*9 + (ox+1)*3 +
// (oy+1) (27 used): the three fields on the 3x3 (x, y) neighbourhood of the
// line. A 16-byte K chunk is a column of ZR rows 16 bytes apart (8-row groups
// SBO = 128 B apart) and chunks sit ZLBO bytes apart, so every row sits 16
// bytes after the previous one and the operand for the neighbour offset oz is
// the same image read from row oz + 1: a descriptor that starts 16 (oz + 1)
// bytes in. Each input value is stored once, not once per stencil copy, and
// the 3x3x3 stencil becomes three K1Z-wide MMA groups, one per oz.
constexpr int ZR = TM + 2;             // image rows
constexpr uint32_t ZLBO = ZR * 16;     // K-chunk stride of the z-line image
constexpr int K1Z = 32;                // layer-1 K per z offset (27 used)

// Operand precision. BF = false: float32 split into TF32 head and tail parts
// (kind::tf32, K = 8 per instruction); BF = true: one bfloat16 part
// (kind::f16 with bf16 inputs and float32 accumulation, K = 16). Either way a
// k-step is 32 bytes of a row, so the layout below is the same in bytes.
//
// Byte offset of element (r, k) in an R-row, K-major, no-swizzle operand image:
// k-steps are sub-images of R*32 bytes; inside one, core matrix (row group r/8,
// 16-byte K chunk) sits at 256*(r/8) + 128*chunk. So the K-direction
// core-matrix stride (LBO) is 128 B and the 8-row-group stride (SBO) 256 B.
// Every access of one k-step stays inside its R*32-byte sub-image.
template <bool BF>
struct Lay {
    static constexpr int ES = BF ? 2 : 4;    // bytes per element
    static constexpr int KS = 32 / ES;       // K per instruction
    static constexpr int EC = 16 / ES;       // elements per 16-byte core-matrix row
    static constexpr int NP = BF ? 1 : 2;    // parts per operand (head, tail)
    __host__ __device__ static constexpr uint32_t off(int R, int r, int k) {
        return (uint32_t)((k / KS) * (R * 32) + (r >> 3) * 256 + ((k / EC) & 1) * 128 + (r & 7) * 16 + (k % EC) * ES);
    }
    static constexpr uint32_t bytes(int R, int K) { return (uint32_t)(R * K * ES); }
    // shared-memory map (bytes); weight images first, in the order of the global image
    static constexpr uint32_t SZ_B1 = 3 * bytes(N1, K1Z), SZ_B2 = bytes(N2, K2), SZ_B3 = bytes(NB3, K3),
                              SZ_B4 = bytes(NB4, K4);
    static constexpr uint32_t S_B1 = 0;
    static constexpr uint32_t S_B2 = S_B1 + NP * SZ_B1;
    static constexpr uint32_t S_VEC = S_B2 + NP * SZ_B2;
    static constexpr uint32_t S_B3 = S_VEC + SZ_VEC;  // backward only
    static constexpr uint32_t S_B4 = S_B3 + NP * SZ_B3;
    static constexpr uint32_t IMG_FWD = S_B3;         // bytes of the image the forward stages
    static constexpr uint32_t IMG_ALL = S_B4 + NP * SZ_B4;
    static_assert((S_B2 | S_VEC | S_B3 | S_B4) % 128 == 0, "128-byte aligned regions");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Shared-memory matrix descriptor: start >> 4, LBO = 128 B, SBO = 256 B,
// descriptor version 1 (bits 46-47), no swizzle, base offset 0.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// The same for the z-line image of layer 1: LBO = ZLBO (K chunks), SBO = 128 B
// (8-row groups), so rows are uniformly 16 bytes apart.
__device__ __forceinline__ uint64_t zdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(ZLBO >> 4) << 16) | ((uint64_t)(128u >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::tf32: D f32, A and B tf32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::f16 with bf16 A and B, D f32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Launch controls of the tensor-core kernels: the bound of every mbarrier wait
// (try_wait polls), and whether the issuing lane issues its MMAs. issue = 0 is
// the failure-detection test hook (pmr_test_stall_mma): nothing is ever in
// flight, every wait for an accumulator runs out, and the kernel takes its
// timeout path (error flag, TMEM freed, return).
struct TcCtl {
    uint32_t wait_limit;
    int issue;
};
constexpr uint32_t kWaitLimit = 1u << 22;      // normal launches
constexpr uint32_t kTestWaitLimit = 1u << 12;  // the stall hook

// bounded wait for the phase; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Store 4 consecutive K values of one row (a 16-byte core-matrix row) as hi and lo parts.
__device__ __forceinline__ void put4(unsigned char* Ahi, unsigned char* Alo, uint32_t off, float a, float b, float c,
                                     float d) {
    const float ha = tf32_hi(a), hb = tf32_hi(b), hc = tf32_hi(c), hd = tf32_hi(d);
    *reinterpret_cast<float4*>(Ahi + off) = make_float4(ha, hb, hc, hd);
    *reinterpret_cast<float4*>(Alo + off) = make_float4(a - ha, b - hb, c - hc, d - hd);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Store 8 consecutive K values of row r starting at k0 (k0 % 8 == 0) in the operand image(s).
template <bool BF>
__device__ __forceinline__ void put8(unsigned char* Ahi, unsigned char* Alo, int r, int k0, const float* v) {
    using L = Lay<BF>;
    if constexpr (BF) {
        *reinterpret_cast<uint4*>(Ahi + L::off(TM, r, k0)) =
            make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                       pack_bf16x2(v[6], v[7]));
    } else {
        put4(Ahi, Alo, L::off(TM, r, k0), v[0], v[1], v[2], v[3]);
        put4(Ahi, Alo, L::off(TM, r, k0 + 4), v[4], v[5], v[6], v[7]);
    }
}

__device__ __forceinline__ int wrapi(int v, int N) { return v < 0 ? v + N : (v >= N ? v - N : v); }

__device__ __forceinline__ float softplusf(float y) { return y > 0.f ? y + log1pf(expf(-y)) : log1pf(expf(y)); }
__device__ __forceinline__ float sigmoidf(float y) {
    return y >= 0.f ? 1.f / (1.f + expf(-y)) : expf(y) / (1.f + expf(y));
}

// issue the MMAs of one layer: D (+)= A x B^T over K; TF32: hi*hi (+ hi*lo + lo*hi), BF16: one product
template <bool BF>
__device__ __forceinline__ void issue_layer(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                            int K, int Rb, int nsplit) {
    const int ksteps = K / Lay<BF>::KS;
    for (int ks = 0; ks < ksteps; ++ks) {
        const uint32_t ao = (uint32_t)ks * (TM * 32), bo = (uint32_t)ks * (Rb * 32);
        if constexpr (BF) {
            mma_bf16(d, sdesc(a_hi + ao), sdesc(b_hi + bo), idesc_bf16(TM, Rb), ks > 0 ? 1u : 0u);
        } else {
            mma_tf32(d, sdesc(a_hi + ao), sdesc(b_hi + bo), idesc_tf32(TM, Rb), ks > 0 ? 1u : 0u);
            if (nsplit > 1) {
                mma_tf32(d, sdesc(a_hi + ao), sdesc(b_lo + bo), idesc_tf32(TM, Rb), 1u);
                mma_tf32(d, sdesc(a_lo + ao), sdesc(b_hi + bo), idesc_tf32(TM, Rb), 1u);
            }
        }
    }
}

struct TileMap {
    FastDiv ntz, nty;
    int N;
    int64_t N3;
};

// Saved activations of the forward: y[N3], layer-1 mask m1[4][N3] (16 bits per
// column block), layer-2 mask m2[4][N3] (8 bits per column block).
struct Saved {
    float* y;
    uint16_t* m1;
    uint8_t* m2;
};

// Compute warps synchronise among themselves on named barrier 1 (the
// MMA-issuing warp never joins it); nbar_and also ANDs a predicate over them.
__device__ __forceinline__ void nbar_sync(uint32_t n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }
__device__ __forceinline__ bool nbar_and(uint32_t n, bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(n)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

constexpr int NTW = NT + 32;  // 16 compute warps + the warp whose lane 0 issues the MMAs

// Forward only, warp-specialised and software-pipelined over the CTA's z-line
// tiles. Warps 0-15 build operands and read accumulators; lane 0 of warp 16
// issues the MMAs. The layer-1 operand A1 and accumulator D1 are double-
// buffered (buffer b = the CTA's tile count mod 2), so layer 1 of the next tile
// runs on the tensor cores while the compute warps read this tile's D1; A2 and
// D2 are single. Per tile t of the CTA (t-1, t+1 its neighbours in the CTA's
// sequence), the issuing lane runs
//   wait A1(t+1), MMA1(t+1) -> D1[b^1]; wait A2(t), MMA2(t) -> D2
// and the compute warps
//   lines(t+1) -> A1[b^1], arrive A1(t+1); wait D2(t-1), D2 -> y, M of t-1
//   (one warp per TMEM lane quadrant, taking turns over the tiles);
//   wait D1(t), relu(D1[b] + b1) -> A2, arrive A2(t).
// No named barrier sits in the loop: warps meet only through the mbarriers.
// Handshakes (mbarriers): "A1 full" [2] and "A2 full" take 512 compute-thread
// arrivals, each after its operand stores (async-proxy fence) and after its
// own reads of the accumulator the next MMA into that buffer overwrites;
// "D1 full" [2] and "D2 full" take tcgen05.commit. One barrier per buffer keeps
// every waiter within one phase of its barrier: a parity wait never sees two
// completed phases.

template <bool BF>
struct LayF {
    using L = Lay<BF>;
    static constexpr int CH = K1Z / L::EC;            // 16-byte K chunks per image row
    static constexpr int CH_USED = (27 + L::EC - 1) / L::EC;  // chunks holding inputs
    static constexpr int TASKS = ZR * CH_USED;        // (row, chunk) stores per tile
    static constexpr int TPT = (TASKS + NT - 1) / NT;  // per compute thread
    static constexpr int KST = K1Z / L::KS;           // k-steps per z offset
    static constexpr uint32_t SZ_A1 = CH * ZLBO, SZ_A2 = L::bytes(TM, K2);
    static constexpr uint32_t A1_BUF = L::NP * SZ_A1;  // one A1 buffer (head and tail parts)
    static constexpr uint32_t S_A1 = L::IMG_FWD;
    static constexpr uint32_t S_A2 = S_A1 + 2 * A1_BUF;
    static constexpr uint32_t S_TAIL = S_A2 + L::NP * SZ_A2;
    // 7 barriers + TMEM slot
    static constexpr uint32_t SMEM = S_TAIL + 64;
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(S_A1 % 128 == 0 && S_A2 % 128 == 0 && S_TAIL % 16 == 0 && SZ_A1 % 128 == 0, "aligned regions");
    static_assert(CH % 2 == 0 && KST * 2 == CH, "a k-step is two 16-byte chunks");
};

// z-line tiles: tile = (x * N + y) * nzt + zt, voxels z0 = 128 zt .. min(z0 + 128, N) - 1
struct ZMap {
    FastDiv nzt, n;
    int N;
    int64_t N3;
};

// mbarriers of the forward
enum : int { FB_A1 = 0, FB_A2 = 2, FB_D1 = 3, FB_D2 = 5, FB_DRAIN = 6, FB_COUNT = 7 };

template <bool TWO_NET, bool BF>
__global__ void __launch_bounds__(NTW, 1)
    k_mlp_tc_fwd(const float* __restrict__ feat, const float4* __restrict__ img, ZMap zm, int ntiles, int nsplit,
              float M_scale, float a, float* __restrict__ M_out, Saved sv, int* __restrict__ err, TcCtl ctl) {
    using L = Lay<BF>;
    using F = LayF<BF>;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A2h = sm + F::S_A2;
    unsigned char* A2l = A2h + (L::NP - 1) * F::SZ_A2;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + F::S_TAIL);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + FB_COUNT);
    const float* vec = reinterpret_cast<const float*>(sm + L::S_VEC);
    const float *b1 = vec, *b2 = vec + 64, *w3 = vec + 96, *b3 = vec + 128;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, cb = warp >> 2;
    const int row = quad * 32 + lane;
    constexpr uint32_t ncols = 256;  // D1 [2] x 64 + D2 32
    const int N = zm.N;
    const int64_t N3 = zm.N3;

    {
        const uint32_t n16 = L::IMG_FWD / 16;
        float4* dst = reinterpret_cast<float4*>(sm);
        for (uint32_t i = tid; i < n16; i += NTW) dst[i] = img[i];
        // the padding chunks of both A1 buffers (columns past the 27 inputs) stay zero
        for (uint32_t i = tid; i < (uint32_t)(F::CH - F::CH_USED) * ZR; i += NTW)
            for (int p = 0; p < 2 * L::NP; ++p)
                *reinterpret_cast<float4*>(sm + F::S_A1 + p * F::SZ_A1 + (F::CH_USED + i / ZR) * ZLBO +
                                           (i % ZR) * 16) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < FB_COUNT; ++b) {
            const uint32_t cnt = b < FB_D1 ? (uint32_t)NT : 1u;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bars + b)), "r"(cnt) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == NT / 32) {
        // ---- MMA issue (one lane)
        if (lane == 0) {
            const uint32_t sA1 = smem_u32(sm + F::S_A1), sA2h = smem_u32(A2h), sA2l = smem_u32(A2l);
            const uint32_t sB1 = smem_u32(sm + L::S_B1);
            constexpr uint32_t SZ_B1OZ = L::bytes(N1, K1Z);
            // layer 1 of the tile in A1 buffer b, into D1 buffer b: the three z offsets
            // of the stencil, each a shifted view of A1
            auto mma1 = [&](int b) {
                const uint32_t hi = sA1 + (uint32_t)b * F::A1_BUF, lo = hi + (L::NP - 1) * F::SZ_A1;
                const uint32_t d = tmem + COL_D1 + (uint32_t)b * N1;
                for (int oz = 0; oz < 3; ++oz)
                    for (int ks = 0; ks < F::KST; ++ks) {
                        const uint32_t ao = (uint32_t)ks * 2 * ZLBO + (uint32_t)oz * 16;
                        const uint32_t bo = (uint32_t)oz * SZ_B1OZ + (uint32_t)ks * (N1 * 32);
                        const uint32_t acc = (oz | ks) ? 1u : 0u;
                        if constexpr (BF) {
                            mma_bf16(d, zdesc(hi + ao), sdesc(sB1 + bo), idesc_bf16(TM, N1), acc);
                        } else {
                            mma_tf32(d, zdesc(hi + ao), sdesc(sB1 + bo), idesc_tf32(TM, N1), acc);
                            if (nsplit > 1) {
                                mma_tf32(d, zdesc(hi + ao), sdesc(sB1 + L::SZ_B1 + bo), idesc_tf32(TM, N1), 1u);
                                mma_tf32(d, zdesc(lo + ao), sdesc(sB1 + bo), idesc_tf32(TM, N1), 1u);
                            }
                        }
                    }
                mma_commit(bars + FB_D1 + b);
            };
            uint32_t pa1 = 0, pa2 = 0;  // phase bits: A1 full (bit b), A2 full
            auto wait_a1 = [&](int b) {
                if (!mbar_wait(bars + FB_A1 + b, (pa1 >> b) & 1u, ctl.wait_limit)) return false;
                pa1 ^= 1u << b;
                tc_fence_after();
                return true;
            };
            int tile = blockIdx.x;
            bool run = tile < ntiles;
            if (run) {
                run = wait_a1(0);
                if (!run) atomicExch(err, 1);
                else if (ctl.issue) mma1(0);  // ctl.issue = 0, the test hook: no D1 ever completes
            }
            for (int it = 0; run && tile < ntiles; tile += gridDim.x, ++it) {
                const int b = it & 1;
                if (tile + (int)gridDim.x < ntiles) {
                    if (!wait_a1(b ^ 1)) {
                        atomicExch(err, 1);
                        break;
                    }
                    if (ctl.issue) mma1(b ^ 1);
                }
                if (!mbar_wait(bars + FB_A2, pa2, ctl.wait_limit)) {
                    atomicExch(err, 1);
                    break;
                }
                pa2 ^= 1;
                tc_fence_after();
                if (ctl.issue) {
                    issue_layer<BF>(tmem + COL_D2, sA2h, sA2l, smem_u32(sm + L::S_B2),
                                    smem_u32(sm + L::S_B2 + L::SZ_B2), K2, N2, nsplit);
                    mma_commit(bars + FB_D2);
                }
            }
            mma_commit(bars + FB_DRAIN);  // completes once every MMA issued above has
            mbar_wait(bars + FB_DRAIN, 0, ctl.wait_limit);
        }
        __syncwarp();
    } else {
        // ---- compute warps
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        uint32_t ph1 = 0, ph2 = 0;  // phase bits: D1 full (bit b), D2 full
        bool ok = true;
        auto tile_origin = [&](int tile, int& x, int& y, int& z0) {
            const uint32_t line = zm.nzt.div((uint32_t)tile);
            z0 = (tile - (int)(line * zm.nzt.d)) * TM;
            x = (int)zm.n.div(line);
            y = (int)line - x * N;
        };
        // this thread's build tasks u = tid + NT m: image row i = u % ZR, chunk q = u / ZR,
        // EC input columns k = q EC + e (k >= 27: padding, zero). Fixed over the tiles:
        // zoff = i - 1 (kNoTask: no task) and, per column, the input's offset from the
        // line's centre element, c N^3 + ox N^2 + oy N (kNoTask: padding). Indices fit in
        // 32 bits (3 N^3 < 2^31 for N <= 512). The bf16 image's 8 columns a chunk would
        // not fit in registers: there the offsets are formed per tile.
        constexpr int EC = L::EC;
        constexpr int kNoTask = INT_MIN;
        constexpr bool KEEP = !BF;
        auto col_off = [&](int m, int e) {
            const int k = ((tid + NT * m) / ZR) * EC + e;
            return k < 27 ? (k / 9) * (int)N3 + ((k / 3) % 3 - 1) * N * N + (k % 3 - 1) * N : kNoTask;
        };
        int zoff[F::TPT], koff[F::TPT][KEEP ? EC : 1];
#pragma unroll
        for (int m = 0; m < F::TPT; ++m) {
            const int u = tid + NT * m;
            zoff[m] = u < F::TASKS ? u % ZR - 1 : kNoTask;
            if constexpr (KEEP)
#pragma unroll
                for (int e = 0; e < EC; ++e) koff[m][e] = col_off(m, e);
        }
        float hv[F::TPT][EC];
        auto load_lines = [&](int tile) {
            if (tile >= ntiles) return;
            int x, y, z0;
            tile_origin(tile, x, y, z0);
            // lines off the mesh's x and y borders need no wrap in x or y
            const bool inner = x > 0 && x < N - 1 && y > 0 && y < N - 1;
            const int centre = (x * N + y) * N;
#pragma unroll
            for (int m = 0; m < F::TPT; ++m) {
                if (zoff[m] == kNoTask) continue;
                int z = z0 + zoff[m];
                z = z < 0 ? z + N : z;
                if (z >= N) z = z >= 2 * N ? z % N : z - N;  // several wraps only when N < 129
#pragma unroll
                for (int e = 0; e < EC; ++e) {
                    float v = 0.f;
                    int ko;
                    if constexpr (KEEP)
                        ko = koff[m][e];
                    else
                        ko = col_off(m, e);
                    if (ko != kNoTask) {
                        if (inner) {
                            v = feat[(uint32_t)(centre + z + ko)];
                        } else {
                            const int k = ((tid + NT * m) / ZR) * EC + e;
                            const int c = k / 9, gx = wrapi(x + (k / 3) % 3 - 1, N), gy = wrapi(y + k % 3 - 1, N);
                            v = feat[(uint32_t)(c * (int)N3 + (gx * N + gy) * N + z)];
                        }
                    }
                    hv[m][e] = v;
                }
            }
        };
        // prefetched lines -> A1 buffer b, then arrive on its "A1 full"
        auto build_A1 = [&](int b) {
            unsigned char* A1h = sm + F::S_A1 + (uint32_t)b * F::A1_BUF;
            unsigned char* A1l = A1h + (L::NP - 1) * F::SZ_A1;  // == A1h with one part
#pragma unroll
            for (int m = 0; m < F::TPT; ++m) {
                const int u = tid + NT * m;
                if (u >= F::TASKS) continue;
                const int q = u / ZR, i = u - q * ZR;
                const uint32_t off = (uint32_t)q * ZLBO + (uint32_t)i * 16;
                if constexpr (BF) {
                    *reinterpret_cast<uint4*>(A1h + off) =
                        make_uint4(pack_bf16x2(hv[m][0], hv[m][1]), pack_bf16x2(hv[m][2], hv[m][3]),
                                   pack_bf16x2(hv[m][4], hv[m][5]), pack_bf16x2(hv[m][6], hv[m][7]));
                } else {
                    put4(A1h, A1l, off, hv[m][0], hv[m][1], hv[m][2], hv[m][3]);
                }
            }
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(bars + FB_A1 + b);
        };
        // bounded wait on a commit barrier. Each thread waits and gives up on its own:
        // no named barrier is left in the loop, so a thread that gives up leaves no
        // other thread waiting without a bound.
        auto wait_commit = [&](int bar, uint32_t& ph, int bit) {
            const bool got = mbar_wait(bars + bar, (ph >> bit) & 1u, ctl.wait_limit);
            ph ^= 1u << bit;
            if (got) tc_fence_after();
            return got;
        };
        // relu(D1[b] + b1) of a tile -> A2 and the layer-1 mask, then arrive on "A2 full"
        auto epilogue1 = [&](int tile, int b) {
            int x, y, z0;
            tile_origin(tile, x, y, z0);
            const int64_t row_vox = ((int64_t)x * N + y) * N + z0 + row;
            float av[16];
            tmem_ld16(lane_base + COL_D1 + (uint32_t)b * N1 + 16 * cb, av);
            uint32_t mask1 = 0;
            float z[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float pre = av[j] + b1[16 * cb + j];
                mask1 |= (pre > 0.f ? 1u : 0u) << j;
                z[j] = fmaxf(pre, 0.f);
            }
            if (sv.m1 && z0 + row < N) sv.m1[cb * N3 + row_vox] = (uint16_t)mask1;
            put8<BF>(A2h, A2l, row, 16 * cb, z);
            put8<BF>(A2h, A2l, row, 16 * cb + 8, z + 8);
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(bars + FB_A2);
        };
        // y = b3 + w3 . relu(D2 + b2) of a tile, its layer-2 masks and the head, by the
        // warp of column block `sel` of each TMEM lane quadrant (one voxel per thread;
        // the column blocks' partial sums are added in the order of a 4-warp split)
        auto epilogue2 = [&](int tile) {
            int x, y, z0;
            tile_origin(tile, x, y, z0);
            const int64_t vox = ((int64_t)x * N + y) * N + z0 + row;
            const bool in = z0 + row < N;
            float p[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float av[16];
                tmem_ld16(lane_base + COL_D2 + 16 * h, av);
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const int blk = 2 * h + g;
                    uint32_t mask2 = 0;
                    float sacc = 0.f;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float pre = av[8 * g + j] + b2[8 * blk + j];
                        mask2 |= (pre > 0.f ? 1u : 0u) << j;
                        sacc = fmaf(w3[8 * blk + j], fmaxf(pre, 0.f), sacc);
                    }
                    p[blk] = sacc;
                    if (sv.m2 && in) sv.m2[blk * N3 + vox] = (uint8_t)mask2;
                }
            }
            if (!in) return;
            const float yv = b3[0] + ((p[0] + p[1]) + (p[2] + p[3]));
            if (sv.y) sv.y[vox] = yv;
            if (TWO_NET) {
                const float pl = sigmoidf(a * yv);
                float u0, u1, u2;
                M_out[vox] = M_scale * pl *
                             mass_net<false>(vec + VEC_MASS, feat[vox], feat[N3 + vox], feat[2 * N3 + vox], 0.f, u0,
                                             u1, u2);
            } else {
                M_out[vox] = M_scale * softplusf(yv);
            }
        };

        int tile = blockIdx.x, prev = -1, last_it = 0;
        load_lines(tile);
        if (tile < ntiles) {
            build_A1(0);
            load_lines(tile + gridDim.x);
        }
        for (int it = 0; tile < ntiles; tile += gridDim.x, ++it, last_it = it) {
            const int b = it & 1, nxt = tile + gridDim.x;
            // (1) the next tile's A1 (its buffer's previous layer 1 and D1 reads are done)
            if (nxt < ntiles) {
                build_A1(b ^ 1);
                load_lines(nxt + gridDim.x);
            }
            // (2) the previous tile's layer 2 (frees A2 and D2); column block
            //     (it - 1) mod 4 reads it
            if (prev >= 0) {
                if (!(ok = wait_commit(FB_D2, ph2, 0))) break;
                if (cb == ((it - 1) & 3)) epilogue2(prev);
            }
            // (3) this tile's layer 1 -> A2
            if (!(ok = wait_commit(FB_D1 + b, ph1, b))) break;
            epilogue1(tile, b);
            prev = tile;
        }
        if (ok && prev >= 0 && (ok = wait_commit(FB_D2, ph2, 0)) && cb == ((last_it - 1) & 3)) epilogue2(prev);
        if (!ok && lane == 0) atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// Backward (input gradient) from the forward's saved activations, warp-
// specialised and software-pipelined like k_mlp_tc_fwd. A3 and the
// accumulators D3 and D4 are double-buffered (buffer = the CTA's tile count
// mod 2), A4 and the g_v staging are single. Per tile t of the CTA (t-1, t+1
// its neighbours in the CTA's sequence), the issuing lane runs
//   wait A4(t), MMA4(t) -> D4[t]; wait A3(t+1), MMA3(t+1) -> D3[t+1]
// and the compute warps
//   wait D4(t-1) (frees A4); wait D3(t), D3[t] [a1 > 0] -> A4, arrive A4(t);
//   g_y(t+1) -> A3[t+1], arrive A3(t+1); D4[t-1] -> g_v -> box sums of t-1,
// so layer 1's input gradient of tile t runs on the tensor cores while the
// compute warps sum the boxes of tile t-1. One barrier per buffer keeps every
// waiter within one phase of its barrier.
// Only the layer-2 and layer-1 weight images (B3 = W2, B4 = W1) and the vector
// block are staged.
template <bool BF>
struct LayB {
    using L = Lay<BF>;
    static constexpr uint32_t IMG_OFF = L::S_VEC;         // staged: vector block, B3, B4 (contiguous in the image)
    static constexpr uint32_t IMG_BYTES = L::IMG_ALL - L::S_VEC;
    static constexpr uint32_t S_VEC = 0, S_B3 = L::S_B3 - L::S_VEC, S_B4 = L::S_B4 - L::S_VEC;
    static constexpr uint32_t SZ_A3 = L::bytes(TM, K3), SZ_A4 = L::bytes(TM, K4);
    static constexpr uint32_t A3_BUF = L::NP * SZ_A3;  // one A3 buffer (head and tail parts)
    static constexpr uint32_t S_A3 = (IMG_BYTES + 127) / 128 * 128;
    static constexpr uint32_t S_A4 = S_A3 + 2 * A3_BUF;
    static constexpr uint32_t S_GV = S_A4 + L::NP * SZ_A4;
    static constexpr int NTS = 27 * TX * TY * HZ;  // z-folded g_v, Ts[27][TX][TY][HZ]
    static constexpr uint32_t S_TAIL = S_GV + 4 * NTS;
    // g_y [TM], centre-value gradients [3 slots][3][TM], 8 barriers + TMEM slot
    static constexpr uint32_t SMEM = S_TAIL + 4 * TM + 4 * 9 * TM + 80;
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(S_B3 % 128 == 0 && S_B4 % 128 == 0 && S_A3 % 128 == 0 && S_A4 % 128 == 0 && S_GV % 16 == 0 &&
                      A3_BUF % 128 == 0 && S_TAIL % 16 == 0,
                  "aligned regions");
    static_assert(IMG_OFF % 16 == 0 && IMG_BYTES % 16 == 0, "16-byte image copy");
};

// mbarriers of the backward
enum : int { BB_A3 = 0, BB_A4 = 2, BB_D3 = 3, BB_D4 = 5, BB_DRAIN = 7, BB_COUNT = 8 };
// TMEM columns of the backward's buffers: D3 [2] x 64, D4 [2] x 96 (at 128-column offsets)
constexpr uint32_t COL_D3B = 0, COL_D4B = 128;

template <bool TWO_NET, bool BF>
__global__ void __launch_bounds__(NTW, 1)
    k_mlp_tc_bwd(const float* __restrict__ feat, const float* __restrict__ gM, const float4* __restrict__ img,
              TileMap tm, int ntiles, int nsplit, float M_scale, float a, float* __restrict__ gbox, Saved sv,
              int* __restrict__ err, TcCtl ctl) {
    using L = Lay<BF>;
    using B = LayB<BF>;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A4h = sm + B::S_A4;
    unsigned char* A4l = A4h + (L::NP - 1) * B::SZ_A4;
    float* gvs = reinterpret_cast<float*>(sm + B::S_GV);  // Ts[27][TX][TY][HZ]
    float* gys = reinterpret_cast<float*>(sm + B::S_TAIL);
    float* gcen = gys + TM;  // [3 slots][3][TM]
    uint64_t* bars = reinterpret_cast<uint64_t*>(gcen + 9 * TM);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + BB_COUNT);
    const float* vec = reinterpret_cast<const float*>(sm + B::S_VEC);
    const float* w3 = vec + 96;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, cb = warp >> 2;
    const int row = quad * 32 + lane;
    constexpr uint32_t ncols = 512;  // D3 [2] at 0, 64; D4 [2] at 128, 256
    const int N = tm.N;
    const int64_t N3 = tm.N3;

    {
        const uint32_t n16 = B::IMG_BYTES / 16;
        const float4* src = img + B::IMG_OFF / 16;
        float4* dst = reinterpret_cast<float4*>(sm);
        for (uint32_t i = tid; i < n16; i += NTW) dst[i] = src[i];
    }
    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < BB_COUNT; ++b) {
            const uint32_t cnt = b < BB_D3 ? (uint32_t)NT : 1u;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bars + b)), "r"(cnt) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == NT / 32) {
        // ---- MMA issue (one lane)
        if (lane == 0) {
            const uint32_t sA3 = smem_u32(sm + B::S_A3), sA4h = smem_u32(A4h), sA4l = smem_u32(A4l);
            auto mma3 = [&](int b) {  // A3 buffer b -> D3 buffer b
                const uint32_t hi = sA3 + (uint32_t)b * B::A3_BUF;
                issue_layer<BF>(tmem + COL_D3B + (uint32_t)b * 64, hi, hi + (L::NP - 1) * B::SZ_A3,
                                smem_u32(sm + B::S_B3), smem_u32(sm + B::S_B3 + L::SZ_B3), K3, NB3, nsplit);
                mma_commit(bars + BB_D3 + b);
            };
            uint32_t pa3 = 0, pa4 = 0;  // phase bits: A3 full (bit b), A4 full
            auto wait_a3 = [&](int b) {
                if (!mbar_wait(bars + BB_A3 + b, (pa3 >> b) & 1u, ctl.wait_limit)) return false;
                pa3 ^= 1u << b;
                tc_fence_after();
                return true;
            };
            int tile = blockIdx.x;
            bool run = tile < ntiles;
            if (run) {
                run = wait_a3(0);
                if (!run) atomicExch(err, 1);
                else if (ctl.issue) mma3(0);  // ctl.issue = 0, the test hook: no D3 ever completes
            }
            for (int it = 0; run && tile < ntiles; tile += gridDim.x, ++it) {
                const int b = it & 1;
                if (!mbar_wait(bars + BB_A4, pa4, ctl.wait_limit)) {
                    atomicExch(err, 1);
                    break;
                }
                pa4 ^= 1;
                tc_fence_after();
                if (ctl.issue) {
                    issue_layer<BF>(tmem + COL_D4B + (uint32_t)b * 128, sA4h, sA4l, smem_u32(sm + B::S_B4),
                                    smem_u32(sm + B::S_B4 + L::SZ_B4), K4, NB4, nsplit);
                    mma_commit(bars + BB_D4 + b);
                }
                if (tile + (int)gridDim.x < ntiles) {
                    if (!wait_a3(b ^ 1)) {
                        atomicExch(err, 1);
                        break;
                    }
                    if (ctl.issue) mma3(b ^ 1);
                }
            }
            mma_commit(bars + BB_DRAIN);  // completes once every MMA issued above has
            mbar_wait(bars + BB_DRAIN, 0, ctl.wait_limit);
        }
        __syncwarp();
    } else {
        // ---- compute warps
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        uint32_t ph3 = 0, ph4 = 0;  // phase bits: D3 full (bit b), D4 full (bit b)
        bool ok = true;
        auto tile_origin = [&](int tile, int& x0, int& y0, int& z0) {
            const uint32_t t2 = tm.ntz.div((uint32_t)tile);
            const int tz = tile - (int)(t2 * tm.ntz.d);
            const int tx = (int)tm.nty.div(t2);
            const int ty = (int)t2 - tx * (int)tm.nty.d;
            x0 = tx * TX;
            y0 = ty * TY;
            z0 = tz * TZ;
        };
        // saved forward state of a tile, loaded one tile ahead: g_M, y and the
        // centre values of rows tid < TM; the masks of this thread's row and column block
        float L_gm = 0.f, L_y = 0.f, L_f[3] = {0.f, 0.f, 0.f};
        uint32_t L_m1 = 0, L_m2 = 0;
        auto load_saved = [&](int tile) {
            if (tile >= ntiles) return;
            int x0, y0, z0;
            tile_origin(tile, x0, y0, z0);
            if (tid < TM) {
                const int gx = x0 + (tid >> 6), gy = y0 + ((tid >> 4) & 3), gz = z0 + (tid & 15);
                const bool in = gx < N && gy < N && gz < N;
                const int64_t v = ((int64_t)gx * N + gy) * N + gz;
                L_gm = in ? gM[v] : 0.f;
                L_y = in ? sv.y[v] : 0.f;
                if (TWO_NET)
#pragma unroll
                    for (int c = 0; c < 3; ++c) L_f[c] = in ? feat[c * N3 + v] : 0.f;
            }
            const int gx = x0 + (row >> 6), gy = y0 + ((row >> 4) & 3), gz = z0 + (row & 15);
            const bool in = gx < N && gy < N && gz < N;
            const int64_t v = ((int64_t)gx * N + gy) * N + gz;
            L_m1 = in ? sv.m1[cb * N3 + v] : 0u;
            L_m2 = in ? sv.m2[cb * N3 + v] : 0u;
        };
        // g_y of the loaded tile, A3 = g_a2 = w3 g_y [a2 > 0] into A3 buffer b, arrive on
        // its "A3 full"; the centre-value gradients (two-network head) into gcen slot `slot`
        auto build_A3 = [&](int tile, int b, int slot) {
            unsigned char* A3h = sm + B::S_A3 + (uint32_t)b * B::A3_BUF;
            unsigned char* A3l = A3h + (L::NP - 1) * B::SZ_A3;  // == A3h with one part
            int x0, y0, z0;
            tile_origin(tile, x0, y0, z0);
            if (tid < TM) {
                const int r = tid;
                const int gx = x0 + (r >> 6), gy = y0 + ((r >> 4) & 3), gz = z0 + (r & 15);
                const bool in = gx < N && gy < N && gz < N;
                const float g = in ? L_gm * M_scale : 0.f;
                if (TWO_NET) {
                    // M = M_scale p m: dM/dy = M_scale m a p (1 - p); dM/dm = M_scale p
                    const float p = sigmoidf(a * L_y);
                    float g0, g1, g2;
                    const float m = mass_net<true>(vec + VEC_MASS, L_f[0], L_f[1], L_f[2], g * p, g0, g1, g2);
                    gys[r] = g * m * a * p * (1.f - p);
                    gcen[(slot * 3 + 0) * TM + r] = g0;
                    gcen[(slot * 3 + 1) * TM + r] = g1;
                    gcen[(slot * 3 + 2) * TM + r] = g2;
                } else {
                    gys[r] = g * sigmoidf(L_y);
                }
            }
            nbar_sync(NT);
            {
                const float g = gys[row];
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = ((L_m2 >> j) & 1u) ? w3[8 * cb + j] * g : 0.f;
                put8<BF>(A3h, A3l, row, 8 * cb, v);
            }
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(bars + BB_A3 + b);
        };
        // bounded wait on a commit barrier, agreed by all compute threads (the box
        // sums below keep named barriers in the loop)
        auto wait_commit = [&](int bar, uint32_t& ph, int bit) {
            const bool got = nbar_and(NT, mbar_wait(bars + bar, (ph >> bit) & 1u, ctl.wait_limit));
            ph ^= 1u << bit;
            if (got) tc_fence_after();
            return got;
        };
        // A4 = g_a1 [a1 > 0] from D3 buffer b, then arrive on "A4 full"
        auto epilogue3 = [&](int b, uint32_t m1) {
            float av[16];
            tmem_ld16(lane_base + COL_D3B + (uint32_t)b * 64 + 16 * cb, av);
#pragma unroll
            for (int j = 0; j < 16; ++j) av[j] = ((m1 >> j) & 1u) ? av[j] : 0.f;
            put8<BF>(A4h, A4l, row, 16 * cb, av);
            put8<BF>(A4h, A4l, row, 16 * cb + 8, av + 8);
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(bars + BB_A4);
        };
        // box cells e = tid + NT j of this thread (fixed over the tiles): field c, cell
        // (hx, hy, hz); the term of (ox, oy) sits at gvs[box_base + ((ox + 1) 3 + oy + 1) *
        // TX TY HZ - (ox TY + oy) HZ], present when bit (ox + 1) 3 + oy + 1 of the cell's
        // 9 mask bits is set (its tile cell lies inside the tile)
        constexpr int NBOX = 3 * HX * HY * HZ, BOX_PER_THREAD = (NBOX + NT - 1) / NT;
        static_assert(BOX_PER_THREAD * 9 <= 32, "mask bits of a thread's box cells in one word");
        int box_base[BOX_PER_THREAD];
        uint32_t box_mask = 0;
#pragma unroll
        for (int j = 0; j < BOX_PER_THREAD; ++j) {
            const int e = tid + NT * j;
            const int c = e / (HX * HY * HZ), rem = e - c * (HX * HY * HZ);
            const int hx = rem / (HY * HZ), hy = (rem / HZ) % HY, hz = rem % HZ;
            box_base[j] = c * 9 * (TX * TY * HZ) + ((hx - 1) * TY + (hy - 1)) * HZ + hz;
            uint32_t msk = 0;
            for (int ox = -1; ox <= 1; ++ox)
                for (int oy = -1; oy <= 1; ++oy) {
                    const int lx = hx - 1 - ox, ly = hy - 1 - oy;
                    if (e < NBOX && lx >= 0 && lx < TX && ly >= 0 && ly < TY) msk |= 1u << ((ox + 1) * 3 + (oy + 1));
                }
            box_mask |= msk << (9 * j);
        }

        // g_v of a tile from D4 buffer b (gcen slot `slot`), folded over the z offset in
        // registers: a thread holds 24 columns = 8 whole (c, ox, oy) triples over oz
        // (k = 3 q + oz + 1), and the voxels z - 1, z + 1 of its row are the neighbouring
        // lanes of its 16-lane group, so T_q(hz) = g_v[q, oz=-1](hz) + g_v[q, 0](hz - 1) +
        // g_v[q, 1](hz - 2) (box z index hz = lz + 1; lane 0 also gives hz = 0, lane 15
        // hz = 17) needs two shuffles per triple. T goes to shared memory as
        // Ts[q][lx][ly][hz] (27 x 2 x 4 x 18; rows outside the mesh give 0). Then the box
        // sums: field c at box cell (hx, hy, hz) collects T of the triples (c, ox, oy) at
        // tile (lx, ly) = (hx - 1 - ox, hy - 1 - oy), in a fixed order.
        auto epilogue4 = [&](int tile, int b, int slot) {
            int x0, y0, z0;
            tile_origin(tile, x0, y0, z0);
            {
                const int lx = row >> 6, ly = (row >> 4) & 3, lz = row & 15;
                const bool in = x0 + lx < N && y0 + ly < N && z0 + lz < N;
                float* Ts = gvs;
                const int cell = (lx * TY + ly) * HZ;
                float trip[8][3];  // [triple][oz + 1]
#pragma unroll
                for (int h = 0; h < 3; ++h) {
                    float av[8];
                    tmem_ld8(lane_base + COL_D4B + (uint32_t)b * 128 + 24 * cb + 8 * h, av);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int k = 24 * cb + 8 * h + j;
                        float v = in ? av[j] : 0.f;
                        if (TWO_NET && k < NI && k % 27 == 13 && in) v += gcen[(slot * 3 + k / 27) * TM + row];
                        av[j] = v;
                    }
                    // a load of 8 columns is not a whole number of triples: regroup
#pragma unroll
                    for (int j = 0; j < 8; ++j) trip[(8 * h + j) / 3][(8 * h + j) % 3] = av[j];
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int q = 8 * cb + t;  // triple: c * 9 + (ox + 1) * 3 + (oy + 1)
                    const float gm1 = trip[t][0], g0 = trip[t][1], gp1 = trip[t][2];
                    float from_up = __shfl_down_sync(0xffffffffu, gm1, 1, 16);  // g_v[-1](lz + 1)
                    float from_dn = __shfl_up_sync(0xffffffffu, gp1, 1, 16);    // g_v[+1](lz - 1)
                    if (lz == 15) from_up = 0.f;
                    if (lz == 0) from_dn = 0.f;
                    if (q < 27) {
                        float* Tq = Ts + q * (TX * TY * HZ) + cell;
                        Tq[lz + 1] = from_up + g0 + from_dn;
                        if (lz == 0) Tq[0] = gm1;
                        if (lz == 15) Tq[17] = gp1;
                    }
                }
            }
            tc_fence_before();
            nbar_sync(NT);
#pragma unroll
            for (int j = 0; j < BOX_PER_THREAD; ++j) {
                const int e = tid + NT * j;
                if (e >= NBOX) break;
                const uint32_t msk = box_mask >> (9 * j);
                float acc = 0.f;
#pragma unroll
                for (int ox = -1; ox <= 1; ++ox)
#pragma unroll
                    for (int oy = -1; oy <= 1; ++oy)
                        if (msk & (1u << ((ox + 1) * 3 + (oy + 1))))
                            acc += gvs[box_base[j] + ((ox + 1) * 3 + (oy + 1)) * (TX * TY * HZ) - (ox * TY + oy) * HZ];
                gbox[(int64_t)tile * NBOX + e] = acc;
            }
            // the next writes of Ts and gcen come after the next tile's barriers
        };

        int tile = blockIdx.x, prev = -1, last_it = 0;
        uint32_t m1_cur = 0;
        load_saved(tile);
        if (tile < ntiles) {
            build_A3(tile, 0, 0);
            m1_cur = L_m1;
            load_saved(tile + gridDim.x);
        }
        for (int it = 0; tile < ntiles; tile += gridDim.x, ++it, last_it = it) {
            const int b = it & 1, nxt = tile + gridDim.x;
            // (1) the previous tile's layer-1 input gradient (frees A4)
            if (prev >= 0 && !(ok = wait_commit(BB_D4 + (b ^ 1), ph4, b ^ 1))) break;
            // (2) this tile's layer-2 input gradient -> A4
            if (!(ok = wait_commit(BB_D3 + b, ph3, b))) break;
            epilogue3(b, m1_cur);
            // (3) the next tile's A3 (its buffer's previous MMA3 and D3 reads are done)
            uint32_t m1_nxt = 0;
            if (nxt < ntiles) {
                build_A3(nxt, b ^ 1, (it + 1) % 3);
                m1_nxt = L_m1;
                load_saved(nxt + gridDim.x);
            }
            // (4) g_v and box sums of the previous tile while this tile's MMA4 runs
            if (prev >= 0) epilogue4(prev, b ^ 1, (it + 2) % 3);
            m1_cur = m1_nxt;
            prev = tile;
        }
        if (ok && prev >= 0) {
            const int b = (last_it - 1) & 1;
            if ((ok = wait_commit(BB_D4 + b, ph4, b))) epilogue4(prev, b, (last_it - 1) % 3);
        }
        if (!ok && tid == 0) atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// host: split into TF32 head and tail (round to nearest, ties away, at bit 13)
float tf32_round(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {
        u += 0x1000u;
        u &= 0xffffe000u;
    }
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// host: float -> bfloat16 bits, round to nearest, ties to even (finite values)
uint16_t bf16_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// B operand (R rows, K columns) into the image: TF32 head and tail parts (the
// tail lo_delta bytes after the head; 0 means right after it), or one bf16 part
template <bool BF>
void put_operand(std::vector<unsigned char>& img, uint32_t base, int R, int K, float (*get)(const float*, int, int),
                 const float* W, uint32_t lo_delta = 0) {
    if (lo_delta == 0) lo_delta = Lay<BF>::bytes(R, K);
    using L = Lay<BF>;
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < K; ++k) {
            const float v = get(W, r, k);
            const uint32_t o = base + L::off(R, r, k);
            if constexpr (BF) {
                const uint16_t h = bf16_bits(v);
                std::memcpy(&img[o], &h, 2);
            } else {
                const float hi = tf32_round(v), lo = v - hi;
                std::memcpy(&img[o], &hi, 4);
                std::memcpy(&img[o + lo_delta], &lo, 4);
            }
        }
}

// layer-1 weights of z offset oz (0..2 for -1..1) on the z-line columns k = c*9 + (ox+1)*3 + (oy+1)
template <int OZ>
float get_B1z(const float* W, int h, int k) {
    if (h >= H1 || k >= 27) return 0.f;
    const int c = k / 9, oxy = k % 9;  // (ox+1)*3 + (oy+1)
    return W[h * NI + c * 27 + oxy * 3 + OZ];
}
float get_B2(const float* W, int h2, int h1) { return (h2 < H2 && h1 < H1) ? W[OFF_W2 + h2 * H1 + h1] : 0.f; }
float get_B3(const float* W, int h1, int h2) { return (h2 < H2 && h1 < H1) ? W[OFF_W2 + h2 * H1 + h1] : 0.f; }
float get_B4(const float* W, int k, int h1) { return (h1 < H1 && k < NI) ? W[h1 * NI + k] : 0.f; }

TileMap tile_map(const pmr_ctx* c, int* ntiles) {
    const int N = c->N;
    const int ntx = (N + TX - 1) / TX, nty = (N + TY - 1) / TY, ntz = (N + TZ - 1) / TZ;
    *ntiles = ntx * nty * ntz;
    TileMap m;
    m.ntz = FastDiv((uint32_t)ntz);
    m.nty = FastDiv((uint32_t)nty);
    m.N = N;
    m.N3 = c->N3;
    return m;
}

// Candidate (tile, box index) pairs of cell x along one axis: the tiles of the
// real cells x+1, x, x-1 (periodic), each holding x at box index (p mod TS) + 1 + d;
// duplicates (the same tile and index reached twice) are dropped.
template <int TS>
__device__ __forceinline__ int axis_boxes(int x, int N, int* t_out, int* b_out) {
    int n = 0;
#pragma unroll
    for (int d = 1; d >= -1; --d) {
        int p = x - d;
        p = p < 0 ? p + N : (p >= N ? p - N : p);
        const int t = p / TS, b = p - t * TS + 1 + d;
        bool dup = false;
        for (int i = 0; i < n; ++i) dup |= (t_out[i] == t && b_out[i] == b);
        if (!dup) {
            t_out[n] = t;
            b_out[n] = b;
            ++n;
        }
    }
    return n;
}

// g_field[c](cell) = sum over the tiles whose box holds the cell, in a fixed order.
__global__ void __launch_bounds__(256) k_stencil_tiles(const float* __restrict__ gbox, int N, int nty, int ntz,
                                                       float* __restrict__ gfeat) {
    const int64_t N3 = (int64_t)N * N * N;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    const int x = (int)(v / ((int64_t)N * N)), y = (int)((v / N) % N), z = (int)(v % N);
    int tx[3], bx[3], ty[3], by[3], tz[3], bz[3];
    const int nx = axis_boxes<TX>(x, N, tx, bx), ny = axis_boxes<TY>(y, N, ty, by), nz = axis_boxes<TZ>(z, N, tz, bz);
    constexpr int BOX = HX * HY * HZ;
    float acc[3] = {0.f, 0.f, 0.f};
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                const int64_t tile = ((int64_t)tx[i] * nty + ty[j]) * ntz + tz[k];
                const float* b = gbox + tile * (3 * BOX) + (bx[i] * HY + by[j]) * HZ + bz[k];
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[c] += b[c * BOX];
            }
#pragma unroll
    for (int c = 0; c < 3; ++c) gfeat[c * N3 + v] = acc[c];
}

template <bool BF>
std::vector<unsigned char> build_image(const float* W) {
    using L = Lay<BF>;
    std::vector<unsigned char> img(L::IMG_ALL, 0);
    // layer 1: the three z-offset sub-images, all heads first, then all tails
    put_operand<BF>(img, L::S_B1, N1, K1Z, get_B1z<0>, W, L::SZ_B1);
    put_operand<BF>(img, L::S_B1 + L::bytes(N1, K1Z), N1, K1Z, get_B1z<1>, W, L::SZ_B1);
    put_operand<BF>(img, L::S_B1 + 2 * L::bytes(N1, K1Z), N1, K1Z, get_B1z<2>, W, L::SZ_B1);
    put_operand<BF>(img, L::S_B2, N2, K2, get_B2, W);
    put_operand<BF>(img, L::S_B3, NB3, K3, get_B3, W);
    put_operand<BF>(img, L::S_B4, NB4, K4, get_B4, W);
    float vec[SZ_VEC / 4] = {};
    for (int h = 0; h < H1; ++h) vec[h] = W[OFF_B1 + h];
    for (int h = 0; h < H2; ++h) vec[64 + h] = W[OFF_B2 + h];
    for (int h = 0; h < H2; ++h) vec[96 + h] = W[OFF_W3 + h];
    vec[128] = W[OFF_B3];
    for (int i = 0; i < kMassWeights; ++i) vec[VEC_MASS + i] = W[OFF_B3 + 1 + i];  // zeros unless head == 1
    std::memcpy(&img[L::S_VEC], vec, SZ_VEC);
    return img;
}

template <bool BF>
int set_smem_attrs(pmr_ctx* c) {
    PMR_TRY(check_cuda(c, cudaFuncSetAttribute(k_mlp_tc_fwd<false, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)LayF<BF>::SMEM), "smem attr"));
    PMR_TRY(check_cuda(c, cudaFuncSetAttribute(k_mlp_tc_fwd<true, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)LayF<BF>::SMEM), "smem attr"));
    PMR_TRY(check_cuda(c, cudaFuncSetAttribute(k_mlp_tc_bwd<false, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)LayB<BF>::SMEM), "smem attr"));
    return check_cuda(c, cudaFuncSetAttribute(k_mlp_tc_bwd<true, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)LayB<BF>::SMEM), "smem attr");
}

template <bool BWD, bool BF>
int launch_tc(pmr_ctx* c, const float* feat, const float* gM, float* M, int nsplit, float a) {
    int ntiles = 0;
    TileMap m = tile_map(c, &ntiles);
    const float4* img = reinterpret_cast<const float4*>(BF ? c->tc_img_bf : c->tc_img);
    const float Ms = (float)c->cfg.M_scale;
    const Saved sv{c->nn_y, c->nn_m1, c->nn_m2};  // written by the forward, read by the backward
    const TcCtl ctl{c->tc_stall ? kTestWaitLimit : kWaitLimit, c->tc_stall ? 0 : 1};
    if (!BWD) {
        // z-line tiles: N^2 lines of ceil(N / 128) segments
        const int nzt = (c->N + TM - 1) / TM;
        ZMap zm;
        zm.nzt = FastDiv((uint32_t)nzt);
        zm.n = FastDiv((uint32_t)c->N);
        zm.N = c->N;
        zm.N3 = c->N3;
        const int nz_tiles = c->N * c->N * nzt;
        const int gz = std::min(nz_tiles, c->num_sms);
        const uint32_t sf = LayF<BF>::SMEM;
        if (c->cfg.head == 1)
            k_mlp_tc_fwd<true, BF><<<gz, NTW, sf, c->stream>>>(feat, img, zm, nz_tiles, nsplit, Ms, a, M, sv,
                                                               c->tc_err, ctl);
        else
            k_mlp_tc_fwd<false, BF><<<gz, NTW, sf, c->stream>>>(feat, img, zm, nz_tiles, nsplit, Ms, a, M, sv,
                                                                c->tc_err, ctl);
        return check_launch(c, "mlp_tc_fwd");
    }
    const int grid = std::min(ntiles, c->num_sms);
    const uint32_t sb = LayB<BF>::SMEM;
    if (c->cfg.head == 1)
        k_mlp_tc_bwd<true, BF><<<grid, NTW, sb, c->stream>>>(feat, gM, img, m, ntiles, nsplit, Ms, a, c->gbox, sv,
                                                          c->tc_err, ctl);
    else
        k_mlp_tc_bwd<false, BF><<<grid, NTW, sb, c->stream>>>(feat, gM, img, m, ntiles, nsplit, Ms, a, c->gbox, sv,
                                                           c->tc_err, ctl);
    return check_launch(c, "mlp_tc_bwd");
}

}  // namespace

// Weight images for the tensor-core kernels (TF32 parts and bf16), built once per context.
int mlp_tc_init(pmr_ctx* c) {
    const float* W = c->W_host.data();
    const std::vector<unsigned char> it = build_image<false>(W), ib = build_image<true>(W);
    PMR_TRY(check_cuda(c, cudaMalloc(&c->tc_img, it.size()), "tc weights"));
    PMR_TRY(check_cuda(c, cudaMemcpy(c->tc_img, it.data(), it.size(), cudaMemcpyHostToDevice), "tc weights"));
    PMR_TRY(check_cuda(c, cudaMalloc(&c->tc_img_bf, ib.size()), "tc weights"));
    PMR_TRY(check_cuda(c, cudaMemcpy(c->tc_img_bf, ib.data(), ib.size(), cudaMemcpyHostToDevice), "tc weights"));
    PMR_TRY(check_cuda(c, cudaMalloc(&c->tc_err, sizeof(int)), "tc flag"));
    PMR_TRY(check_cuda(c, cudaMemset(c->tc_err, 0, sizeof(int)), "tc flag"));
    PMR_TRY(set_smem_attrs<false>(c));
    return set_smem_attrs<true>(c);
}

void mlp_tc_free(pmr_ctx* c) {
    cudaFree(c->tc_img);
    cudaFree(c->tc_img_bf);
    c->tc_img_bf = nullptr;
    cudaFree(c->tc_err);
    c->tc_img = nullptr;
    c->tc_err = nullptr;
}

int mlp_tc_box_floats(int N) {
    return ((N + TX - 1) / TX) * ((N + TY - 1) / TY) * ((N + TZ - 1) / TZ) * 3 * HX * HY * HZ;
}

// input gradient of the three fields from the per-tile box sums of mlp_tc_backward_gv
int stencil_tiles(pmr_ctx* c, float* gfeat) {
    k_stencil_tiles<<<nblocks(c->N3, 256), 256, 0, c->stream>>>(c->gbox, c->N, (c->N + TY - 1) / TY,
                                                                (c->N + TZ - 1) / TZ, gfeat);
    return check_launch(c, "stencil_tiles");
}

// nsplit: 3 = TF32 head/tail products (float32 accuracy), 1 = plain TF32, 0 = bf16 operands
int mlp_tc_forward(pmr_ctx* c, const float* feat, float* M, int nsplit, float a) {
    return nsplit == 0 ? launch_tc<false, true>(c, feat, nullptr, M, 0, a)
                       : launch_tc<false, false>(c, feat, nullptr, M, nsplit, a);
}

int mlp_tc_backward_gv(pmr_ctx* c, const float* feat, const float* gM, int nsplit, float a) {
    return nsplit == 0 ? launch_tc<true, true>(c, feat, gM, nullptr, 0, a)
                       : launch_tc<true, false>(c, feat, gM, nullptr, nsplit, a);
}

}  // namespace pmr

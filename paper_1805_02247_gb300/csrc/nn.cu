// The light-matter network of Sec. 2 on the mesh: three Gaussian-smoothed
// density fields (Sec. 2.2), the 3x3x3 neighbourhood of each voxel (81 inputs),
// two ReLU layers of 50 and 30 units and a softplus output (Sec. 2.1), and
// its input gradient for the adjoint.
//
// Float32 path: one thread per voxel, the 81 inputs staged with their halo in
// shared memory, all 5661 weights passed by value in the kernel parameter
// space (constant bank) so every FMA takes its weight as a constant operand
// and concurrent launches with different weights cannot interfere.
#include <algorithm>

#include "common.cuh"

namespace pmr {
namespace {

constexpr int NI = 81, H1 = 50, H2 = 30;
constexpr int OFF_B1 = H1 * NI, OFF_W2 = OFF_B1 + H1, OFF_B2 = OFF_W2 + H2 * H1, OFF_W3 = OFF_B2 + H2,
              OFF_B3 = OFF_W3 + H2, NW = OFF_B3 + 1;

struct Weights {
    float w[NW + kMassWeights];  // trunk, then the mass network (two-network head)
};

// tile of voxels per block, z fastest
constexpr int TX = 4, TY = 8, TZ = 8, HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int kT = TX * TY * TZ;

__device__ __forceinline__ int wrapi(int v, int N) { return v < 0 ? v + N : (v >= N ? v - N : v); }

// Stage the three fields on the (TX+2)(TY+2)(TZ+2) halo tile.
__device__ __forceinline__ void load_tile(float* s, const float* __restrict__ f, int N, int64_t N3, int x0, int y0,
                                          int z0) {
    for (int t = threadIdx.x; t < 3 * HX * HY * HZ; t += blockDim.x) {
        int c = t / (HX * HY * HZ), r = t % (HX * HY * HZ);
        int hx = r / (HY * HZ), hy = (r / HZ) % HY, hz = r % HZ;
        int gx = wrapi(x0 + hx - 1, N), gy = wrapi(y0 + hy - 1, N), gz = wrapi(z0 + hz - 1, N);
        s[t] = f[c * N3 + ((int64_t)gx * N + gy) * N + gz];
    }
}

__device__ __forceinline__ float softplusf(float y) { return y > 0.f ? y + log1pf(expf(-y)) : log1pf(expf(y)); }
__device__ __forceinline__ float sigmoidf(float y) {
    return y >= 0.f ? 1.f / (1.f + expf(-y)) : expf(y) / (1.f + expf(y));
}

// First layer pre-activations a1 = W1 v + b1 from the staged tile.
__device__ __forceinline__ void layer1(const Weights& W, const float* s, int lx, int ly, int lz, float* a1) {
#pragma unroll
    for (int h = 0; h < H1; ++h) a1[h] = W.w[OFF_B1 + h];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int ox = 0; ox < 3; ++ox)
#pragma unroll
            for (int oy = 0; oy < 3; ++oy)
#pragma unroll
                for (int oz = 0; oz < 3; ++oz) {
                    const int k = c * 27 + ox * 9 + oy * 3 + oz;
                    const float v = s[((c * HX + lx + ox) * HY + ly + oy) * HZ + lz + oz];
#pragma unroll
                    for (int h = 0; h < H1; ++h) a1[h] = fmaf(W.w[h * NI + k], v, a1[h]);
                }
}

__device__ __forceinline__ void layer2(const Weights& W, const float* a1, float* a2) {
#pragma unroll
    for (int h = 0; h < H2; ++h) a2[h] = W.w[OFF_B2 + h];
#pragma unroll
    for (int i = 0; i < H1; ++i) {
        const float z = fmaxf(a1[i], 0.f);
#pragma unroll
        for (int h = 0; h < H2; ++h) a2[h] = fmaf(W.w[OFF_W2 + h * H1 + i], z, a2[h]);
    }
}

__device__ __forceinline__ float layer3(const Weights& W, const float* a2) {
    float y = W.w[OFF_B3];
#pragma unroll
    for (int h = 0; h < H2; ++h) y = fmaf(W.w[OFF_W3 + h], fmaxf(a2[h], 0.f), y);
    return y;
}

// the voxel's own three field values (centre of the staged tile)
__device__ __forceinline__ void centre(const float* s, int lx, int ly, int lz, float f[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] = s[((c * HX + lx + 1) * HY + ly + 1) * HZ + lz + 1];
}

__global__ void __launch_bounds__(kT) k_mlp_fwd(const Weights W, const float* __restrict__ feat, int N, float M_scale,
                                                int head, float a, float* __restrict__ M) {
    __shared__ float s[3 * HX * HY * HZ];
    const int64_t N3 = (int64_t)N * N * N;
    const int x0 = blockIdx.z * TX, y0 = blockIdx.y * TY, z0 = blockIdx.x * TZ;
    load_tile(s, feat, N, N3, x0, y0, z0);
    __syncthreads();
    const int lx = threadIdx.x / (TY * TZ), ly = (threadIdx.x / TZ) % TY, lz = threadIdx.x % TZ;
    const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
    if (gx >= N || gy >= N || gz >= N) return;
    float a1[H1], a2[H2];
    layer1(W, s, lx, ly, lz, a1);
    layer2(W, a1, a2);
    const float y = layer3(W, a2);
    float out;
    if (head == 1) {
        float f[3];
        centre(s, lx, ly, lz, f);
        float u0, u1, u2;
        out = M_scale * sigmoidf(a * y) * mass_net<false>(W.w + NW, f[0], f[1], f[2], 0.f, u0, u1, u2);
    } else {
        out = M_scale * softplusf(y);
    }
    M[((int64_t)gx * N + gy) * N + gz] = out;
}

// Per voxel: recompute the forward, back-propagate gM to the 81 inputs and
// write them to gv[81][N3] (each input row is later gathered to its voxel).
__global__ void __launch_bounds__(kT) k_mlp_bwd(const Weights W, const float* __restrict__ feat,
                                                const float* __restrict__ gM, int N, float M_scale, int head,
                                                float a, float* __restrict__ gv) {
    __shared__ float s[3 * HX * HY * HZ];
    const int64_t N3 = (int64_t)N * N * N;
    const int x0 = blockIdx.z * TX, y0 = blockIdx.y * TY, z0 = blockIdx.x * TZ;
    load_tile(s, feat, N, N3, x0, y0, z0);
    __syncthreads();
    const int lx = threadIdx.x / (TY * TZ), ly = (threadIdx.x / TZ) % TY, lz = threadIdx.x % TZ;
    const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
    if (gx >= N || gy >= N || gz >= N) return;
    const int64_t vox = ((int64_t)gx * N + gy) * N + gz;
    float a1[H1], a2[H2];
    layer1(W, s, lx, ly, lz, a1);
    layer2(W, a1, a2);
    const float y = layer3(W, a2);
    float gy_, gc[3] = {0.f, 0.f, 0.f};
    if (head == 1) {
        // M = M_scale p m: dM/dy = M_scale m a p (1 - p); dM/dm = M_scale p
        float f[3];
        centre(s, lx, ly, lz, f);
        const float p = sigmoidf(a * y), g = gM[vox] * M_scale;
        const float m = mass_net<true>(W.w + NW, f[0], f[1], f[2], g * p, gc[0], gc[1], gc[2]);
        gy_ = g * m * a * p * (1.f - p);
    } else {
        gy_ = gM[vox] * M_scale * sigmoidf(y);
    }
    float g2[H2];
#pragma unroll
    for (int h = 0; h < H2; ++h) g2[h] = a2[h] > 0.f ? W.w[OFF_W3 + h] * gy_ : 0.f;
    float g1[H1];
#pragma unroll
    for (int i = 0; i < H1; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int h = 0; h < H2; ++h) acc = fmaf(W.w[OFF_W2 + h * H1 + i], g2[h], acc);
        g1[i] = a1[i] > 0.f ? acc : 0.f;
    }
#pragma unroll
    for (int k = 0; k < NI; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int h = 0; h < H1; ++h) acc = fmaf(W.w[h * NI + k], g1[h], acc);
        if (k % 27 == 13) acc += gc[k / 27];  // the mass network reads the centre values
        gv[k * N3 + vox] = acc;
    }
}

// g_c(y) = sum_o gv[c*27 + o](y - o): the transpose of the stencil gather.
__global__ void k_stencil_T(const float* __restrict__ gv, int N, float* __restrict__ gfeat) {
    const int64_t N3 = (int64_t)N * N * N;
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    const int x = (int)(v / ((int64_t)N * N)), y = (int)((v / N) % N), z = (int)(v % N);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int ox = -1; ox <= 1; ++ox)
#pragma unroll
            for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
                for (int oz = -1; oz <= 1; ++oz) {
                    const int k = c * 27 + (ox + 1) * 9 + (oy + 1) * 3 + (oz + 1);
                    const int64_t src = ((int64_t)wrapi(x - ox, N) * N + wrapi(y - oy, N)) * N + wrapi(z - oz, N);
                    acc += gv[k * N3 + src];
                }
        gfeat[c * N3 + v] = acc;
    }
}

dim3 mlp_grid(int N) { return dim3((N + TZ - 1) / TZ, (N + TY - 1) / TY, (N + TX - 1) / TX); }

}  // namespace

int nn_features(pmr_ctx* c, const float* delta) {
    const double cell = c->cfg.L / c->N;
    Mul mul[3];
    for (int j = 0; j < 3; ++j) {
        const double R = c->cfg.R_feat[j] / cell;
        mul[j] = Mul{R > 0 ? MUL_GAUSS : MUL_ONE, 0, 1.0f, (float)(R * R), 0};
    }
    float* outs[3] = {c->feat, c->feat + c->N3, c->feat + 2 * c->N3};
    return conv_1toN(c, delta, outs, mul, 3);
}

static_assert(sizeof(Weights) <= 32000, "weights must fit the kernel parameter space");

// tensor-core operand mode of nn_path: 0 -> TF32 head/tail (3 products), 1 -> TF32, 3 -> bf16
int tc_split(const pmr_ctx* c) { return c->cfg.nn_path == 0 ? 3 : (c->cfg.nn_path == 1 ? 1 : 0); }

// nn_path 0: tensor cores, 3xTF32 (float32 accuracy); 1: tensor cores, TF32;
// 2: float32 CUDA cores.
int mlp_forward(pmr_ctx* c, const float* feat, float* M, float a) {
    if (c->cfg.nn_path != 2) return mlp_tc_forward(c, feat, M, tc_split(c), a);
    static_assert(NW == 5661, "weight layout");
    Weights W;
    std::copy(c->W_host.begin(), c->W_host.begin() + (NW + kMassWeights), W.w);
    k_mlp_fwd<<<mlp_grid(c->N), kT, 0, c->stream>>>(W, feat, c->N, (float)c->cfg.M_scale, c->cfg.head, a, M);
    return check_launch(c, "mlp_fwd");
}

int stencil_transpose(pmr_ctx* c, const float* gv, float* gfeat) {
    k_stencil_T<<<nblocks(c->N3, 256), 256, 0, c->stream>>>(gv, c->N, gfeat);
    return check_launch(c, "stencil_T");
}

int mlp_backward(pmr_ctx* c, const float* feat, const float* gM, float* gfeat, float a) {
    if (c->cfg.nn_path != 2) {
        PMR_TRY(mlp_tc_backward_gv(c, feat, gM, tc_split(c), a));
        return stencil_tiles(c, gfeat);
    }
    Weights W;
    std::copy(c->W_host.begin(), c->W_host.begin() + (NW + kMassWeights), W.w);
    k_mlp_bwd<<<mlp_grid(c->N), kT, 0, c->stream>>>(W, feat, gM, c->N, (float)c->cfg.M_scale, c->cfg.head, a,
                                                     c->gv);
    PMR_TRY(check_launch(c, "mlp_bwd"));
    return stencil_transpose(c, c->gv, gfeat);
}

}  // namespace pmr

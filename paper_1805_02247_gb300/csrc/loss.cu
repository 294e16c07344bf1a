// Loss of Eq. (loss) (Sec. 5.1): the Gaussian prior of Eq. (priorpdf) on the
// half-array modes and the smoothed displaced-log-normal residual of
// Eq. (probnoise), with the annealed residual smoothing of Sec. 5.2, plus the
// elementwise parts of their gradients. Sums are float64 and deterministic:
// a fixed grid accumulates per-block partials that one block adds in order.
#include <cmath>

#include "common.cuh"

namespace pmr {
namespace {

constexpr int kRT = 256;
constexpr int kRB = 1024;  // reduction blocks (fixed => fixed summation order)

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
    }
    return t;  // valid in thread 0
}

__global__ void k_sumsq_part(const float* __restrict__ v, int64_t n, double* __restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x = v[i];
        acc += x * x;
    }
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// out[slot] = scale * sum(part)
__global__ void k_final(const double* __restrict__ part, int nb, double scale, double* __restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[i];
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = scale * t;
}

// prior: 1/2 sum_half w |s|^2 / P~ (k != 0)
__global__ void k_prior_part(const float2* __restrict__ s, int N, int P, const double* __restrict__ inv_pow,
                             double* __restrict__ part) {
    __shared__ double sh[32];
    const int64_t NH = (int64_t)N * N * P;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < NH; i += (int64_t)gridDim.x * blockDim.x) {
        const int kz = (int)(i % P);
        const int iy = (int)((i / P) % N), ix = (int)(i / ((int64_t)P * N));
        const int nx = (2 * ix <= N) ? ix : ix - N, ny = (2 * iy <= N) ? iy : iy - N;
        const float w = (kz == 0 || 2 * kz == N) ? 1.0f : 2.0f;
        const float2 v = s[i];
        // per-mode term in float32, accumulated in float64
        acc += (double)(w * (v.x * v.x + v.y * v.y) * (float)inv_pow[nx * nx + ny * ny + kz * kz]);
    }
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// grad += w s / P~ (k != 0); grad(0) = 0
__global__ void k_prior_grad(const float2* __restrict__ s, float2* __restrict__ g, int N, int P,
                             const double* __restrict__ inv_pow) {
    const int64_t NH = (int64_t)N * N * P;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NH) return;
    const int kz = (int)(i % P);
    const int iy = (int)((i / P) % N), ix = (int)(i / ((int64_t)P * N));
    const int nx = (2 * ix <= N) ? ix : ix - N, ny = (2 * iy <= N) ? iy : iy - N;
    const int n2 = nx * nx + ny * ny + kz * kz;
    if (n2 == 0) {
        g[i] = make_float2(0.f, 0.f);
        return;
    }
    const float w = (kz == 0 || 2 * kz == N) ? 1.0f : 2.0f;
    const float f = w * (float)inv_pow[n2];
    const float2 v = s[i];
    float2 o = g[i];
    o.x = fmaf(f, v.x, o.x);
    o.y = fmaf(f, v.y, o.y);
    g[i] = o;
}

// r = mu + log(M_R + M0) - log(D_R + M0), evaluated as mu + log1p((M_R - D_R) / (D_R + M0))
// so that float32 keeps the residual's relative precision (the two logs are
// ~28 and differ by O(0.1)).
__global__ void k_log_residual(const float* __restrict__ MR, const float* __restrict__ DR, int64_t n, float mu,
                               float M0, float* __restrict__ r) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = MR[i], b = DR[i];
    r[i] = mu + log1pf((a - b) / (b + M0));
}

// g_MR = c * g / (M_R + M0)
__global__ void k_div_mass(float* __restrict__ g, const float* __restrict__ MR, int64_t n, float cst, float M0) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    g[i] = cst * g[i] / (MR[i] + M0);
}

}  // namespace

int reduce_sum_sq(pmr_ctx* c, const float* v, int64_t n, double scale, double* out_dev) {
    k_sumsq_part<<<kRB, kRT, 0, c->stream>>>(v, n, c->red_part);
    PMR_TRY(check_launch(c, "sumsq"));
    k_final<<<1, kRT, 0, c->stream>>>(c->red_part, kRB, scale, out_dev);
    return check_launch(c, "final");
}

int prior_value(pmr_ctx* c, const float2* s, double* out_dev) {
    k_prior_part<<<kRB, kRT, 0, c->stream>>>(s, c->N, c->P, c->inv_power_tab, c->red_part);
    PMR_TRY(check_launch(c, "prior"));
    k_final<<<1, kRT, 0, c->stream>>>(c->red_part, kRB, 0.5, out_dev);
    return check_launch(c, "final");
}

int prior_grad_add(pmr_ctx* c, const float2* s, float2* grad) {
    k_prior_grad<<<nblocks(c->NH, kRT), kRT, 0, c->stream>>>(s, grad, c->N, c->P, c->inv_power_tab);
    return check_launch(c, "prior_grad");
}

static Mul gauss_mul(const pmr_ctx* c, double R_mpc) {
    const double R = R_mpc / (c->cfg.L / c->N);
    return Mul{R > 0 ? MUL_GAUSS : MUL_ONE, 0, 1.0f, (float)(R * R), 0};
}

static int smooth_into(pmr_ctx* c, const float* in, double R_mpc, float* out) {
    if (R_mpc <= 0.0) {
        if (in == out) return PMR_OK;
        return check_cuda(c, cudaMemcpyAsync(out, in, sizeof(float) * c->N3, cudaMemcpyDeviceToDevice, c->stream),
                          "copy");
    }
    Mul m = gauss_mul(c, R_mpc);
    float* outs[1] = {out};
    return conv_1toN(c, in, outs, &m, 1);
}

// Forward residual: c->M holds M_NN. Leaves M_R in c->MR and r_s in c->rs.
int residual_forward(pmr_ctx* c, const float* data, const pmr_anneal* an, double* L_res_dev) {
    PMR_TRY(smooth_into(c, c->M, c->cfg.R_M, c->MR));
    PMR_TRY(smooth_into(c, data, c->cfg.R_M, c->DR));
    k_log_residual<<<nblocks(c->N3, kRT), kRT, 0, c->stream>>>(c->MR, c->DR, c->N3, (float)c->cfg.mu_N,
                                                                (float)an->M0, c->gm);
    PMR_TRY(check_launch(c, "log_residual"));
    PMR_TRY(smooth_into(c, c->gm, an->R_sm, c->rs));
    return reduce_sum_sq(c, c->rs, c->N3, c->cfg.f_eff / (4.0 * c->cfg.sigma_N2), L_res_dev);
}

// dL_res/dM_NN = S_RM [ (f_eff / (2 sigma^2)) S_Rsm(r_s) / (M_R + M0) ]
int residual_backward(pmr_ctx* c, const pmr_anneal* an, float* gM) {
    PMR_TRY(smooth_into(c, c->rs, an->R_sm, c->gm));
    k_div_mass<<<nblocks(c->N3, kRT), kRT, 0, c->stream>>>(c->gm, c->MR, c->N3,
                                                            (float)(c->cfg.f_eff / (2.0 * c->cfg.sigma_N2)),
                                                            (float)an->M0);
    PMR_TRY(check_launch(c, "div_mass"));
    return smooth_into(c, c->gm, c->cfg.R_M, gM);
}

namespace {
__global__ void k_loss_out(const double* __restrict__ red, double* __restrict__ out) {
    if (threadIdx.x == 0) {
        out[0] = red[0] + red[1];
        out[1] = red[0];
        out[2] = red[1];
    }
}
}  // namespace

// {total, prior, residual} of the last evaluation into a device array, on the stream
int loss_to_device(pmr_ctx* c, double* out_dev) {
    k_loss_out<<<1, 32, 0, c->stream>>>(c->red_out, out_dev);
    return check_launch(c, "loss_out");
}

int check_finite(pmr_ctx* c, const double* v, int n, double* host) {
    PMR_TRY(check_cuda(c, cudaMemcpyAsync(host, v, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "readback"));
    PMR_TRY(check_cuda(c, cudaStreamSynchronize(c->stream), "sync"));
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(host[i])) return fail(c, PMR_ENAN, "loss is not finite (is M_R + M0 > 0 everywhere?)");
    return PMR_OK;
}

}  // namespace pmr

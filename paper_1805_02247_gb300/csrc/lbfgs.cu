// L-BFGS (Sec. 5.2) on the device in float64: deterministic dot products and
// the two-loop recursion with every scalar kept on the device, so a direction
// costs no host round trip. Vectors are the half-array modes viewed as 2*NH
// reals (real and imaginary parts are independent variables, Sec. 5.1).
#include "common.cuh"

namespace pmr {
namespace {

constexpr int kT = 256;
constexpr int kB = 1024;

__global__ void k_dot_part(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                           double* __restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(a[i], b[i], acc);
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        double t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
        if (lane == 0) part[blockIdx.x] = t;
    }
}

__global__ void k_dot_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[i];
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        double t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
        if (lane == 0) *out = t;
    }
}

// Coefficient forms used by the recursion (all scalars device-resident):
//  mode 0 (first loop):  alpha_i = rho_i * dot;  q -= alpha_i * y_i
//  mode 1 (second loop): beta = rho_i * dot;     r += (alpha_i - beta) * s_i
//  mode 2 (scaling):     r = (sy / yy) * q       (dot = sy, dot2 = yy)
//  mode 3:               d = -r
__global__ void k_two_loop_axpy(double* __restrict__ y, const double* __restrict__ x, int64_t n, int mode,
                                const double* __restrict__ dot, const double* __restrict__ dot2, double rho,
                                double* __restrict__ alpha_slot) {
    double coef;
    if (mode == 0) coef = -rho * (*dot);
    else if (mode == 1) coef = (*alpha_slot) - rho * (*dot);
    else if (mode == 2) coef = (*dot) / (*dot2);
    else coef = -1.0;
    if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) *alpha_slot = rho * (*dot);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (mode == 0 || mode == 1) y[i] = fma(coef, x[i], y[i]);
        else y[i] = coef * x[i];
    }
}

__global__ void k_c64_to_f64(const float* __restrict__ a, double* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)a[i];
}

__global__ void k_f64_to_c64(const double* __restrict__ a, float* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)a[i];
}

// y = base + alpha * x  (alpha from device or host)
__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ alpha_dev,
                       double alpha_host, int64_t n, const double* __restrict__ base) {
    const double a = alpha_dev ? *alpha_dev : alpha_host;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], base ? base[i] : y[i]);
}

constexpr int kGrid = 4 * 152;

// y = scale * D x with D = P~(k) / w_k on every (real, imaginary) entry of the
// half array (0 at k = 0): the Gaussian prior's inverse Hessian.
__global__ void k_prior_h0(double* __restrict__ y, const double* __restrict__ x, int64_t nreal, int N, FastDiv fP,
                           FastDiv fN, const double* __restrict__ inv_pow, double scale) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nreal; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(j >> 1);
        const uint32_t t = fP.div(i);
        const int kz = (int)(i - t * fP.d);
        const uint32_t ixu = fN.div(t);
        const int iy = (int)(t - ixu * fN.d), ix = (int)ixu;
        const int nx = 2 * ix <= N ? ix : ix - N, ny = 2 * iy <= N ? iy : iy - N;
        const double ip = inv_pow[nx * nx + ny * ny + kz * kz];
        const double w = (kz == 0 || 2 * kz == N) ? 1.0 : 2.0;
        y[j] = ip > 0.0 ? scale * x[j] / (w * ip) : 0.0;
    }
}

}  // namespace

int prior_h0_apply(pmr_ctx* c, double* y, const double* x, double scale) {
    k_prior_h0<<<kGrid, kT, 0, c->stream>>>(y, x, 2 * c->NH, c->N, FastDiv((uint32_t)c->P), FastDiv((uint32_t)c->N),
                                             c->inv_power_tab, scale);
    return check_launch(c, "prior_h0");
}

int dot64(pmr_ctx* c, const double* a, const double* b, int64_t n, double* out_dev) {
    k_dot_part<<<kB, kT, 0, c->stream>>>(a, b, n, c->red_part);
    PMR_TRY(check_launch(c, "dot_part"));
    k_dot_final<<<1, kT, 0, c->stream>>>(c->red_part, kB, out_dev);
    return check_launch(c, "dot_final");
}

int c64_to_f64(pmr_ctx* c, const float2* a, double* out, int64_t nh) {
    k_c64_to_f64<<<nblocks(2 * nh, kT), kT, 0, c->stream>>>(reinterpret_cast<const float*>(a), out, 2 * nh);
    return check_launch(c, "c64_to_f64");
}

int f64_to_c64(pmr_ctx* c, const double* a, float2* out, int64_t nh) {
    k_f64_to_c64<<<nblocks(2 * nh, kT), kT, 0, c->stream>>>(a, reinterpret_cast<float*>(out), 2 * nh);
    return check_launch(c, "f64_to_c64");
}

int axpy64(pmr_ctx* c, double* y, const double* x, const double* alpha_dev, double alpha_host, int64_t n,
           const double* base) {
    k_axpy<<<kGrid, kT, 0, c->stream>>>(y, x, alpha_dev, alpha_host, n, base);
    return check_launch(c, "axpy");
}

// d = -H g. S, Y are rings of capacity m: pair t (0 = oldest) sits in slot (head + t) % m.
// rho_host[slot] = 1 / (s.y) of that slot.
int lbfgs_two_loop(pmr_ctx* c, const double* g, const double* S, const double* Y, int k, int head, int m, int64_t n,
                   const double* rho_host, double* d, bool prior_h0) {
    double* q = d;
    double* sc = c->lb.scal;  // [0]: dot, [1]: dot2
    PMR_TRY(check_cuda(c, cudaMemcpyAsync(q, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "copy"));
    for (int t = k - 1; t >= 0; --t) {
        const int slot = (head + t) % m;
        PMR_TRY(dot64(c, S + (int64_t)slot * n, q, n, sc));
        k_two_loop_axpy<<<kGrid, kT, 0, c->stream>>>(q, Y + (int64_t)slot * n, n, 0, sc, nullptr,
                                                    rho_host[slot], c->lb.alpha + slot);
        PMR_TRY(check_launch(c, "two_loop_0"));
    }
    const int newest = (head + k - 1) % m;
    if (prior_h0) {
        // r = gamma D q, gamma = s^T y / y^T D y of the newest pair; lb.yk is free
        // scratch here (it holds the candidate pair only after the line search)
        double* Dy = c->lb.yk;
        PMR_TRY(prior_h0_apply(c, Dy, Y + (int64_t)newest * n, 1.0));
        PMR_TRY(dot64(c, S + (int64_t)newest * n, Y + (int64_t)newest * n, n, sc));
        PMR_TRY(dot64(c, Y + (int64_t)newest * n, Dy, n, sc + 1));
        PMR_TRY(prior_h0_apply(c, q, q, 1.0));
        k_two_loop_axpy<<<kGrid, kT, 0, c->stream>>>(q, q, n, 2, sc, sc + 1, 0.0, nullptr);
        PMR_TRY(check_launch(c, "two_loop_scale"));
    } else {
        PMR_TRY(dot64(c, S + (int64_t)newest * n, Y + (int64_t)newest * n, n, sc));
        PMR_TRY(dot64(c, Y + (int64_t)newest * n, Y + (int64_t)newest * n, n, sc + 1));
        k_two_loop_axpy<<<kGrid, kT, 0, c->stream>>>(q, q, n, 2, sc, sc + 1, 0.0, nullptr);
        PMR_TRY(check_launch(c, "two_loop_scale"));
    }
    for (int t = 0; t < k; ++t) {
        const int slot = (head + t) % m;
        PMR_TRY(dot64(c, Y + (int64_t)slot * n, q, n, sc));
        k_two_loop_axpy<<<kGrid, kT, 0, c->stream>>>(q, S + (int64_t)slot * n, n, 1, sc, nullptr,
                                                    rho_host[slot], c->lb.alpha + slot);
        PMR_TRY(check_launch(c, "two_loop_1"));
    }
    k_two_loop_axpy<<<kGrid, kT, 0, c->stream>>>(q, q, n, 3, nullptr, nullptr, 0.0, nullptr);
    return check_launch(c, "two_loop_neg");
}

int lbfgs_alloc(pmr_ctx* c) {
    pmr::LBFGS& L = c->lb;
    L.m = c->cfg.lbfgs_m;
    L.n = 2 * c->NH;
    const size_t v = sizeof(double) * (size_t)L.n;
    PMR_TRY(check_cuda(c, cudaMalloc(&L.x, v), "lbfgs"));
    PMR_TRY(check_cuda(c, cudaMalloc(&L.g, v), "lbfgs"));
    PMR_TRY(check_cuda(c, cudaMalloc(&L.d, v), "lbfgs"));
    PMR_TRY(check_cuda(c, cudaMalloc(&L.xt, v), "lbfgs"));
    PMR_TRY(check_cuda(c, cudaMalloc(&L.gt, v), "lbfgs"));
    PMR_TRY(check_cuda(c, cudaMalloc(&L.yk, v), "lbfgs"));
    PMR_TRY(check_cuda(c, cudaMalloc(&L.S, v * L.m), "lbfgs"));
    PMR_TRY(check_cuda(c, cudaMalloc(&L.Y, v * L.m), "lbfgs"));
    PMR_TRY(check_cuda(c, cudaMalloc(&L.alpha, sizeof(double) * L.m), "lbfgs"));
    PMR_TRY(check_cuda(c, cudaMalloc(&L.scal, sizeof(double) * 8), "lbfgs"));
    PMR_TRY(check_cuda(c, cudaMalloc(&L.gk, sizeof(float2) * c->NH), "lbfgs"));
    L.rho_host.assign(L.m, 0.0);
    return PMR_OK;
}

void lbfgs_free(pmr_ctx* c) {
    pmr::LBFGS& L = c->lb;
    for (double* p : {L.x, L.g, L.d, L.xt, L.gt, L.yk, L.S, L.Y, L.alpha, L.scal}) cudaFree(p);
    cudaFree(L.gk);
    L = pmr::LBFGS{};
}

}  // namespace pmr

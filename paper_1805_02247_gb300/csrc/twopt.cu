// Two-point statistics of Sec. 4.3 on the GPU: binned auto and cross power
// spectra of two mesh fields, from which r_c = P_hN / sqrt(P_hh P_NN),
// s = P_hh (1 - r_c^2) and TF = sqrt(P_NN / P_hh) follow.
//
// Shell i holds the modes with integer wavevector norm i + 1/2 <= |n| < i + 3/2
// (k = 2 pi n / L), i < N/2. The half-array entries of each shell are listed
// once per context (host counting sort by shell); one block per shell then
// sums its modes in a fixed order in float64, so the result is deterministic.
#include <cmath>

#include "common.cuh"

namespace pmr {
namespace {

constexpr int kT = 256;

__global__ void __launch_bounds__(kT) k_shell_reduce(const float2* __restrict__ A, const float2* __restrict__ B,
                                                     const uint32_t* __restrict__ order,
                                                     const uint32_t* __restrict__ off, int P, int N,
                                                     double* __restrict__ out) {
    __shared__ double sh[4][kT / 32];
    const int b = blockIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (uint32_t j = off[b] + threadIdx.x; j < off[b + 1]; j += kT) {
        const uint32_t idx = order[j];
        const int kz = (int)(idx % (uint32_t)P);
        const double w = (kz == 0 || 2 * kz == N) ? 1.0 : 2.0;
        const float2 a = A[idx], c = B[idx];
        acc[0] += w;
        acc[1] += w * ((double)a.x * a.x + (double)a.y * a.y);
        acc[2] += w * ((double)c.x * c.x + (double)c.y * c.y);
        acc[3] += w * ((double)a.x * c.x + (double)a.y * c.y);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double v = acc[q];
        for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
        if (lane == 0) sh[q][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < kT / 32; ++w) v += sh[threadIdx.x][w];
        out[threadIdx.x * gridDim.x + b] = v;
    }
}

// list the half-array entries of each shell (ascending index inside a shell)
int build_shells(pmr_ctx* c) {
    if (c->shell_order) return PMR_OK;
    const int N = c->N, P = c->P, nb = N / 2;
    std::vector<uint32_t> cnt(nb + 1, 0), shell((size_t)c->NH);
    for (int64_t i = 0; i < c->NH; ++i) {
        const int kz = (int)(i % P), iy = (int)((i / P) % N), ix = (int)(i / ((int64_t)P * N));
        const int nx = 2 * ix <= N ? ix : ix - N, ny = 2 * iy <= N ? iy : iy - N;
        const double r = std::sqrt((double)(nx * nx + ny * ny + kz * kz));
        const int s = (int)std::floor(r - 0.5);
        shell[i] = (s >= 0 && s < nb) ? (uint32_t)s : 0xffffffffu;
        if (shell[i] != 0xffffffffu) cnt[s + 1]++;
    }
    for (int s = 0; s < nb; ++s) cnt[s + 1] += cnt[s];
    std::vector<uint32_t> order(cnt[nb]), fill(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < c->NH; ++i)
        if (shell[i] != 0xffffffffu) order[fill[shell[i]]++] = (uint32_t)i;
    PMR_TRY(check_cuda(c, cudaMalloc(&c->shell_order, sizeof(uint32_t) * order.size()), "shells"));
    PMR_TRY(check_cuda(c, cudaMalloc(&c->shell_off, sizeof(uint32_t) * (nb + 1)), "shells"));
    PMR_TRY(check_cuda(c, cudaMalloc(&c->shell_out, sizeof(double) * 4 * nb), "shells"));
    PMR_TRY(check_cuda(c, cudaMemcpy(c->shell_order, order.data(), sizeof(uint32_t) * order.size(),
                                     cudaMemcpyHostToDevice), "shells"));
    return check_cuda(c, cudaMemcpy(c->shell_off, cnt.data(), sizeof(uint32_t) * (nb + 1), cudaMemcpyHostToDevice),
                      "shells");
}

}  // namespace

void twopt_free(pmr_ctx* c) {
    cudaFree(c->shell_order);
    cudaFree(c->shell_off);
    cudaFree(c->shell_out);
    c->shell_order = c->shell_off = nullptr;
    c->shell_out = nullptr;
}

}  // namespace pmr

using namespace pmr;

extern "C" int pmr_power_spectra(pmr_ctx* c, const float* a, const float* b, double* out) {
    if (!c) return fail(nullptr, PMR_EINVAL, "context is NULL");
    if (!a || !b || !out) return fail(c, PMR_EINVAL, "NULL argument");
    PMR_TRY(build_shells(c));
    PMR_TRY(fft_r2c(c, a, c->cA));
    PMR_TRY(fft_r2c(c, b, c->cB));
    const int nb = c->N / 2;
    k_shell_reduce<<<nb, kT, 0, c->stream>>>(c->cA, c->cB, c->shell_order, c->shell_off, c->P, c->N, c->shell_out);
    PMR_TRY(check_launch(c, "shell_reduce"));
    std::vector<double> h(4 * nb);
    PMR_TRY(check_cuda(c, cudaMemcpyAsync(h.data(), c->shell_out, sizeof(double) * 4 * nb, cudaMemcpyDeviceToHost,
                                          c->stream), "readback"));
    PMR_TRY(check_cuda(c, cudaStreamSynchronize(c->stream), "sync"));
    const double norm = std::pow(c->cfg.L, 3) / std::pow((double)c->N, 6);
    for (int i = 0; i < nb; ++i) {
        const double n = h[i];
        out[i] = n;
        for (int q = 1; q < 4; ++q) out[q * nb + i] = n > 0 ? h[q * nb + i] / n * norm : 0.0;
    }
    return PMR_OK;
}

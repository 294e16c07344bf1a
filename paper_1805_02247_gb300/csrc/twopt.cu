// Two-point statistics of Sec. 4.3 on the GPU: binned auto and cross power
// spectra of two mesh fields, from which r_c = P_hN / sqrt(P_hh P_NN),
// s = P_hh (1 - r_c^2) and TF = sqrt(P_NN / P_hh) follow.
//
// Shell i holds the modes with integer wavevector norm i + 1/2 <= |n| < i + 3/2
// (k = 2 pi n / L), i < N/2. The half-array entries of each shell are listed
// once per context (host counting sort by shell); one block per shell then
// sums its modes in a fixed order in float64, so the result is deterministic,
// and one thread per shell forms the spectra and the statistics.
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

// Per shell, from the sums: mode count, the three spectra P = sum / count * L^3 / N^6,
// and r_c = P_ab / sqrt(P_aa P_bb), s = P_aa (1 - r_c^2), TF = sqrt(P_bb / P_aa)
// (a = h, the truth or data; b = N, the model). Rows of out: [7][nb]. A shell
// without modes gives zero spectra; a zero spectrum gives NaN statistics (0/0).
__global__ void k_shell_stats(double* __restrict__ sums, int nb, double norm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    const double n = sums[i];
    double P[3];
    for (int q = 0; q < 3; ++q) P[q] = n > 0 ? sums[(q + 1) * nb + i] / n * norm : 0.0;
    const double rc = P[2] / sqrt(P[0] * P[1]);
    for (int q = 0; q < 3; ++q) sums[(q + 1) * nb + i] = P[q];
    sums[4 * nb + i] = rc;
    sums[5 * nb + i] = P[0] * (1.0 - rc * rc);
    sums[6 * nb + i] = sqrt(P[1] / P[0]);
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
    PMR_TRY(check_cuda(c, cudaMalloc(&c->shell_out, sizeof(double) * 7 * nb), "shells"));
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

namespace {

// spectra and statistics of Sec. 4.3 into c->shell_out [7][N/2], then `rows` rows to the host
int two_point(pmr_ctx* c, const float* a, const float* b, double* out, int rows) {
    if (!c) return fail(nullptr, PMR_EINVAL, "context is NULL");
    if (!a || !b || !out) return fail(c, PMR_EINVAL, "NULL argument");
    PMR_TRY(build_shells(c));
    PMR_TRY(fft_r2c(c, a, c->cA));
    PMR_TRY(fft_r2c(c, b, c->cB));
    const int nb = c->N / 2;
    k_shell_reduce<<<nb, kT, 0, c->stream>>>(c->cA, c->cB, c->shell_order, c->shell_off, c->P, c->N, c->shell_out);
    PMR_TRY(check_launch(c, "shell_reduce"));
    const double norm = std::pow(c->cfg.L, 3) / std::pow((double)c->N, 6);
    k_shell_stats<<<nblocks(nb, 128), 128, 0, c->stream>>>(c->shell_out, nb, norm);
    PMR_TRY(check_launch(c, "shell_stats"));
    PMR_TRY(check_cuda(c, cudaMemcpyAsync(out, c->shell_out, sizeof(double) * rows * nb, cudaMemcpyDeviceToHost,
                                          c->stream), "readback"));
    return check_cuda(c, cudaStreamSynchronize(c->stream), "sync");
}

}  // namespace

extern "C" int pmr_power_spectra(pmr_ctx* c, const float* a, const float* b, double* out) {
    return two_point(c, a, b, out, 4);
}

extern "C" int pmr_two_point(pmr_ctx* c, const float* h, const float* m, double* out) {
    return two_point(c, h, m, out, 7);
}

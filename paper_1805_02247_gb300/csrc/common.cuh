// Shared declarations of the sm_103a reconstruction library (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "pmrecon.h"

namespace pmr {

// Division by a run-time constant d (1 <= d < 2^31) of n < 2^31 without a
// divide instruction: q = (umulhi(n, mul) + n) >> shift (Granlund-Montgomery).
struct FastDiv {
    uint32_t d, mul, shift;
    FastDiv() : d(1), mul(1), shift(0) {}
    explicit FastDiv(uint32_t dd) : d(dd) {
        uint32_t l = 0;
        while ((uint64_t(1) << l) < dd) ++l;
        shift = l;
        mul = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - dd)) / dd + 1);
    }
#ifdef __CUDACC__
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(n, mul) + n) >> shift; }
    __device__ __forceinline__ uint32_t mod(uint32_t n) const { return n - div(n) * d; }
#endif
};

// The mass network of the paper's two-network head (Sec. 2.1): 3 -> 20 -> 10
// -> 1, ELU hidden units, linear output, on the three fields at the voxel.
// Weights (301): Wm1[20][3] @0, bm1[20] @60, Wm2[10][20] @80, bm2[10] @280,
// wm3[10] @290, bm3 @300.
constexpr int kMassWeights = 301;
#ifdef __CUDACC__
__device__ __forceinline__ float elu_f(float x) { return x > 0.f ? x : expm1f(x); }
__device__ __forceinline__ float elu_grad_f(float x) { return x > 0.f ? 1.f : expf(x); }

// m = NNm(f0, f1, f2); with GRAD also g_c = gm * dm/df_c. Only the 10
// second-layer values stay live; first-layer units are recomputed as needed.
// Inlined, with scalar outputs, so no stack array or call sits in the kernels.
__device__ __forceinline__ float mass_net_l1(const float* __restrict__ w, float f0, float f1, float f2, int j) {
    return w[60 + j] + w[3 * j] * f0 + w[3 * j + 1] * f1 + w[3 * j + 2] * f2;
}

template <bool GRAD>
__device__ __forceinline__ float mass_net(const float* __restrict__ w, float f0, float f1, float f2, float gm,
                                          float& g0, float& g1, float& g2) {
    float p2[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) p2[i] = w[280 + i];
#pragma unroll 1
    for (int j = 0; j < 20; ++j) {
        const float h = elu_f(mass_net_l1(w, f0, f1, f2, j));
#pragma unroll
        for (int i = 0; i < 10; ++i) p2[i] = fmaf(w[80 + 20 * i + j], h, p2[i]);
    }
    float m = w[300];
#pragma unroll
    for (int i = 0; i < 10; ++i) m = fmaf(w[290 + i], elu_f(p2[i]), m);
    if (GRAD) {
#pragma unroll
        for (int i = 0; i < 10; ++i) p2[i] = gm * w[290 + i] * elu_grad_f(p2[i]);  // now d/d(pre-activation 2)
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 1
        for (int j = 0; j < 20; ++j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < 10; ++i) s = fmaf(w[80 + 20 * i + j], p2[i], s);
            s *= elu_grad_f(mass_net_l1(w, f0, f1, f2, j));
            a0 = fmaf(w[3 * j], s, a0);
            a1 = fmaf(w[3 * j + 1], s, a1);
            a2 = fmaf(w[3 * j + 2], s, a2);
        }
        g0 = a0;
        g1 = a1;
        g2 = a2;
    }
    return m;
}
#endif

// Radix schedule of a 1D FFT of length n (Stockham autosort, radices 4/3/2),
// with the per-stage divisors the butterflies need.
struct Radix {
    int n;
    int nr;
    int r[12];
    FastDiv ns[12];   // Ns of stage s (product of the earlier radices)
    FastDiv nrd[12];  // n / r[s]
};

Radix make_radix(int n);
bool radix_ok(int n);

// Fourier-space multiplier applied inside the fused x-pass.
enum MulType : int { MUL_ONE = 0, MUL_GAUSS = 1, MUL_ODD = 2, MUL_POWER = 3, MUL_HESS = 4 };
struct Mul {
    int type;     // MulType
    int j;        // component for MUL_ODD (0=x, 1=y, 2=z)
    float scale;  // overall factor
    float R2;     // Gaussian: R^2 in grid units
    int weighted; // multiply by the half-array weight w(kz) (2 interior, 1 on kz=0, N/2)
    int i2;       // second component for MUL_HESS (k_j k_i2 / k^2)
};

struct FFTPlan {
    int N = 0, M = 0, P = 0;
    Radix rN{}, rM{};
    float2* twN = nullptr;  // exp(-2 pi i t / N), t < N (device)
    float2* twM = nullptr;  // exp(-2 pi i t / M), t < M (device)
};

// Stored L-BFGS history on the device (float64), oldest first in a ring.
struct LBFGS {
    int m = 0, k = 0, head = 0;  // capacity, stored pairs, slot of the oldest pair
    int64_t n = 0;               // real dof (2 * N * N * P)
    double* x = nullptr;         // current point (float64 master copy)
    double* g = nullptr;         // gradient at x
    double* d = nullptr;         // direction
    double* xt = nullptr;        // trial point
    double* gt = nullptr;        // gradient at the trial point
    double* yk = nullptr;        // candidate correction pair (s in d, y here)
    double* S = nullptr;         // [m][n]
    double* Y = nullptr;         // [m][n]
    double* alpha = nullptr;     // [m] first-loop coefficients (device)
    double* scal = nullptr;      // device scalars (dots)
    float2* gk = nullptr;        // float32 gradient of the last evaluation (half array)
    std::vector<double> rho_host;  // 1 / (s.y) per slot
    bool have_f = false;
    double f = 0, f_prior = 0, f_res = 0;
    pmr_anneal an{};
};

}  // namespace pmr

struct pmr_ctx {
    pmr_config cfg{};
    cudaStream_t stream = nullptr;
    std::string err;
    int device = 0;

    int N = 0, P = 0;
    int64_t N3 = 0, NH = 0;  // N^3 real cells, N*N*P complex entries

    // growth and stepping (host, float64)
    double D0 = 0, Gp0 = 0;
    double D2_0 = 0, Gp2_0 = 0;  // second-order LPT growth at a0 (lpt_order == 2)
    float* lpt_H = nullptr;      // [6][N^3] phi_xx, phi_yy, phi_zz, phi_xy, phi_xz, phi_yz of the last ICs
    float* lpt_G = nullptr;      // [6][N^3] their adjoint
    std::vector<double> kick, drift;

    pmr::FFTPlan plan;
    float* power_tab = nullptr;     // sqrt(P~/N^3) by integer |n|^2 (device, float32)
    double* inv_power_tab = nullptr; // 1/P~ by integer |n|^2 (device, float64; 0 at n=0)
    int ntab = 0;

    float* W = nullptr;  // network weights (device copy)
    std::vector<float> W_host;  // same, on the host (launch parameters)
    uint32_t* shell_order = nullptr;  // half-array entries listed by |k| shell (two-point statistics)
    uint32_t* shell_off = nullptr;
    double* shell_out = nullptr;
    float* tc_img = nullptr;    // tensor-core operand images of the weights (TF32 head + tail)
    float* tc_img_bf = nullptr; // the same as bfloat16
    int* tc_err = nullptr;      // set by a tensor-core kernel whose barrier wait timed out
    bool tc_stall = false;      // failure-detection test hook: tensor-core kernels issue no MMAs
    int num_sms = 0;

    // particle state: displacement from the lattice point, [3][N3]
    float* disp = nullptr;  // (nsteps+1) checkpoints, [step][3][N3]
    float* mom = nullptr;   // [3][N3]
    float* lam_x = nullptr;
    float* lam_p = nullptr;
    bool have_forward = false;
    int64_t fwd_id = 0;  // counts completed forward sweeps (pmr_forward_id)

    // cell sort
    uint32_t* keys = nullptr;
    uint32_t* perm = nullptr;
    uint32_t* cell_start = nullptr;  // N3 + 1
    uint32_t* counts = nullptr;      // N3
    uint32_t* scan_part = nullptr;
    uint32_t* long_list = nullptr;   // cells whose segment needs the block sort
    uint32_t* long_count = nullptr;
    uint32_t* sort_tmp = nullptr;    // N3 scratch for the block sort
    // per-step sort of the path's positions, kept from the forward sweep for the
    // adjoint: slot s holds perm [N3] and cell offsets [N3 + 1] of x_s, s = 0..nsteps
    uint32_t* perm_all = nullptr;
    float* sfrac = nullptr;      // [3][N^3] fractional offsets in the order of perm (paint)
    float* sfrac_all = nullptr;  // [nsteps+1][3][N^3] the same for every step's sort (reused by the adjoint)
    uint32_t* start_all = nullptr;

    // meshes
    float* delta = nullptr;
    float* F = nullptr;     // 3 * N3 scratch (forces of standalone calls, adjoint temporaries)
    float* F_all = nullptr; // [nsteps][3][N^3] the force of every step of the forward sweep, kept for the adjoint
    float* feat = nullptr;  // 3 * N3
    float* M = nullptr;
    float* MR = nullptr;
    float* DR = nullptr;
    float* rs = nullptr;
    float* gm = nullptr;    // N3 scratch mesh
    float* gm2 = nullptr;   // N3 scratch mesh
    float* gfeat = nullptr; // 3 * N3
    float* gv = nullptr;    // 81 * N3 network input-gradient scratch (CUDA-core network)
    float* gbox = nullptr;  // per-tile box sums of the input gradient (tensor-core network)
    float* nn_y = nullptr;      // tensor-core network forward, saved per voxel for its backward: y [N3],
    uint16_t* nn_m1 = nullptr;  // layer-1 ReLU mask [4][N3] (16 columns each),
    uint8_t* nn_m2 = nullptr;   // layer-2 ReLU mask [4][N3] (8 columns each)
    float2* cA = nullptr;   // complex work arrays, NH each
    float2* cB = nullptr;
    float2* c3 = nullptr;   // 3 * NH

    // reductions
    double* red_part = nullptr;  // per-block partials
    double* red_out = nullptr;   // device scalars
    int red_blocks = 0;

    pmr::LBFGS lb;

    // launch accounting: every kernel launch passes check_launch(); with
    // timing on, an event is recorded after each launch on the context stream
    int64_t launches = 0;
    bool timing = false;
    // optional CUDA graph of one loss_and_grad evaluation (pmr_use_graphs)
    bool graphs = false;
    cudaGraphExec_t g_exec = nullptr;
    const float2* g_s = nullptr;
    const float* g_data = nullptr;
    float2* g_grad = nullptr;
    pmr_anneal g_an{};
    int64_t g_launches = 0;  // kernel launches inside the graph
    std::vector<cudaEvent_t> ev_pool;
    std::vector<const char*> ev_names;
    size_t ev_used = 0;
};

namespace pmr {

// error helpers ----------------------------------------------------------------
int fail(pmr_ctx* c, int code, const std::string& msg);
int check_cuda(pmr_ctx* c, cudaError_t e, const char* what);
int check_launch(pmr_ctx* c, const char* what);

#define PMR_TRY(expr)               \
    do {                            \
        int _rc = (expr);           \
        if (_rc != PMR_OK) return _rc; \
    } while (0)

// host cosmology (cosmo.cpp) -----------------------------------------------------
double growth_D(double a, double om);
double growth_dDda(double a, double om);
double growth_Gp(double a, double om);
double growth_Gf(double a, double om);
double bbks_amplitude(double sigma8, double gamma);
double bbks_power(double k, double amp, double gamma);

// FFT module (fft.cu) -----------------------------------------------------------
int fft_init(pmr_ctx* c);
void fft_free(pmr_ctx* c);
// real -> half complex (unnormalised)
int fft_r2c(pmr_ctx* c, const float* in, float2* out);
// half complex (full k-space) -> real, with 1/N^3; destroys `work` (NH)
int fft_c2r(pmr_ctx* c, const float2* in, float* out, float2* work);
// real in -> nout real outs, out_j = irfft(mul_j * rfft(in))
int conv_1toN(pmr_ctx* c, const float* in, float* const* out, const Mul* mul, int nout);
// nin real ins -> real out = irfft(sum_i mul_i * rfft(in_i))
int conv_Nto1(pmr_ctx* c, const float* const* in, const Mul* mul, int nin, float* out);
// k-space in (half array) -> nout real outs, out_j = irfft(mul_j * in)
int k_to_real(pmr_ctx* c, const float2* in, float* const* out, const Mul* mul, int nout);
// nin real ins -> k-space out = sum_i mul_i * rfft(in_i)
int real_to_k(pmr_ctx* c, const float* const* in, const Mul* mul, int nin, float2* out);
// out += sum_i mul_i rfft(in_i)
int real_to_k_add(pmr_ctx* c, const float* const* in, const Mul* mul, int nin, float2* out);

// PM kernels (pm.cu) ------------------------------------------------------------
// positions are either explicit absolute positions (lattice == false) or
// lattice + displacement (lattice == true; q from the particle index)
int cell_sort(pmr_ctx* c, const float* pos, int64_t np, bool lattice, uint32_t* keys_out);
int paint(pmr_ctx* c, const float* pos, int64_t np, bool lattice, const float* mass, int nmass,
          float scale, float offset, float* const* rho);
int readout(pmr_ctx* c, const float* field, const float* pos, int64_t np, bool lattice, float* out);
int readout_grad(pmr_ctx* c, const float* field, const float* pos, int64_t np, bool lattice,
                 float scale, bool accumulate, float* out);
int za_ics(pmr_ctx* c, const float2* s_k, float* disp, float* mom);
int kick_drift(pmr_ctx* c, const float* F, const float* disp_in, float* disp_out, float* mom, float kick,
               float drift);
int za_adjoint(pmr_ctx* c, const float* lam_x, const float* lam_p, float2* grad);
int lpt_ics(pmr_ctx* c, const float2* s_k, float* disp, float* mom);
int pm_init(pmr_ctx* c);
int lpt_adjoint(pmr_ctx* c, const float2* s_k, const float* lam_x, const float* lam_p, float2* grad, bool have_H);
int pm_forward_impl(pmr_ctx* c, const float2* s_k);
int pm_adjoint_impl(pmr_ctx* c, const float* gfin, float2* grad);  // gfin: gradient w.r.t. the final density
int density_from(pmr_ctx* c, const float* disp, float* delta);
// sfrac (nullable): also write the particles' fractional offsets in sorted order, [3][np]
int cell_sort_into(pmr_ctx* c, const float* pos, int64_t np, bool lattice, uint32_t* keys_out, uint32_t* perm,
                   uint32_t* start, float* sfrac);
// sfrac (nullable): the offsets written by the sort that produced perm/start
int paint_with(pmr_ctx* c, const float* pos, int64_t np, bool lattice, const uint32_t* perm, const uint32_t* start,
               const float* sfrac, const float* mass, int nmass, float scale, float offset, float* const* rho);
// density of step s's positions; sort == true sorts them into slot s first,
// otherwise slot s must already hold their sort (from the forward sweep)
int density_slot(pmr_ctx* c, int s, const float* disp, float* delta, bool sort);

// network (nn.cu) ---------------------------------------------------------------
int nn_features(pmr_ctx* c, const float* delta);  // -> c->feat
// a: logistic sharpness of the two-network head (ignored by the softplus head)
int mlp_forward(pmr_ctx* c, const float* feat, float* M, float a);
int mlp_backward(pmr_ctx* c, const float* feat, const float* gM, float* gfeat, float a);
int stencil_transpose(pmr_ctx* c, const float* gv, float* gfeat);

void twopt_free(pmr_ctx* c);

// network on tcgen05 tensor cores (mlp_tc.cu) -----------------------------------
int mlp_tc_init(pmr_ctx* c);
void mlp_tc_free(pmr_ctx* c);
int mlp_tc_forward(pmr_ctx* c, const float* feat, float* M, int nsplit, float a);
int mlp_tc_backward_gv(pmr_ctx* c, const float* feat, const float* gM, int nsplit, float a);  // -> c->gbox
int mlp_tc_box_floats(int N);               // size of c->gbox
int stencil_tiles(pmr_ctx* c, float* gfeat);  // c->gbox -> input gradient of the three fields

// loss (loss.cu) ----------------------------------------------------------------
int residual_forward(pmr_ctx* c, const float* data, const pmr_anneal* an, double* L_res_dev);
int residual_backward(pmr_ctx* c, const pmr_anneal* an, float* gM);
int prior_value(pmr_ctx* c, const float2* s, double* out_dev);
int prior_grad_add(pmr_ctx* c, const float2* s, float2* grad);
int reduce_sum_sq(pmr_ctx* c, const float* v, int64_t n, double scale, double* out_dev);
int check_finite(pmr_ctx* c, const double* v, int n, double* host);
int loss_to_device(pmr_ctx* c, double* out_dev);
// PMR_ETIMEOUT (and the flag cleared) if a tensor-core kernel's wait ran out
// since the last check; synchronises the stream
int check_tc_timeout(pmr_ctx* c);

// L-BFGS (lbfgs.cu) -------------------------------------------------------------
int lbfgs_alloc(pmr_ctx* c);
void lbfgs_free(pmr_ctx* c);
int lbfgs_two_loop(pmr_ctx* c, const double* g, const double* S, const double* Y, int k, int head, int m,
                   int64_t n, const double* rho_host, double* d, bool prior_h0);
// y = scale * diag(P~ / w) x over the half-array reals (the prior's inverse Hessian)
int prior_h0_apply(pmr_ctx* c, double* y, const double* x, double scale);
int dot64(pmr_ctx* c, const double* a, const double* b, int64_t n, double* out_dev);
int c64_to_f64(pmr_ctx* c, const float2* a, double* out, int64_t nh);
int f64_to_c64(pmr_ctx* c, const double* a, float2* out, int64_t nh);
int axpy64(pmr_ctx* c, double* y, const double* x, const double* alpha_dev, double alpha_host, int64_t n,
           const double* base);

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace pmr

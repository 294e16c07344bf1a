// C ABI of the reconstruction library: context lifetime, validation, the
// workspace layout, and the host orchestration of the forward model, its
// adjoint, the loss and the L-BFGS step (Sec. 3, 5.1, 5.2).
#include <cmath>
#include <cstring>

#include "common.cuh"

using namespace pmr;

namespace pmr {

static thread_local std::string g_create_err;

int fail(pmr_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_err = msg;
    return code;
}

int check_cuda(pmr_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return PMR_OK;
    return fail(c, e == cudaErrorMemoryAllocation ? PMR_ENOMEM : PMR_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

static void record_event(pmr_ctx* c, const char* what) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->ev_pool.push_back(e);
        c->ev_names.push_back(nullptr);
    }
    cudaEventRecord(c->ev_pool[c->ev_used], c->stream);
    c->ev_names[c->ev_used] = what;
    c->ev_used++;
}

int check_tc_timeout(pmr_ctx* c) {
    if (!c->tc_err) return check_cuda(c, cudaStreamSynchronize(c->stream), "sync");
    int flag = 0;
    PMR_TRY(check_cuda(c, cudaMemcpyAsync(&flag, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "rb"));
    PMR_TRY(check_cuda(c, cudaStreamSynchronize(c->stream), "sync"));
    if (!flag) return PMR_OK;
    PMR_TRY(check_cuda(c, cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->stream), "clear flag"));
    PMR_TRY(check_cuda(c, cudaStreamSynchronize(c->stream), "sync"));
    return fail(c, PMR_ETIMEOUT, "a tensor-core network kernel's barrier wait ran out; the kernel freed its tensor "
                                 "memory and returned, its outputs are invalid");
}

int check_launch(pmr_ctx* c, const char* what) {
    int rc = check_cuda(c, cudaGetLastError(), what);
    if (rc == PMR_OK) {
        c->launches++;
        if (c->timing) record_event(c, what);
    }
    return rc;
}

}  // namespace pmr

namespace {

constexpr int kNW = 5661 + kMassWeights;  // trunk + mass network (the latter only with head == 1)

int n_weights(const pmr_config* cfg) { return 5661 + (cfg->head == 1 ? kMassWeights : 0); }

float logistic_a(const pmr_anneal* an) { return an ? (float)an->a_logistic : 3.0f; }

// The network sees f_i = sum_j C_ij delta_Rj (Sec. 2.2's mixed features) but
// the kernels read the three smoothed fields delta_Rj: W1'[h][j*27 + o] =
// sum_i W1[h][i*27 + o] C_ij, and the mass network's (head 1, on the voxel's
// own three features) Wm1'[k][j] = sum_i Wm1[k][i] C_ij. Products in double.
void fold_feature_mix(const pmr_config* cfg, float* W) {
    const float* C = cfg->feat_mix;
    bool ident = true;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) ident &= C[3 * i + j] == (i == j ? 1.0f : 0.0f);
    if (ident) return;
    for (int h = 0; h < 50; ++h)
        for (int o = 0; o < 27; ++o) {
            double src[3], dst[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < 3; ++i) src[i] = W[h * 81 + i * 27 + o];
            for (int j = 0; j < 3; ++j)
                for (int i = 0; i < 3; ++i) dst[j] += src[i] * (double)C[3 * i + j];
            for (int j = 0; j < 3; ++j) W[h * 81 + j * 27 + o] = (float)dst[j];
        }
    if (cfg->head == 1) {
        float* Wm1 = W + 5661;
        for (int k = 0; k < 20; ++k) {
            double src[3], dst[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < 3; ++i) src[i] = Wm1[3 * k + i];
            for (int j = 0; j < 3; ++j)
                for (int i = 0; i < 3; ++i) dst[j] += src[i] * (double)C[3 * i + j];
            for (int j = 0; j < 3; ++j) Wm1[3 * k + j] = (float)dst[j];
        }
    }
}

const char* validate(const pmr_config* cfg) {
    if (!cfg) return "config is NULL";
    const int N = cfg->N;
    if (N < 8 || N > 512 || N % 2 || !radix_ok(N) || !radix_ok(N / 2)) return "N must be 2^a 3^b, even, 8..512";
    if (!(cfg->L > 0)) return "L must be > 0";
    if (cfg->nsteps < 1 || cfg->nsteps > 1000) return "nsteps must be 1..1000";
    if (!(cfg->a0 > 0 && cfg->a0 < 1)) return "a0 must be in (0, 1)";
    if (!(cfg->omega_m > 0 && cfg->omega_m <= 1)) return "omega_m must be in (0, 1]";
    if (!(cfg->sigma8 > 0) || !(cfg->gamma_bbks > 0)) return "sigma8 and gamma_bbks must be > 0";
    for (int j = 0; j < 3; ++j)
        if (!(cfg->R_feat[j] >= 0)) return "R_feat must be >= 0";
    for (int j = 0; j < 9; ++j)
        if (!std::isfinite(cfg->feat_mix[j])) return "feat_mix must be finite";
    if (!(cfg->R_M >= 0)) return "R_M must be >= 0";
    if (!(cfg->sigma_N2 > 0)) return "sigma_N2 must be > 0";
    if (!(cfg->M_scale > 0)) return "M_scale must be > 0";
    if (!std::isfinite(cfg->mu_N) || !std::isfinite(cfg->f_eff)) return "mu_N and f_eff must be finite";
    if (cfg->lbfgs_m < 1 || cfg->lbfgs_m > 64) return "lbfgs_m must be 1..64";
    if (!(cfg->lbfgs_tol >= 0)) return "lbfgs_tol must be >= 0";
    if (cfg->nn_path < 0 || cfg->nn_path > 3) return "nn_path must be 0, 1, 2 or 3";
    if (cfg->head < 0 || cfg->head > 1) return "head must be 0 or 1";
    if (cfg->lpt_order < 1 || cfg->lpt_order > 2) return "lpt_order must be 1 or 2";
    return nullptr;
}

struct Sizes {
    size_t bytes = 0;
};

// Every device buffer of a context, in one place (allocation and the footprint query).
template <class F>
void for_each_buffer(const pmr_config& cfg, pmr_ctx* c, F alloc) {
    const int64_t N = cfg.N, N3 = N * N * N, P = N / 2 + 1, NH = N * N * P;
    const int64_t nb_scan = (N3 + 1023) / 1024;
    alloc((void**)(c ? &c->disp : nullptr), sizeof(float) * 3 * N3 * (cfg.nsteps + 1));
    alloc((void**)(c ? &c->mom : nullptr), sizeof(float) * 3 * N3);
    alloc((void**)(c ? &c->lam_x : nullptr), sizeof(float) * 3 * N3);
    alloc((void**)(c ? &c->lam_p : nullptr), sizeof(float) * 3 * N3);
    alloc((void**)(c ? &c->keys : nullptr), sizeof(uint32_t) * N3);
    alloc((void**)(c ? &c->perm : nullptr), sizeof(uint32_t) * N3);
    alloc((void**)(c ? &c->cell_start : nullptr), sizeof(uint32_t) * (N3 + 1));
    alloc((void**)(c ? &c->counts : nullptr), sizeof(uint32_t) * N3);
    alloc((void**)(c ? &c->scan_part : nullptr), sizeof(uint32_t) * nb_scan);
    alloc((void**)(c ? &c->long_list : nullptr), sizeof(uint32_t) * N3);
    alloc((void**)(c ? &c->long_count : nullptr), sizeof(uint32_t) * 4);
    alloc((void**)(c ? &c->sort_tmp : nullptr), sizeof(uint32_t) * N3);
    alloc((void**)(c ? &c->perm_all : nullptr), sizeof(uint32_t) * N3 * (cfg.nsteps + 1));
    alloc((void**)(c ? &c->start_all : nullptr), sizeof(uint32_t) * (N3 + 1) * (cfg.nsteps + 1));
    alloc((void**)(c ? &c->sfrac : nullptr), sizeof(float) * 3 * N3);
    alloc((void**)(c ? &c->sfrac_all : nullptr), sizeof(float) * 3 * N3 * (cfg.nsteps + 1));
    alloc((void**)(c ? &c->delta : nullptr), sizeof(float) * N3);
    alloc((void**)(c ? &c->F : nullptr), sizeof(float) * 3 * N3);
    alloc((void**)(c ? &c->F_all : nullptr), sizeof(float) * 3 * N3 * (cfg.nsteps > 0 ? cfg.nsteps : 1));
    alloc((void**)(c ? &c->feat : nullptr), sizeof(float) * 3 * N3);
    alloc((void**)(c ? &c->M : nullptr), sizeof(float) * N3);
    alloc((void**)(c ? &c->MR : nullptr), sizeof(float) * N3);
    alloc((void**)(c ? &c->DR : nullptr), sizeof(float) * N3);
    alloc((void**)(c ? &c->rs : nullptr), sizeof(float) * N3);
    alloc((void**)(c ? &c->gm : nullptr), sizeof(float) * N3);
    alloc((void**)(c ? &c->gm2 : nullptr), sizeof(float) * N3);
    alloc((void**)(c ? &c->gfeat : nullptr), sizeof(float) * 3 * N3);
    if (cfg.nn_path == 2) alloc((void**)(c ? &c->gv : nullptr), sizeof(float) * 81 * N3);
    else {
        alloc((void**)(c ? &c->gbox : nullptr), sizeof(float) * (size_t)mlp_tc_box_floats((int)N));
        alloc((void**)(c ? &c->nn_y : nullptr), sizeof(float) * N3);
        alloc((void**)(c ? &c->nn_m1 : nullptr), sizeof(uint16_t) * 4 * N3);
        alloc((void**)(c ? &c->nn_m2 : nullptr), sizeof(uint8_t) * 4 * N3);
    }
    alloc((void**)(c ? &c->cA : nullptr), sizeof(float2) * NH);
    alloc((void**)(c ? &c->cB : nullptr), sizeof(float2) * NH);
    alloc((void**)(c ? &c->c3 : nullptr), sizeof(float2) * 3 * NH);
    alloc((void**)(c ? &c->red_part : nullptr), sizeof(double) * 1024);
    alloc((void**)(c ? &c->red_out : nullptr), sizeof(double) * 8);
    alloc((void**)(c ? &c->W : nullptr), sizeof(float) * kNW);
    alloc((void**)(c ? &c->power_tab : nullptr), sizeof(float) * (3 * (N / 2) * (N / 2) + 1));
    alloc((void**)(c ? &c->inv_power_tab : nullptr), sizeof(double) * (3 * (N / 2) * (N / 2) + 1));
    if (cfg.lpt_order == 2) {
        alloc((void**)(c ? &c->lpt_H : nullptr), sizeof(float) * 6 * N3);
        alloc((void**)(c ? &c->lpt_G : nullptr), sizeof(float) * 6 * N3);
    }
}

size_t lbfgs_bytes(const pmr_config& cfg) {
    const int64_t N = cfg.N, NH = N * N * (N / 2 + 1);
    return sizeof(double) * 2 * NH * (6 + 2 * (size_t)cfg.lbfgs_m) + sizeof(float2) * NH + sizeof(double) * 80;
}

void free_all(pmr_ctx* c) {
    for_each_buffer(c->cfg, c, [](void** p, size_t) {
        if (p && *p) cudaFree(*p);
        if (p) *p = nullptr;
    });
    fft_free(c);
    mlp_tc_free(c);
    twopt_free(c);
    lbfgs_free(c);
}

int check_ctx(pmr_ctx* c) { return c ? PMR_OK : fail(nullptr, PMR_EINVAL, "context is NULL"); }

// total, prior, residual into host[0..2]
int finish_loss(pmr_ctx* c, double* host) {
    double v[2];
    PMR_TRY(check_tc_timeout(c));
    PMR_TRY(check_finite(c, c->red_out, 2, v));
    host[0] = v[0] + v[1];
    host[1] = v[0];
    host[2] = v[1];
    return PMR_OK;
}

Mul gauss(const pmr_ctx* c, double R_mpc) {
    const double R = R_mpc / (c->cfg.L / c->N);
    return Mul{R > 0 ? MUL_GAUSS : MUL_ONE, 0, 1.0f, (float)(R * R), 0};
}

// grad_delta = sum_c S_{R_c} gfeat_c
int features_T(pmr_ctx* c, const float* gfeat, float* out) {
    Mul mul[3];
    for (int j = 0; j < 3; ++j) mul[j] = gauss(c, c->cfg.R_feat[j]);
    const float* ins[3] = {gfeat, gfeat + c->N3, gfeat + 2 * c->N3};
    return conv_Nto1(c, ins, mul, 3, out);
}

int loss_and_grad_impl(pmr_ctx* c, const float2* s, const float* data, const pmr_anneal* an, double* host,
                       float2* grad) {
    const int64_t N3 = c->N3;
    const float* dfin = c->disp + (int64_t)c->cfg.nsteps * 3 * N3;
    // forward
    PMR_TRY(pm_forward_impl(c, s));
    PMR_TRY(density_slot(c, c->cfg.nsteps, dfin, c->delta, true));
    PMR_TRY(nn_features(c, c->delta));
    PMR_TRY(mlp_forward(c, c->feat, c->M, logistic_a(an)));
    PMR_TRY(residual_forward(c, data, an, c->red_out + 1));
    PMR_TRY(prior_value(c, s, c->red_out));
    // adjoint
    PMR_TRY(residual_backward(c, an, c->gm2));
    PMR_TRY(mlp_backward(c, c->feat, c->gm2, c->gfeat, logistic_a(an)));
    PMR_TRY(features_T(c, c->gfeat, c->gm2));
    PMR_TRY(pm_adjoint_impl(c, c->gm2, grad));
    PMR_TRY(prior_grad_add(c, s, grad));
    if (host) return finish_loss(c, host);
    return PMR_OK;
}

}  // namespace

extern "C" {

void pmr_default_config(pmr_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->N = 32;
    cfg->L = 100.0;
    cfg->nsteps = 3;
    cfg->a0 = 0.1;
    cfg->omega_m = 0.3175;
    cfg->sigma8 = 0.8;
    cfg->gamma_bbks = 0.21;
    cfg->R_feat[0] = 1.0;
    cfg->R_feat[1] = 2.0;
    cfg->R_feat[2] = 4.0;
    for (int j = 0; j < 9; ++j) cfg->feat_mix[j] = (j % 4 == 0) ? 1.0f : 0.0f;
    cfg->R_M = 3.0;
    cfg->sigma_N2 = 0.25;
    cfg->mu_N = 0.0;
    cfg->f_eff = 1.0;
    cfg->M_scale = 1e12;
    cfg->lbfgs_m = 10;
    cfg->lbfgs_tol = 1e-3;
    cfg->nn_path = 0;
    cfg->head = 0;
    cfg->lpt_order = 1;
}

size_t pmr_workspace_bytes(const pmr_config* cfg) {
    if (validate(cfg)) return 0;
    size_t total = 0;
    for_each_buffer(*cfg, nullptr, [&](void**, size_t b) { total += (b + 255) / 256 * 256; });
    total += lbfgs_bytes(*cfg);
    total += sizeof(float2) * (cfg->N + cfg->N / 2);  // twiddles
    return total;
}

const char* pmr_last_error(const pmr_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

int pmr_create(const pmr_config* cfg, const float* nn_weights_dev, void* stream, pmr_ctx** out) {
    if (!out) return fail(nullptr, PMR_EINVAL, "out is NULL");
    *out = nullptr;
    if (const char* why = validate(cfg)) return fail(nullptr, PMR_EINVAL, why);
    if (!nn_weights_dev) return fail(nullptr, PMR_EINVAL, "nn_weights_dev is NULL");
    pmr_ctx* c = new pmr_ctx();
    c->cfg = *cfg;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (c->num_sms < 1) c->num_sms = 1;
    const int N = cfg->N;
    c->N = N;
    c->P = N / 2 + 1;
    c->N3 = (int64_t)N * N * N;
    c->NH = (int64_t)N * N * c->P;

    // growth factors and the kick/drift coefficients that make Zel'dovich trajectories exact
    const double om = cfg->omega_m;
    c->D0 = growth_D(cfg->a0, om);
    c->Gp0 = growth_Gp(cfg->a0, om);
    c->D2_0 = -3.0 / 7.0 * c->D0 * c->D0;    // second-order growth, D2 = -3/7 D1^2
    c->Gp2_0 = -6.0 / 7.0 * c->D0 * c->Gp0;  // a^3 E dD2/da
    const int n = cfg->nsteps;
    for (int i = 0; i < n; ++i) {
        const double ai = cfg->a0 + (1.0 - cfg->a0) * i / n, aj = cfg->a0 + (1.0 - cfg->a0) * (i + 1) / n;
        const double ah = 0.5 * (ai + aj);
        const double ap = (i == 0) ? cfg->a0 : 0.5 * (cfg->a0 + (1.0 - cfg->a0) * (i - 1) / n + ai);
        c->kick.push_back((growth_Gp(ah, om) - growth_Gp(ap, om)) / growth_Gf(ai, om));
        c->drift.push_back((growth_D(aj, om) - growth_D(ai, om)) / growth_Gp(ah, om));
    }

    int rc = PMR_OK;
    for_each_buffer(*cfg, c, [&](void** p, size_t b) {
        if (rc == PMR_OK) rc = check_cuda(c, cudaMalloc(p, b), "workspace");
    });
    if (rc == PMR_OK) rc = fft_init(c);
    if (rc == PMR_OK) rc = pm_init(c);
    if (rc == PMR_OK) rc = lbfgs_alloc(c);
    if (rc == PMR_OK) {
        // linear power P~ = P(k) N^6 / L^3 on integer |n|^2, k = 2 pi |n| / L
        const int ntab = 3 * (N / 2) * (N / 2) + 1;
        c->ntab = ntab;
        const double amp = bbks_amplitude(cfg->sigma8, cfg->gamma_bbks);
        const double n6v = std::pow((double)N, 6) / std::pow(cfg->L, 3), n3 = (double)c->N3;
        std::vector<float> sq(ntab);
        std::vector<double> inv(ntab);
        for (int t = 0; t < ntab; ++t) {
            const double k = 2.0 * M_PI * std::sqrt((double)t) / cfg->L;
            const double Pt = (t == 0) ? 0.0 : bbks_power(k, amp, cfg->gamma_bbks) * n6v;
            sq[t] = (float)std::sqrt(Pt / n3);
            inv[t] = (t == 0) ? 0.0 : 1.0 / Pt;
        }
        rc = check_cuda(c, cudaMemcpy(c->power_tab, sq.data(), sizeof(float) * ntab, cudaMemcpyHostToDevice), "table");
        if (rc == PMR_OK)
            rc = check_cuda(c, cudaMemcpy(c->inv_power_tab, inv.data(), sizeof(double) * ntab, cudaMemcpyHostToDevice),
                            "table");
    }
    if (rc == PMR_OK) {
        const int nw = n_weights(cfg);
        c->W_host.assign(kNW, 0.0f);
        rc = check_cuda(c, cudaMemcpy(c->W_host.data(), nn_weights_dev, sizeof(float) * nw, cudaMemcpyDeviceToHost),
                        "weights");
        if (rc == PMR_OK) {
            fold_feature_mix(cfg, c->W_host.data());
            rc = check_cuda(c, cudaMemcpy(c->W, c->W_host.data(), sizeof(float) * kNW, cudaMemcpyHostToDevice),
                            "weights");
        }
        if (rc == PMR_OK) rc = mlp_tc_init(c);
    }
    if (rc != PMR_OK) {
        g_create_err = c->err;
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return PMR_OK;
}

int pmr_destroy(pmr_ctx* c) {
    if (!c) return PMR_OK;
    cudaStreamSynchronize(c->stream);
    if (c->g_exec) cudaGraphExecDestroy(c->g_exec);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    free_all(c);
    delete c;
    return PMR_OK;
}

int pmr_set_stream(pmr_ctx* c, void* stream) {
    PMR_TRY(check_ctx(c));
    if (c->graphs && !stream) return fail(c, PMR_EINVAL, "CUDA graphs need a non-default stream");
    if (c->g_exec) cudaGraphExecDestroy(c->g_exec);
    c->g_exec = nullptr;
    c->g_s = nullptr;
    c->stream = (cudaStream_t)stream;
    return PMR_OK;
}

int pmr_linear_field(pmr_ctx* c, const float* white, double amplitude, void* s_k) {
    PMR_TRY(check_ctx(c));
    if (!white || !s_k) return fail(c, PMR_EINVAL, "NULL argument");
    Mul m{MUL_POWER, 0, (float)amplitude, 0.f, 0};
    const float* ins[1] = {white};
    return real_to_k(c, ins, &m, 1, (float2*)s_k);
}

int pm_forward(pmr_ctx* c, const void* s_k, float* delta_out) {
    PMR_TRY(check_ctx(c));
    if (!s_k || !delta_out) return fail(c, PMR_EINVAL, "NULL argument");
    PMR_TRY(pm_forward_impl(c, (const float2*)s_k));
    return density_slot(c, c->cfg.nsteps, c->disp + (int64_t)c->cfg.nsteps * 3 * c->N3, delta_out, true);
}

int pm_adjoint(pmr_ctx* c, const float* grad_delta, void* grad_s_k) {
    PMR_TRY(check_ctx(c));
    if (!grad_delta || !grad_s_k) return fail(c, PMR_EINVAL, "NULL argument");
    if (!c->have_forward) return fail(c, PMR_ESTATE, "pm_adjoint needs a pm_forward on this context first");
    return pm_adjoint_impl(c, grad_delta, (float2*)grad_s_k);
}

int nn_halo_map(pmr_ctx* c, const float* delta, float* mass_out, const pmr_anneal* an) {
    PMR_TRY(check_ctx(c));
    if (!delta || !mass_out) return fail(c, PMR_EINVAL, "NULL argument");
    PMR_TRY(nn_features(c, delta));
    return mlp_forward(c, c->feat, mass_out, logistic_a(an));
}

int nn_halo_map_adjoint(pmr_ctx* c, const float* delta, const float* grad_mass, float* grad_delta,
                        const pmr_anneal* an) {
    PMR_TRY(check_ctx(c));
    if (!delta || !grad_mass || !grad_delta) return fail(c, PMR_EINVAL, "NULL argument");
    PMR_TRY(nn_features(c, delta));
    // the tensor-core backward starts from the forward's saved activations
    if (c->cfg.nn_path != 2) PMR_TRY(mlp_forward(c, c->feat, c->M, logistic_a(an)));
    PMR_TRY(mlp_backward(c, c->feat, grad_mass, c->gfeat, logistic_a(an)));
    return features_T(c, c->gfeat, grad_delta);
}

namespace {
void drop_graph(pmr_ctx* c) {
    if (c->g_exec) cudaGraphExecDestroy(c->g_exec);
    c->g_exec = nullptr;
    c->g_s = nullptr;
}

bool same_anneal(const pmr_anneal& a, const pmr_anneal& b) {
    return a.R_sm == b.R_sm && a.M0 == b.M0 && a.a_logistic == b.a_logistic;
}
}  // namespace

// One evaluation; with graphs on, the launches of loss_and_grad_impl for these
// (s, data, an, grad) are captured once and replayed as one graph launch.
static int evaluate(pmr_ctx* c, const float2* s, const float* data, const pmr_anneal* an, double* host,
                    float2* grad) {
    if (!c->graphs) return loss_and_grad_impl(c, s, data, an, host, grad);
    if (!c->g_exec || c->g_s != s || c->g_data != data || c->g_grad != grad || !same_anneal(c->g_an, *an)) {
        drop_graph(c);
        const bool timing = c->timing;
        const int64_t l0 = c->launches;
        c->timing = false;
        PMR_TRY(check_cuda(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture"));
        const int rc = loss_and_grad_impl(c, s, data, an, nullptr, grad);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        c->timing = timing;
        c->g_launches = c->launches - l0;
        c->launches = l0;
        if (rc != PMR_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        PMR_TRY(check_cuda(c, e, "end capture"));
        const cudaError_t ei = cudaGraphInstantiate(&c->g_exec, g, 0);
        cudaGraphDestroy(g);
        PMR_TRY(check_cuda(c, ei, "graph instantiate"));
        c->g_s = s;
        c->g_data = data;
        c->g_grad = grad;
        c->g_an = *an;
    }
    PMR_TRY(check_cuda(c, cudaGraphLaunch(c->g_exec, c->stream), "graph launch"));
    c->launches += c->g_launches;
    if (host) return finish_loss(c, host);
    return PMR_OK;
}

int pmr_use_graphs(pmr_ctx* c, int enable) {
    PMR_TRY(check_ctx(c));
    if (enable && !c->stream) return fail(c, PMR_EINVAL, "CUDA graphs need a context created on a non-default stream");
    if (!enable) drop_graph(c);
    c->graphs = enable != 0;
    return PMR_OK;
}

int loss_and_grad(pmr_ctx* c, const void* s_k, const float* data_mass, const pmr_anneal* an, double* loss_out,
                  void* grad_s_k) {
    PMR_TRY(check_ctx(c));
    if (!s_k || !data_mass || !an || !grad_s_k) return fail(c, PMR_EINVAL, "NULL argument");
    if (!(an->R_sm >= 0) || !std::isfinite(an->M0)) return fail(c, PMR_EINVAL, "anneal: R_sm >= 0, finite M0");
    bool dev_out = false;
    if (loss_out) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, loss_out) != cudaSuccess) cudaGetLastError();  // plain host memory
        else dev_out = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
    }
    if (!dev_out) return evaluate(c, (const float2*)s_k, data_mass, an, loss_out, (float2*)grad_s_k);
    // device destination: enqueue the copy, no host read-back and no synchronisation
    PMR_TRY(evaluate(c, (const float2*)s_k, data_mass, an, nullptr, (float2*)grad_s_k));
    return loss_to_device(c, loss_out);
}

int pmr_sync(pmr_ctx* c) {
    PMR_TRY(check_ctx(c));
    return check_tc_timeout(c);
}

int pmr_test_stall_mma(pmr_ctx* c, int enable) {
    PMR_TRY(check_ctx(c));
    if (c->cfg.nn_path == 2) return fail(c, PMR_EINVAL, "the CUDA-core network (nn_path 2) has no tensor-core waits");
    c->tc_stall = enable != 0;
    if (c->g_exec) drop_graph(c);  // a captured graph holds the launch controls
    return PMR_OK;
}

int pmr_lbfgs_reset(pmr_ctx* c) {
    PMR_TRY(check_ctx(c));
    c->lb.k = 0;
    c->lb.head = 0;
    c->lb.have_f = false;
    return PMR_OK;
}

int recon_step(pmr_ctx* c, void* s_k_v, const float* data, const pmr_anneal* an, double* loss_out, int* converged) {
    PMR_TRY(check_ctx(c));
    if (!s_k_v || !data || !an) return fail(c, PMR_EINVAL, "NULL argument");
    float2* s_k = (float2*)s_k_v;
    LBFGS& L = c->lb;
    const int64_t n = L.n;
    double host[3];
    if (!L.have_f || an->R_sm != L.an.R_sm || an->M0 != L.an.M0 || an->a_logistic != L.an.a_logistic) {
        L.k = 0;
        L.head = 0;
        PMR_TRY(evaluate(c, s_k, data, an, host, L.gk));
        PMR_TRY(c64_to_f64(c, s_k, L.x, c->NH));
        PMR_TRY(c64_to_f64(c, L.gk, L.g, c->NH));
        L.f = host[0];
        L.have_f = true;
        L.an = *an;
    }
    double sc[3];
    double gd = 0.0;
    if (L.k > 0) {
        PMR_TRY(lbfgs_two_loop(c, L.g, L.S, L.Y, L.k, L.head, L.m, n, L.rho_host.data(), L.d, true));
        PMR_TRY(dot64(c, L.g, L.d, n, L.scal + 2));
        PMR_TRY(check_cuda(c, cudaMemcpyAsync(sc, L.scal + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "rb"));
        PMR_TRY(check_cuda(c, cudaStreamSynchronize(c->stream), "sync"));
        gd = sc[0];
        if (!(gd < 0)) {
            L.k = 0;
            L.head = 0;
        }
    }
    if (L.k == 0) {
        // first step: -H0 g with H0 = diag(P~ / w), the prior's inverse Hessian
        PMR_TRY(prior_h0_apply(c, L.d, L.g, -1.0));
        PMR_TRY(dot64(c, L.g, L.d, n, L.scal + 2));
        PMR_TRY(check_cuda(c, cudaMemcpyAsync(sc, L.scal + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "rb"));
        PMR_TRY(check_cuda(c, cudaStreamSynchronize(c->stream), "sync"));
        gd = sc[0];
        if (!(gd < 0)) return fail(c, PMR_ELINESEARCH, "zero gradient");
    }
    const double c1 = 1e-4;
    double t = 1.0, fnew = 0.0;
    bool ok = false;
    for (int it = 0; it < 20; ++it) {
        PMR_TRY(axpy64(c, L.xt, L.d, nullptr, t, n, L.x));
        PMR_TRY(f64_to_c64(c, L.xt, s_k, c->NH));
        int rc = evaluate(c, s_k, data, an, host, L.gk);
        if (rc != PMR_OK && rc != PMR_ENAN) return rc;
        if (rc == PMR_OK && host[0] <= L.f + c1 * t * gd) {
            fnew = host[0];
            ok = true;
            break;
        }
        t *= 0.5;
    }
    if (!ok) {
        PMR_TRY(f64_to_c64(c, L.x, s_k, c->NH));
        return fail(c, PMR_ELINESEARCH, "no Armijo step within 20 halvings");
    }
    PMR_TRY(c64_to_f64(c, L.gk, L.gt, c->NH));
    // candidate pair s = xt - x (into d), y = gt - g
    PMR_TRY(axpy64(c, L.d, L.x, nullptr, -1.0, n, L.xt));
    PMR_TRY(axpy64(c, L.yk, L.g, nullptr, -1.0, n, L.gt));
    PMR_TRY(dot64(c, L.d, L.yk, n, L.scal + 3));
    PMR_TRY(dot64(c, L.d, L.d, n, L.scal + 4));
    PMR_TRY(dot64(c, L.yk, L.yk, n, L.scal + 5));
    PMR_TRY(check_cuda(c, cudaMemcpyAsync(sc, L.scal + 3, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "rb"));
    PMR_TRY(check_cuda(c, cudaStreamSynchronize(c->stream), "sync"));
    if (sc[0] > 1e-10 * std::sqrt(sc[1] * sc[2])) {
        int slot;
        if (L.k < L.m) {
            slot = (L.head + L.k) % L.m;
            L.k++;
        } else {
            slot = L.head;
            L.head = (L.head + 1) % L.m;
        }
        PMR_TRY(check_cuda(c, cudaMemcpyAsync(L.S + (int64_t)slot * n, L.d, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                              c->stream), "copy"));
        PMR_TRY(check_cuda(c, cudaMemcpyAsync(L.Y + (int64_t)slot * n, L.yk, sizeof(double) * n,
                                              cudaMemcpyDeviceToDevice, c->stream), "copy"));
        L.rho_host[slot] = 1.0 / sc[0];
    }
    std::swap(L.x, L.xt);
    std::swap(L.g, L.gt);
    const double fold = L.f;
    L.f = fnew;
    if (converged) *converged = (fold - fnew) < c->cfg.lbfgs_tol * std::fabs(fold) ? 1 : 0;
    if (loss_out) {
        loss_out[0] = host[0];
        loss_out[1] = host[1];
        loss_out[2] = host[2];
    }
    return PMR_OK;
}

int pmr_cell_sort(pmr_ctx* c, const float* x, int64_t np, uint32_t* keys, uint32_t* perm, uint32_t* cell_start) {
    PMR_TRY(check_ctx(c));
    if (!x || !keys || !perm || !cell_start) return fail(c, PMR_EINVAL, "NULL argument");
    if (np < 0 || np > c->N3) return fail(c, PMR_EINVAL, "np must be in [0, N^3]");
    PMR_TRY(cell_sort(c, x, np, false, keys));
    if (np > 0)
        PMR_TRY(check_cuda(c, cudaMemcpyAsync(perm, c->perm, sizeof(uint32_t) * np, cudaMemcpyDeviceToDevice, c->stream),
                           "copy"));
    return check_cuda(c, cudaMemcpyAsync(cell_start, c->cell_start, sizeof(uint32_t) * (c->N3 + 1),
                                         cudaMemcpyDeviceToDevice, c->stream), "copy");
}

int pmr_paint(pmr_ctx* c, const float* x, int64_t np, const float* mass, float* rho) {
    PMR_TRY(check_ctx(c));
    if ((!x && np > 0) || !rho) return fail(c, PMR_EINVAL, "NULL argument");
    if (np < 0 || np > c->N3) return fail(c, PMR_EINVAL, "np must be in [0, N^3]");
    PMR_TRY(cell_sort(c, x, np, false, nullptr));
    float* outs[1] = {rho};
    return paint(c, x, np, false, mass, 1, 1.0f, 0.0f, outs);
}

int pmr_readout(pmr_ctx* c, const float* field, const float* x, int64_t np, float* out) {
    PMR_TRY(check_ctx(c));
    if (!field || ((!x || !out) && np > 0) || np < 0) return fail(c, PMR_EINVAL, "bad argument");
    if (np == 0) return PMR_OK;
    return readout(c, field, x, np, false, out);
}

int pmr_readout_grad(pmr_ctx* c, const float* field, const float* x, int64_t np, float* out) {
    PMR_TRY(check_ctx(c));
    if (!field || ((!x || !out) && np > 0) || np < 0) return fail(c, PMR_EINVAL, "bad argument");
    if (np == 0) return PMR_OK;
    return readout_grad(c, field, x, np, false, 1.0f, false, out);
}

int pmr_rfft(pmr_ctx* c, const float* in, void* out) {
    PMR_TRY(check_ctx(c));
    if (!in || !out) return fail(c, PMR_EINVAL, "NULL argument");
    return fft_r2c(c, in, (float2*)out);
}

int pmr_irfft(pmr_ctx* c, const void* in, float* out) {
    PMR_TRY(check_ctx(c));
    if (!in || !out) return fail(c, PMR_EINVAL, "NULL argument");
    return fft_c2r(c, (const float2*)in, out, c->cB);
}

int pmr_force(pmr_ctx* c, const float* delta, float* F) {
    PMR_TRY(check_ctx(c));
    if (!delta || !F) return fail(c, PMR_EINVAL, "NULL argument");
    Mul m[3];
    for (int j = 0; j < 3; ++j) m[j] = Mul{MUL_ODD, j, (float)(1.5 * c->cfg.omega_m), 0.f, 0};
    float* outs[3] = {F, F + c->N3, F + 2 * c->N3};
    return conv_1toN(c, delta, outs, m, 3);
}

int pmr_smooth(pmr_ctx* c, const float* in, double R, float* out) {
    PMR_TRY(check_ctx(c));
    if (!in || !out || !(R >= 0)) return fail(c, PMR_EINVAL, "bad argument");
    if (R == 0)
        return check_cuda(c, cudaMemcpyAsync(out, in, sizeof(float) * c->N3, cudaMemcpyDeviceToDevice, c->stream), "copy");
    Mul m = gauss(c, R);
    float* outs[1] = {out};
    return conv_1toN(c, in, outs, &m, 1);
}

int pmr_za_ics(pmr_ctx* c, const void* s_k, float* disp, float* mom) {
    PMR_TRY(check_ctx(c));
    if (!s_k || !disp || !mom) return fail(c, PMR_EINVAL, "NULL argument");
    return za_ics(c, (const float2*)s_k, disp, mom);
}

int pmr_lpt_ics(pmr_ctx* c, const void* s_k, float* disp, float* mom) {
    PMR_TRY(check_ctx(c));
    if (!s_k || !disp || !mom) return fail(c, PMR_EINVAL, "NULL argument");
    if (c->cfg.lpt_order == 2) c->have_forward = false;  // replaces the Hessian pm_adjoint needs
    return lpt_ics(c, (const float2*)s_k, disp, mom);
}

int pmr_lpt_ics_adjoint(pmr_ctx* c, const void* s_k, const float* lam_x, const float* lam_p, void* grad_s_k) {
    PMR_TRY(check_ctx(c));
    if (!s_k || !lam_x || !lam_p || !grad_s_k) return fail(c, PMR_EINVAL, "NULL argument");
    if (c->cfg.lpt_order == 2) c->have_forward = false;
    return lpt_adjoint(c, (const float2*)s_k, lam_x, lam_p, (float2*)grad_s_k, false);
}

int pmr_growth(const pmr_config* cfg, double a, double* D, double* Gp, double* Gf) {
    if (!cfg || !(a > 0 && a <= 1.5)) return fail(nullptr, PMR_EINVAL, "bad argument");
    if (D) *D = growth_D(a, cfg->omega_m);
    if (Gp) *Gp = growth_Gp(a, cfg->omega_m);
    if (Gf) *Gf = growth_Gf(a, cfg->omega_m);
    return PMR_OK;
}

int64_t pmr_launch_count(const pmr_ctx* c) { return c ? c->launches : -1; }

int64_t pmr_forward_id(const pmr_ctx* c) { return (c && c->have_forward) ? c->fwd_id : -1; }

int pmr_timing(pmr_ctx* c, int enable) {
    PMR_TRY(check_ctx(c));
    c->timing = enable != 0;
    c->ev_used = 0;
    if (c->timing) record_event(c, "begin");
    return PMR_OK;
}

int pmr_timing_report(pmr_ctx* c, char* buf, size_t len) {
    PMR_TRY(check_ctx(c));
    if (!buf || len == 0) return fail(c, PMR_EINVAL, "NULL buffer");
    PMR_TRY(check_cuda(c, cudaStreamSynchronize(c->stream), "sync"));
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<int64_t> cnt;
    for (size_t i = 1; i < c->ev_used; ++i) {
        float t = 0.f;
        PMR_TRY(check_cuda(c, cudaEventElapsedTime(&t, c->ev_pool[i - 1], c->ev_pool[i]), "elapsed"));
        const std::string nm = c->ev_names[i];
        size_t k = 0;
        while (k < names.size() && names[k] != nm) ++k;
        if (k == names.size()) {
            names.push_back(nm);
            ms.push_back(0.0);
            cnt.push_back(0);
        }
        ms[k] += t;
        cnt[k] += 1;
    }
    std::string out;
    for (size_t k = 0; k < names.size(); ++k)
        out += names[k] + " " + std::to_string(cnt[k]) + " " + std::to_string(ms[k]) + "\n";
    std::strncpy(buf, out.c_str(), len - 1);
    buf[len - 1] = 0;
    c->ev_used = 0;
    if (c->timing) record_event(c, "begin");
    return out.size() < len ? PMR_OK : fail(c, PMR_EINVAL, "report truncated");
}

int pmr_lbfgs_direction(pmr_ctx* c, const double* g, const double* S, const double* Y, int k, int64_t n, double* d) {
    PMR_TRY(check_ctx(c));
    if (!g || !d || (k > 0 && (!S || !Y))) return fail(c, PMR_EINVAL, "NULL argument");
    if (k < 1 || k > c->cfg.lbfgs_m || n < 1 || n > c->lb.n) return fail(c, PMR_EINVAL, "need 1 <= k <= lbfgs_m, n <= 2 N^2 (N/2+1)");
    std::vector<double> rho(k), sy(k);
    for (int t = 0; t < k; ++t) {
        PMR_TRY(dot64(c, S + (int64_t)t * n, Y + (int64_t)t * n, n, c->red_out + 2));
        PMR_TRY(check_cuda(c, cudaMemcpyAsync(&sy[t], c->red_out + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                           "rb"));
        PMR_TRY(check_cuda(c, cudaStreamSynchronize(c->stream), "sync"));
        rho[t] = 1.0 / sy[t];
    }
    return lbfgs_two_loop(c, g, S, Y, k, 0, k, n, rho.data(), d, false);
}

}  // extern "C"

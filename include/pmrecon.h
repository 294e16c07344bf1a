/*
 * pmrecon.h - C ABI of the GB300 (sm_103a) reconstruction hot path of
 * Modi, Feng & Seljak (2018), "Cosmological reconstruction from galaxy light:
 * neural network based light-matter connection".
 *
 * One call of loss_and_grad() evaluates the loss of Eq. (loss) (Sec. 5.1) at
 * the linear modes s(k) and its gradient w.r.t. s(k): Zel'dovich initial
 * conditions at a0, nsteps particle-mesh kick/drift steps (Sec. 3), the
 * 27-point, 3-field, 81-50-30-1 network of Sec. 2 on the final density, the
 * smoothed displaced-log-normal residual (Eq. probnoise) with the annealed
 * residual smoothing of Sec. 5.2, the Gaussian prior (Eq. priorpdf), and the
 * hand-written adjoint of all of it. recon_step() is one L-BFGS iteration
 * (Sec. 5.2) around it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named *_dev, and every array argument unless stated otherwise,
 *   are CUDA device pointers owned by the caller; the library never frees them
 *   and keeps no reference after the call returns.
 * - Real meshes are float32 [N][N][N], C order (z fastest).
 * - Fourier arrays ("c64") are interleaved complex float32 in the half layout
 *   [N][N][N/2+1] (the real-to-complex layout), with the field defined as
 *   f(x) = N^-3 sum_k s(k) exp(i k.x). Real and imaginary parts of every entry
 *   are independent real variables (Sec. 5.1); gradients are w.r.t. them.
 * - Particle arrays are float32 SoA [3][np] in grid units (cell = L/N Mpc/h);
 *   the j-th component of particle i is at p[j*np + i].
 * - All work is enqueued on the context's stream and is asynchronous unless a
 *   function says it synchronises (those that return host scalars do).
 * - Every function returns PMR_OK (0) or a negative PMR_E* code; the message
 *   of the last failure is available from pmr_last_error(). A failed call
 *   leaves output buffers in an unspecified state but the context usable.
 */
#ifndef PMRECON_H
#define PMRECON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMR_OK 0
#define PMR_EINVAL (-1)      /* bad argument or configuration */
#define PMR_ENOMEM (-2)      /* device allocation failed */
#define PMR_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed */
#define PMR_ENAN (-4)        /* loss is not finite (e.g. M_R + M0 <= 0) */
#define PMR_ELINESEARCH (-5) /* no Armijo step within 20 halvings */
#define PMR_ESTATE (-6)      /* call order violated (e.g. adjoint before forward) */
#define PMR_ETIMEOUT (-7)    /* a tensor-core kernel's bounded barrier wait ran out (its outputs are
                                invalid; the kernel freed its tensor memory and the context stays usable) */

/* Problem definition. pmr_default_config() fills the synthetic 32^3 workload. */
typedef struct pmr_config {
    int N;              /* mesh side; N = 2^a 3^b, 8 <= N <= 512; one particle per cell */
    double L;           /* box side, Mpc/h */
    int nsteps;         /* PM kick-drift steps, uniform in a from a0 to 1 (Sec. 3: 5) */
    double a0;          /* scale factor of the initial conditions (Sec. 3: z = 9) */
    double omega_m;     /* Sec. 3: 0.3175 (flat LCDM) */
    double sigma8;      /* linear amplitude of the BBKS spectrum */
    double gamma_bbks;  /* BBKS shape parameter */
    double R_feat[3];   /* Gaussian scales of the three smoothed density fields, Mpc/h (Sec. 2.2);
                           0 = the unsmoothed density */
    float feat_mix[9];  /* row-major 3x3 C: the network's input fields are f_i = sum_j C_ij delta_Rj
                           (Sec. 2.2 uses delta_0, delta_R1, delta_R1 - delta_R2: R_feat = {0, R1, R2},
                           C = {1,0,0, 0,1,0, 0,1,-1}); identity by default. pmr_create folds C into the
                           first-layer weights (and the mass network's, head == 1), so it costs nothing */
    double R_M;         /* smoothing of model and data mass inside the log, Mpc/h (Sec. 4.2: 3) */
    double sigma_N2;    /* noise variance of Eq. (loss) (Sec. 5.3: 0.25) */
    double mu_N;        /* offset of Eq. (loss) */
    double f_eff;       /* effective-points factor of Eq. (loss) (Sec. 5.1: 1) */
    double M_scale;     /* halo mass per unit softplus output, M_sun/h */
    int lbfgs_m;        /* L-BFGS memory (correction pairs), 1..64 */
    double lbfgs_tol;   /* relative loss decrease that counts as converged (Sec. 5.3: 1e-3) */
    int nn_path;        /* network arithmetic: 0 = tensor cores (tcgen05), each operand split
                           into two TF32 parts, float32 accuracy (default); 1 = tensor cores,
                           plain TF32 (~1e-3 relative); 2 = float32 CUDA cores; 3 = tensor
                           cores with bfloat16 operands and float32 accumulation (~3e-3) */
    int head;           /* 0 = one network with a softplus output, M = M_scale ln(1 + e^y);
                           1 = the paper's two networks (Sec. 2.1), M = M_scale *
                           logistic(y, a) * NNm(f), NNm = 3-20-10-1 ELU net on the voxel's
                           three fields; its 301 weights follow the 5661 of pmr_create */
    int lpt_order;      /* initial conditions (Sec. 3): 1 = Zel'dovich; 2 = second-order LPT,
                           x = q + D1 psi1 + D2 psi2, D2 = -3/7 D1^2, psi2 = grad phi2 with
                           lap phi2 = sum_{i<j} (phi_ii phi_jj - phi_ij^2) of the first-order
                           potential (lap phi = delta). Needs 12 more float32 meshes. */
} pmr_config;

/* Per-stage annealing parameters of Sec. 5.2. */
typedef struct pmr_anneal {
    double R_sm;       /* Gaussian smoothing of the residual, Mpc/h; 0 = none */
    double M0;         /* nuisance mass added inside the log, M_sun/h (Eq. var) */
    double a_logistic; /* sharpness of the logistic position output (Eq. logistic;
                          annealed 1, 2, 3); used when head == 1 */
} pmr_anneal;

typedef struct pmr_ctx pmr_ctx;

/* Fills *cfg with the defaults: N=32, L=100, nsteps=3, a0=0.1, omega_m=0.3175,
 * sigma8=0.8, Gamma=0.21, R_feat={1,2,4}, feat_mix=identity, R_M=3, sigma_N2=0.25, mu_N=0,
 * f_eff=1, M_scale=1e12, lbfgs_m=10, lbfgs_tol=1e-3, nn_path=0, head=0,
 * lpt_order=1. */
void pmr_default_config(pmr_config* cfg);

/* Device bytes pmr_create() will allocate for this configuration (used to
 * admit jobs by HBM footprint). Returns 0 for an invalid configuration. */
size_t pmr_workspace_bytes(const pmr_config* cfg);

/* Creates a context: validates cfg, allocates the workspace on the current
 * device, computes the growth factors and the linear power table on the host
 * (float64), and copies the network weights.
 * nn_weights_dev: device float32[5661] laid out W1[50][81], b1[50], W2[30][50],
 *   b2[30], w3[30], b3; input index c*27 + (ox+1)*9 + (oy+1)*3 + (oz+1) for
 *   field c and neighbour offset (ox,oy,oz) (Sec. 2.1-2.2); with head == 1,
 *   float32[5962]: the same followed by the mass network's Wm1[20][3], bm1[20],
 *   Wm2[10][20], bm2[10], wm3[10], bm3. Copied.
 * stream: a cudaStream_t (NULL = legacy default stream). */
int pmr_create(const pmr_config* cfg, const float* nn_weights_dev, void* stream, pmr_ctx** out);
int pmr_destroy(pmr_ctx* ctx);
int pmr_set_stream(pmr_ctx* ctx, void* stream);

/* Serving aid (no counterpart in the paper): with enable != 0, the launches of
 * one loss_and_grad evaluation (the ~480 kernels of the ICs, PM steps, network,
 * loss and adjoint) are captured once into a CUDA graph and replayed as one
 * graph launch for every later evaluation with the same s_k, data, anneal
 * parameters and gradient buffer (recon_step's line-search trials, repeated
 * loss_and_grad calls); any change re-captures. Results are identical to the
 * direct launches. Capture is thread-local, so other threads may keep using
 * CUDA meanwhile. Needs a context on a non-default stream (PMR_EINVAL
 * otherwise); enable = 0 drops the graph. */
int pmr_use_graphs(pmr_ctx* ctx, int enable);
const char* pmr_last_error(const pmr_ctx* ctx);

/* ---------------------------------------------------------------- the path */

/* Linear modes from white noise: s(k) = amplitude * sqrt(P(k) N^6 / L^3 / N^3)
 * * rfft(white)(k), s(0) = 0, so <|s|^2> = amplitude^2 P(k) N^6/L^3 (the
 * Gaussian field of Eq. priorpdf; amplitude^2 = 0.1 gives the 10%-power
 * starting point of Sec. 5.3). white: float32 mesh. s_k: c64 half array. */
int pmr_linear_field(pmr_ctx* ctx, const float* white, double amplitude, void* s_k);

/* Forward PM model (Sec. 3): s(k) -> final overdensity delta = rho/rho_bar - 1
 * (CIC, Sec. 2). Stores the per-step particle positions in the context for
 * pm_adjoint(). s_k: c64 half array; delta_out: float32 mesh. */
int pm_forward(pmr_ctx* ctx, const void* s_k, float* delta_out);

/* Adjoint of the last pm_forward() on this context (Sec. 5.2, PM derivatives
 * written by hand): grad_s_k = (d delta/d s)^T grad_delta, from the per-step
 * positions, sorts and force fields the forward stored. Returns PMR_ESTATE
 * without a forward. */
int pm_adjoint(pmr_ctx* ctx, const float* grad_delta, void* grad_s_k);

/* Network halo-mass map (Sec. 2): delta -> three Gaussian-smoothed fields,
 * mixed by feat_mix -> per-voxel 81-50-30-1 ReLU network on the 3x3x3
 * neighbourhood -> M_scale * softplus(y), or with head == 1 M_scale *
 * logistic(y, a) * NNm (Sec. 2.1). delta, mass_out: float32 meshes.
 * an: only a_logistic is read (NULL means a = 3). */
int nn_halo_map(pmr_ctx* ctx, const float* delta, float* mass_out, const pmr_anneal* an);

/* Adjoint of nn_halo_map at delta: grad_delta = (dM/d delta)^T grad_mass.
 * The network's gradient depends on where it is taken, so delta is an
 * argument (the call recomputes the forward at delta first). */
int nn_halo_map_adjoint(pmr_ctx* ctx, const float* delta, const float* grad_mass, float* grad_delta,
                        const pmr_anneal* an);

/* Loss of Eq. (loss) at s(k) and its gradient (Sec. 5.1-5.2).
 * data_mass: float32 mesh of the observed halo mass M^data (unsmoothed).
 * loss_out: double[3] = {total, prior, residual}, or NULL (nothing returned).
 *   A HOST pointer: the call synchronises the stream, returns PMR_ENAN for a
 *   non-finite loss and PMR_ETIMEOUT for a timed-out tensor-core wait. A
 *   DEVICE pointer: the values are written on the stream, the call does not
 *   synchronise (a non-finite loss shows as NaN/Inf in loss_out; pmr_sync()
 *   reports a timed-out wait).
 * grad_s_k: c64 half array, may alias nothing else. */
int loss_and_grad(pmr_ctx* ctx, const void* s_k, const float* data_mass, const pmr_anneal* an,
                  double* loss_out, void* grad_s_k);

/* One L-BFGS iteration (Sec. 5.2) on s(k) in place: two-loop direction from the
 * context's history (float64 on the device), Armijo backtracking (step 1,
 * halved up to 20 times, c1 = 1e-4), history update. The initial inverse
 * Hessian is gamma D with D = P~(k)/w_k, the Gaussian prior's exact inverse
 * Hessian, and gamma = s^T y / y^T D y of the newest pair. The first call after
 * pmr_lbfgs_reset() (or after any annealing parameter changes) evaluates the
 * gradient at s first and searches along -D g.
 * loss_out: HOST double[3] of the accepted point. converged: HOST int, set to 1
 * when (L_old - L_new) < lbfgs_tol * |L_old| (Sec. 5.3 stop rule). Synchronises. */
int recon_step(pmr_ctx* ctx, void* s_k, const float* data_mass, const pmr_anneal* an,
               double* loss_out, int* converged);
int pmr_lbfgs_reset(pmr_ctx* ctx);

/* -------------------------------------------- single steps (for parity tests) */

/* Cell keys and stable counting sort of np particles (CIC, Sec. 2):
 * key = (floor(wx) N + floor(wy)) N + floor(wz) with w = fmod(u, N), +N if
 * negative (float32), 0 if the result is N. perm lists particle indices by
 * (key, index); cell_start[N^3+1] holds segment offsets. keys, perm: uint32[np]. */
int pmr_cell_sort(pmr_ctx* ctx, const float* x, int64_t np, uint32_t* keys, uint32_t* perm,
                  uint32_t* cell_start);

/* CIC density by a cell-sorted segmented gather (no float atomics; fixed
 * summation order): rho(c) = sum of mass * CIC weight over the particles of
 * the 8 bins c - o, each bin's corner sums taken over its particles in sorted
 * order and then combined along z, y and x in a fixed order, so repeated calls
 * give the same bits. mass: float32[np] or NULL for unit mass. rho: float32 mesh. */
int pmr_paint(pmr_ctx* ctx, const float* x, int64_t np, const float* mass, float* rho);

/* The same deterministic CIC paint as pmr_paint(), for callers that cannot
 * allocate device memory. The paper has no counterpart: this entry point exists
 * for the library's users. pmr_paint() needs a context, and pmr_create() calls
 * cudaMalloc; code that runs while a CUDA graph is being captured, framework
 * plug-ins whose host owns every device allocation, and loops that must not
 * let cudaMalloc/cudaFree synchronise the device cannot make that call. This
 * variant allocates nothing: its sorting scratch (about 9.4 MB) is one fixed
 * array in device memory that every GPU loading the library holds until the
 * process exits. Limits: 8 <= N <= 64 (N^3 <= 262144 cells) and
 * 0 <= np <= N^3 particles (the bounds of pmr_paint() on a context);
 * other sizes return PMR_EINVAL. The first call on a device looks up the array's
 * device address (with that device current), so make that first call before
 * any stream capture. All calls share the one array, whose contents are left
 * from the previous call: calls whose work overlaps on the GPU (different
 * streams, or the same stream from several host threads without ordering)
 * race and must be serialised by the caller.
 * x: float32 [3][np] absolute positions (same wrap rule as pmr_cell_sort);
 * mass: float32[np] or NULL for unit mass; rho: float32 [N][N][N] output;
 * stream: cudaStream_t or NULL. Errors: PMR_EINVAL, PMR_ECUDA (message from
 * pmr_last_error(NULL)). */
int pmr_paint_noalloc(int N, const float* x, int64_t np, const float* mass, float* rho, void* stream);

/* CIC interpolation of a mesh at np positions (the transpose of paint). */
int pmr_readout(pmr_ctx* ctx, const float* field, const float* x, int64_t np, float* out);

/* Gradient of CIC interpolation w.r.t. position: out[3][np]. */
int pmr_readout_grad(pmr_ctx* ctx, const float* field, const float* x, int64_t np, float* out);

/* Real-to-complex 3D FFT (unnormalised) and its inverse (with 1/N^3, imaginary
 * parts of self-conjugate entries ignored). in/out per the conventions above. */
int pmr_rfft(pmr_ctx* ctx, const float* in, void* out);
int pmr_irfft(pmr_ctx* ctx, const void* in, float* out);

/* PM force F = -grad phi, lap phi = 1.5 Omega_m delta, spectral (i k / k^2,
 * zero at k = 0 and on each component's Nyquist plane). F: float32 [3][N^3]. */
int pmr_force(pmr_ctx* ctx, const float* delta, float* F);

/* Gaussian smoothing exp(-k^2 R^2 / 2), R in Mpc/h; R = 0 copies. */
int pmr_smooth(pmr_ctx* ctx, const float* in, double R, float* out);

/* Zel'dovich ICs at a0 (Sec. 3): x = q + D(a0) psi, p = G_p(a0) psi with
 * psi_k = i k s_k / k^2 (k = 2 pi n / N in grid units). Returns the
 * displacement disp = x - q (q = the particle's lattice point, particle index
 * (ix N + iy) N + iz) and p, both float32 [3][N^3]. */
int pmr_za_ics(pmr_ctx* ctx, const void* s_k, float* disp, float* p);

/* Initial conditions of the configured order (lpt_order; Sec. 3). Order 1 is
 * pmr_za_ics; order 2 adds D2 psi2 to the displacement and Gp2 psi2 to p,
 * with D2 = -3/7 D1^2 and Gp2 = a^3 E dD2/da = -6/7 D1 G_p. Same layouts. */
int pmr_lpt_ics(pmr_ctx* ctx, const void* s_k, float* disp, float* p);

/* Adjoint of pmr_lpt_ics at s_k: grad_s_k = (d disp/ds)^T lam_x + (d p/ds)^T lam_p
 * (c64 half array, overwritten). lam_x, lam_p: float32 [3][N^3]. The
 * second-order term is quadratic in s, so its adjoint depends on s_k.
 * With lpt_order == 2 both calls replace state pm_adjoint needs: the next
 * pm_adjoint returns PMR_ESTATE until pm_forward runs again. */
int pmr_lpt_ics_adjoint(pmr_ctx* ctx, const void* s_k, const float* lam_x, const float* lam_p, void* grad_s_k);

/* Growth factors the stepping uses (float64, host): D(a), G_p(a), G_f(a). */
int pmr_growth(const pmr_config* cfg, double a, double* D, double* Gp, double* Gf);

/* L-BFGS two-loop direction d = -H g (Sec. 5.2) for k pairs, float64 device
 * vectors of length n: S and Y are [k][n], oldest first. */
int pmr_lbfgs_direction(pmr_ctx* ctx, const double* g, const double* S, const double* Y, int k,
                        int64_t n, double* d);

/* Two-point statistics of Sec. 4.3: binned auto and cross power spectra of two
 * float32 meshes a (e.g. the data, "h") and b (the model, "N"), from which the
 * host forms r_c = P_ab / sqrt(P_aa P_bb), s = P_aa (1 - r_c^2) and
 * TF = sqrt(P_bb / P_aa). Shell i (i < N/2) holds the modes with integer
 * wavevector norm i + 1/2 <= |n| < i + 3/2, k = 2 pi n / L (nominal k =
 * (i + 1) 2 pi / L h/Mpc); modes are counted over the full grid.
 * P_ab = L^3 / N^6 < Re(A conj B) > with A = unnormalised DFT of a.
 * out: HOST double[4][N/2] = {mode counts, P_aa, P_bb, P_ab} ((Mpc/h)^3).
 * The first call allocates the context's shell table. Synchronises. */
int pmr_power_spectra(pmr_ctx* ctx, const float* a, const float* b, double* out);

/* The statistics of Sec. 4.3 per |k| shell, formed on the device in float64
 * from the spectra of pmr_power_spectra() with a = h (the truth or data) and
 * b = m (the model): cross-correlation r_c = P_hm / sqrt(P_hh P_mm),
 * stochasticity s = P_hh (1 - r_c^2) ((Mpc/h)^3) and transfer function
 * TF = sqrt(P_mm / P_hh). Shells as in pmr_power_spectra(); a shell whose
 * spectrum is zero gives NaN statistics.
 * out: HOST double[7][N/2] = {mode counts, P_hh, P_mm, P_hm, r_c, s, TF}.
 * Synchronises. */
int pmr_two_point(pmr_ctx* ctx, const float* h, const float* m, double* out);

/* Synchronises the context's stream and reports what the asynchronous calls
 * since the last report could not: PMR_ETIMEOUT if a tensor-core network
 * kernel's bounded wait ran out (the flag is cleared), PMR_ECUDA for a failed
 * kernel. */
int pmr_sync(pmr_ctx* ctx);

/* Failure-detection test hook (no counterpart in the paper). With enable != 0
 * the tensor-core network kernels of this context issue no MMAs and bound their
 * barrier waits at a short limit, so every wait for an accumulator runs out:
 * each kernel records the timeout, waits for nothing in flight, frees its
 * tensor memory and returns, and the next synchronising call reports
 * PMR_ETIMEOUT. enable = 0 restores normal launches. PMR_EINVAL for nn_path 2. */
int pmr_test_stall_mma(pmr_ctx* ctx, int enable);

/* ------------------------------------------------------------- instrumentation */

/* Number of kernels this context has launched since creation. */
int64_t pmr_launch_count(const pmr_ctx* ctx);

/* Identifier of the forward trajectory (Sec. 5.2: the stored per-step particle
 * positions) that the next pm_adjoint() would differentiate: a count of the
 * forward sweeps this context has completed (pm_forward, loss_and_grad,
 * recon_step each run one), or -1 when there is none (no forward yet, a failed
 * sweep, or a call that replaced the state pm_adjoint needs). A caller that
 * holds the value from its own forward can detect that another call has
 * replaced the trajectory since. No synchronisation. */
int64_t pmr_forward_id(const pmr_ctx* ctx);

/* Per-kernel timing with CUDA events on the context stream. enable != 0
 * starts recording one event after every kernel launch (cost: one event
 * record per launch); pmr_timing_report() synchronises the stream and writes
 * one line per kernel name, "name launches total_ms", attributing to each
 * launch the time since the previous recorded event (kernels run back to
 * back on one stream, so this is the kernel's duration plus any idle gap),
 * then restarts the window. buf: host char[len]. */
int pmr_timing(pmr_ctx* ctx, int enable);
int pmr_timing_report(pmr_ctx* ctx, char* buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* PMRECON_H */

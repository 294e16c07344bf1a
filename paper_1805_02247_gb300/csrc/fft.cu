// 3D real FFTs on the N^3 mesh as three shared-memory passes (z, y, x),
// with the Fourier-space multipliers of the method (PM Green's function and
// gradient, Gaussian smoothing, Zel'dovich displacement, linear power) fused
// into the x-pass, where every element holds its full (kx, ky, kz) value.
//
// Layouts: real [x][y][z]; half complex [x][y][kz], kz < P = N/2 + 1.
// Forward r2c = z-pass (real rows -> P complex), y-pass, x-pass.
// Inverse c2r = x-pass, y-pass, z-pass (P complex -> real rows, 1/N^3).
// Each pass reads and writes the array once (HBM bound); 1D transforms are
// mixed-radix (4, 3, 2) Stockham autosort in shared memory with float64-built
// twiddle tables.
#include <cmath>
#include <map>
#include <mutex>

#include "common.cuh"

namespace pmr {

bool radix_ok(int n) {
    if (n < 2) return false;
    while (n % 4 == 0) n /= 4;
    while (n % 3 == 0) n /= 3;
    while (n % 2 == 0) n /= 2;
    return n == 1;
}

Radix make_radix(int n) {
    Radix r{};
    r.n = n;
    int m = n;
    while (m % 4 == 0 && m > 4) { r.r[r.nr++] = 4; m /= 4; }
    while (m % 3 == 0 && m > 1) { r.r[r.nr++] = 3; m /= 3; }
    if (m == 4) { r.r[r.nr++] = 4; m = 1; }
    if (m == 2) { r.r[r.nr++] = 2; m = 1; }
    int Ns = 1;
    for (int s = 0; s < r.nr; ++s) {
        r.ns[s] = FastDiv((uint32_t)Ns);
        r.nrd[s] = FastDiv((uint32_t)(n / r.r[s]));
        Ns *= r.r[s];
    }
    return r;
}

namespace {

constexpr int kThreads = 256;
constexpr int kCols = 8;      // columns (kz) per y/x-pass tile
constexpr int kRows = 8;      // real rows per z-pass tile
constexpr int kColsT = kCols, kColsLog = 3;
static_assert((1 << kColsLog) == kCols, "kCols is a power of two");

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// R-point DFT in registers; INV uses exp(+2 pi i / R).
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
    if constexpr (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        float2 t2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        // forward: -i * d, inverse: +i * d
        float2 t3 = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else {  // R == 3
        const float h = 0.86602540378443864676f;  // sqrt(3)/2
        float2 a = v[0], s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
        float2 m = make_float2(a.x - 0.5f * s.x, a.y - 0.5f * s.y);
        // +-i h d
        float2 r = INV ? make_float2(-h * d.y, h * d.x) : make_float2(h * d.y, -h * d.x);
        v[0] = cadd(a, s);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
}

// One Stockham stage over `ncols` independent transforms of length n; element
// (m, c) lives at buf[m*es + c*cs]. COLFAST maps consecutive threads to
// consecutive columns (es = ncols, cs = 1 layouts).
template <int R, bool INV, bool COLFAST>
__device__ __forceinline__ void stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                      const float2* __restrict__ tw, int n, const FastDiv& nsd, const FastDiv& nrd,
                                      int ncols, int es, int cs) {
    const int Ns = (int)nsd.d;
    const int nR = n / R;
    const int W = nR * ncols;
    const int tstride = n / (Ns * R);
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        int c, j;
        if (COLFAST) { c = w & (kColsT - 1); j = w >> kColsLog; }
        else { c = (int)nrd.div((uint32_t)w); j = w - c * nR; }
        const int jq = (int)nsd.div((uint32_t)j);
        const int k = j - jq * Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            v[r] = src[(j + r * nR) * es + c * cs];
            if (r > 0) {
                float2 t = tw[r * k * tstride];
                if (INV) t.y = -t.y;
                v[r] = cmul(v[r], t);
            }
        }
        dft<R, INV>(v);
        const int idxD = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(idxD + r * Ns) * es + c * cs] = v[r];
    }
}

// Full transform; data starts in a, b is scratch; returns the buffer holding
// the result. Ends with __syncthreads().
template <bool INV, bool COLFAST>
__device__ float2* smem_fft(float2* a, float2* b, const float2* tw, const Radix& rd, int ncols, int es, int cs) {
    float2* src = a;
    float2* dst = b;
    for (int s = 0; s < rd.nr; ++s) {
        const int R = rd.r[s];
        if (R == 4) stage<4, INV, COLFAST>(src, dst, tw, rd.n, rd.ns[s], rd.nrd[s], ncols, es, cs);
        else if (R == 2) stage<2, INV, COLFAST>(src, dst, tw, rd.n, rd.ns[s], rd.nrd[s], ncols, es, cs);
        else stage<3, INV, COLFAST>(src, dst, tw, rd.n, rd.ns[s], rd.nrd[s], ncols, es, cs);
        __syncthreads();
        float2* t = src; src = dst; dst = t;
    }
    return src;
}

__device__ __forceinline__ void load_twiddles(float2* s_tw, const float2* g_tw, int n) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) s_tw[t] = g_tw[t];
}

// Tile loads with every global load of a thread issued before the first
// shared-memory store, so a block keeps its whole tile in flight.
constexpr int kMaxPer = 16;  // (512 * kCols) / kThreads

// column tile: element t = m * kCols + c at in[base + m * es + c], c < cw valid
__device__ __forceinline__ void load_col_tile(float2* A, const float2* in, int64_t base, int64_t es,
                                              int n, int cw) {
    const int T = n * kCols;
    float2 r[kMaxPer];
#pragma unroll
    for (int q = 0; q < kMaxPer; ++q) {
        const int t = threadIdx.x + q * kThreads;
        const int m = t / kCols, c = t % kCols;
        r[q] = (t < T && c < cw) ? in[base + m * es + c] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < kMaxPer; ++q) {
        const int t = threadIdx.x + q * kThreads;
        if (t < T) A[t] = r[q];
    }
}

// Row tiles of the z-pass: one warp per row (kThreads / 32 == kRows), lanes
// stride along the row, so no index needs a division.
constexpr int kMaxRowPer = 9;  // ceil((512/2 + 1) / 32)
static_assert(kThreads / 32 == kRows, "one warp per z-pass row");

// rows r < rows of len complex each at src[r * len + m] -> A[r * ld + m];
// every load of a thread is issued before its first shared-memory store
__device__ __forceinline__ void load_row_tile(float2* A, const float2* __restrict__ src, int len, int ld, int rows) {
    const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 v[kMaxRowPer];
#pragma unroll
    for (int i = 0; i < kMaxRowPer; ++i) {
        const int m = lane + 32 * i;
        v[i] = (r < rows && m < len) ? src[(int64_t)r * len + m] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < kMaxRowPer; ++i) {
        const int m = lane + 32 * i;
        if (m < len) A[r * ld + m] = v[i];
    }
}

// ----------------------------------------------------------------------------- z passes

// Real rows of length N -> P = N/2+1 complex, through one complex FFT of
// length M = N/2 on z_m = x_2m + i x_2m+1 and the even/odd split
// X_k = E_k + exp(-2 pi i k / N) O_k.
__global__ void __launch_bounds__(kThreads) k_z_r2c(const float* __restrict__ in, float2* __restrict__ out,
                                                      int64_t nrows, int N, Radix rM,
                                                      const float2* __restrict__ twM, const float2* __restrict__ twN) {
    extern __shared__ float2 sm[];
    const int M = N / 2, P = M + 1, ld = M + 1;
    float2* s_twM = sm;
    float2* s_twN = s_twM + M;
    float2* A = s_twN + N;
    float2* B = A + kRows * ld;
    load_twiddles(s_twM, twM, M);
    load_twiddles(s_twN, twN, N);
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    const int rows = (int)min((int64_t)kRows, nrows - row0);
    load_row_tile(A, reinterpret_cast<const float2*>(in + row0 * N), M, ld, rows);
    __syncthreads();
    float2* Z = smem_fft<false, false>(A, B, s_twM, rM, kRows, 1, ld);
    const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (r < rows) {
        for (int k = lane; k < P; k += 32) {
            float2 zk = Z[r * ld + (k == M ? 0 : k)];
            float2 zc = Z[r * ld + (k == 0 ? 0 : M - k)];
            zc.y = -zc.y;
            float2 e = cscale(cadd(zk, zc), 0.5f);
            float2 dd = csub(zk, zc);
            float2 o = make_float2(0.5f * dd.y, -0.5f * dd.x);  // -i/2 (zk - zc)
            out[(row0 + r) * P + k] = cadd(e, cmul(s_twN[k], o));
        }
    }
}

// P complex -> real rows with scale; the imaginary parts of X_0 and X_M are
// ignored (they carry no information for a real signal).
__global__ void __launch_bounds__(kThreads) k_z_c2r(const float2* __restrict__ in, float* __restrict__ out,
                                                      int64_t nrows, int N, float scale, Radix rM,
                                                      const float2* __restrict__ twM, const float2* __restrict__ twN) {
    extern __shared__ float2 sm[];
    const int M = N / 2, P = M + 1, ld = M + 1;
    float2* s_twM = sm;
    float2* s_twN = s_twM + M;
    float2* X = s_twN + N;
    float2* A = X + kRows * ld;
    float2* B = A + kRows * ld;
    load_twiddles(s_twM, twM, M);
    load_twiddles(s_twN, twN, N);
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    const int rows = (int)min((int64_t)kRows, nrows - row0);
    load_row_tile(X, in + row0 * P, P, ld, rows);
    __syncthreads();
    const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = lane; k < M; k += 32) {
        float2 xk = X[r * ld + k];
        float2 xc = X[r * ld + (M - k)];
        if (k == 0) {  // X_0 and X_M: imaginary parts carry nothing for a real signal
            xk.y = 0.f;
            xc.y = 0.f;
        }
        xc.y = -xc.y;
        float2 e = cscale(cadd(xk, xc), 0.5f);
        float2 w = s_twN[k];
        w.y = -w.y;  // exp(+2 pi i k / N)
        float2 o = cmul(cscale(csub(xk, xc), 0.5f), w);
        A[r * ld + k] = make_float2(e.x - o.y, e.y + o.x);  // e + i o
    }
    __syncthreads();
    float2* z = smem_fft<true, false>(A, B, s_twM, rM, kRows, 1, ld);
    float2* dst = reinterpret_cast<float2*>(out + row0 * N);
    const float s = scale * 2.0f / (float)N;
    if (r < rows)
        for (int m = lane; m < M; m += 32) dst[(int64_t)r * M + m] = cscale(z[r * ld + m], s);
}

// ----------------------------------------------------------------------------- y / x passes

struct ColGeom {
    int n;               // transform length (N)
    int ncols;           // P
    int64_t es;          // element stride along the transform axis
    int64_t os;          // stride of the outer (tile row) index
};

// Plain column pass (y-pass, or an x-pass without multipliers).
template <bool INV>
// in and out may be the same array (in-place pass): each block reads its whole
// tile before writing it, and tiles are disjoint.
__global__ void __launch_bounds__(kThreads) k_col(const float2* in, float2* out,
                                                    ColGeom g, Radix rd, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    const int n = g.n;
    float2* s_tw = sm;
    float2* A = s_tw + n;
    float2* B = A + n * kCols;
    load_twiddles(s_tw, tw, n);
    const int c0 = blockIdx.x * kCols;
    const int cw = min(kCols, g.ncols - c0);
    const int64_t base = (int64_t)blockIdx.y * g.os + c0;
    load_col_tile(A, in, base, g.es, n, cw);
    __syncthreads();
    float2* R = smem_fft<INV, true>(A, B, s_tw, rd, kCols, kCols, 1);
    for (int t = threadIdx.x; t < n * kCols; t += blockDim.x) {
        int m = t / kCols, c = t % kCols;
        if (c < cw) out[base + m * g.es + c] = R[t];
    }
}

struct XFused {
    const float2* in[3];
    float2* out[3];
    int nin, nout;
    int fwd;  // forward transform along x before the multiply
    int inv;  // inverse transform along x after it
    int acc;  // add the result to out instead of storing it
    Mul mul[3];
    const float* ptab;  // sqrt power table for MUL_POWER
    // all multipliers are MUL_ODD with j = their index and one scale and
    // weighting: the shared factor scale/k^2 is applied once per element
    int odd3;
};

__device__ __forceinline__ float2 apply_mul(const Mul& m, float2 v, int nx, int ny, int kz, int N,
                                            const float* __restrict__ ptab) {
    const float twopi_n = 6.28318530717958647692f / (float)N;
    float f = m.scale;
    if (m.weighted) f *= (kz == 0 || 2 * kz == N) ? 1.0f : 2.0f;
    if (m.type == MUL_ONE) return cscale(v, f);
    const int n2 = nx * nx + ny * ny + kz * kz;
    if (m.type == MUL_POWER) return cscale(v, f * ptab[n2]);
    const float kx = twopi_n * nx, ky = twopi_n * ny, kzf = twopi_n * kz;
    const float k2 = kx * kx + ky * ky + kzf * kzf;
    if (m.type == MUL_GAUSS) return cscale(v, f * expf(-0.5f * k2 * m.R2));
    if (m.type == MUL_HESS) {
        // k_j k_i2 / k^2, zero at k = 0; for j != i2 also zero where either
        // component is the Nyquist frequency (an odd factor there)
        const int na = (m.j == 0) ? nx : (m.j == 1) ? ny : kz;
        const int nb = (m.i2 == 0) ? nx : (m.i2 == 1) ? ny : kz;
        if (n2 == 0 || (m.j != m.i2 && (2 * abs(na) == N || 2 * abs(nb) == N))) return make_float2(0.f, 0.f);
        return cscale(v, f * (twopi_n * na) * (twopi_n * nb) / k2);
    }
    // MUL_ODD: i k_j / k^2, zero at k = 0 and on the Nyquist plane of component j
    const int nj = (m.j == 0) ? nx : (m.j == 1) ? ny : kz;
    if (n2 == 0 || 2 * abs(nj) == N) return make_float2(0.f, 0.f);
    const float kj = twopi_n * nj;
    const float a = f * kj / k2;
    return make_float2(-a * v.y, a * v.x);
}

// the parts of MUL_ODD: f / k^2 (0 at k = 0), and k_j (0 on the Nyquist plane of j)
__device__ __forceinline__ float odd_g(const Mul& m, int nx, int ny, int kz, int N) {
    const int n2 = nx * nx + ny * ny + kz * kz;
    if (n2 == 0) return 0.f;
    const float twopi_n = 6.28318530717958647692f / (float)N;
    float f = m.scale;
    if (m.weighted) f *= (kz == 0 || 2 * kz == N) ? 1.0f : 2.0f;
    const float kx = twopi_n * nx, ky = twopi_n * ny, kzf = twopi_n * kz;
    return f / (kx * kx + ky * ky + kzf * kzf);
}
__device__ __forceinline__ float odd_k(int j, int nx, int ny, int kz, int N) {
    const int nj = (j == 0) ? nx : (j == 1) ? ny : kz;
    return 2 * abs(nj) == N ? 0.f : (6.28318530717958647692f / (float)N) * nj;
}

// x-pass with multipliers. Tile: outer index = ky row, columns = kz block,
// transform axis = x. nin == 1: out_j = [inv] mul_j * [fwd] in_0.
// nin > 1: out_0 = [inv] sum_i mul_i * [fwd] in_i.
__global__ void __launch_bounds__(kThreads) k_x_fused(XFused p, ColGeom g, Radix rd, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    const int n = g.n, N = n;
    float2* s_tw = sm;
    float2* A = s_tw + n;
    float2* B = A + n * kCols;
    float2* K = B + n * kCols;  // kept k-space tile (nin == 1) or accumulator (nin > 1)
    load_twiddles(s_tw, tw, n);
    const int c0 = blockIdx.x * kCols;
    const int cw = min(kCols, g.ncols - c0);
    const int oy = blockIdx.y;
    const int ny = (2 * oy <= N) ? oy : oy - N;
    const int64_t base = (int64_t)oy * g.os + c0;
    const int T = n * kCols;

    if (p.nin == 1) {
        load_col_tile(A, p.in[0], base, g.es, n, cw);
        __syncthreads();
        const float2* src = A;
        if (p.fwd) src = smem_fft<false, true>(A, B, s_tw, rd, kCols, kCols, 1);
        for (int t = threadIdx.x; t < T; t += blockDim.x) K[t] = src[t];
        __syncthreads();
        for (int o = 0; o < p.nout; ++o) {
            for (int t = threadIdx.x; t < T; t += blockDim.x) {
                int m = t / kCols, c = t % kCols;
                int nx = (2 * m <= N) ? m : m - N;
                // padding columns (kz > N/2) stay zero and never index the power table
                A[t] = (c < cw) ? apply_mul(p.mul[o], K[t], nx, ny, c0 + c, N, p.ptab) : make_float2(0.f, 0.f);
            }
            __syncthreads();
            const float2* R = A;
            if (p.inv) R = smem_fft<true, true>(A, B, s_tw, rd, kCols, kCols, 1);
            for (int t = threadIdx.x; t < T; t += blockDim.x) {
                int m = t / kCols, c = t % kCols;
                if (c < cw) {
                    float2* d = p.out[o] + base + m * g.es + c;
                    *d = p.acc ? cadd(*d, R[t]) : R[t];
                }
            }
            __syncthreads();
        }
    } else {
        for (int t = threadIdx.x; t < T; t += blockDim.x) K[t] = make_float2(0.f, 0.f);
        for (int i = 0; i < p.nin; ++i) {
            load_col_tile(A, p.in[i], base, g.es, n, cw);
            __syncthreads();
            const float2* src = A;
            if (p.fwd) src = smem_fft<false, true>(A, B, s_tw, rd, kCols, kCols, 1);
            for (int t = threadIdx.x; t < T; t += blockDim.x) {
                int m = t / kCols, c = t % kCols;
                int nx = (2 * m <= N) ? m : m - N;
                if (c < cw) K[t] = cadd(K[t], apply_mul(p.mul[i], src[t], nx, ny, c0 + c, N, p.ptab));
            }
            __syncthreads();
        }
        const float2* R = K;
        if (p.inv) R = smem_fft<true, true>(K, A, s_tw, rd, kCols, kCols, 1);
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            int m = t / kCols, c = t % kCols;
            if (c < cw) {
                float2* d = p.out[0] + base + m * g.es + c;
                *d = p.acc ? cadd(*d, R[t]) : R[t];
            }
        }
    }
}

// ----------------------------------------------------------------------------- register column FFTs
//
// Column passes for N = N1 N2 with both factors small: a block takes 16
// adjacent columns (one 128-byte line per row) and each 1D transform runs as
// two rounds of small DFTs held in registers, with one transpose through
// shared memory in between (the four-step decomposition):
//   forward order:  x[N2 n1 + n2]  --DFT_N1 over n1, x W^(n2 k1), DFT_N2 over n2-->  X[k1 + N1 k2]
//   inverse order:  X[k1 + N1 k2]  --DFT_N2 over k2, x W^(n2 k1), DFT_N1 over k1-->  x[n2 + N2 n1]
// Either order computes a DFT of either sign. A thread owns one column and a
// set of n2 (rows N2 n1 + n2) or of k1 (rows k1 + N1 k2), so every global
// access of a warp is two full 128-byte rows and no index needs a division.

constexpr int kRC = 16;  // columns per tile

// R-point DFT in registers, R = 2^a 3^b: X[k + s q] = sum_j W_R^(jk) S_j[k] W_r^(jq),
// S_j the s-point DFT of x[r m + j]. W_R^u = tw[u * TWS] (tw = W_N table).
template <int R, bool INV, int TWS>
__device__ __forceinline__ void dft_reg(float2* v, const float2* tw) {
    if constexpr (R == 2 || R == 3 || R == 4) {
        dft<R, INV>(v);
    } else if constexpr (R > 4) {
        constexpr int r = (R % 4 == 0) ? 4 : (R % 2 == 0) ? 2 : 3;
        constexpr int s = R / r;
        float2 sub[r][s];
#pragma unroll
        for (int j = 0; j < r; ++j)
#pragma unroll
            for (int m = 0; m < s; ++m) sub[j][m] = v[r * m + j];
#pragma unroll
        for (int j = 0; j < r; ++j) dft_reg<s, INV, TWS * r>(sub[j], tw);
#pragma unroll
        for (int k = 0; k < s; ++k) {
            float2 t[r];
#pragma unroll
            for (int j = 0; j < r; ++j) {
                if (j == 0 || k == 0) {
                    t[j] = sub[j][k];
                } else {
                    float2 w = tw[j * k * TWS];
                    if (INV) w.y = -w.y;
                    t[j] = cmul(sub[j][k], w);
                }
            }
            dft<r, INV>(t);
#pragma unroll
            for (int q = 0; q < r; ++q) v[k + s * q] = t[q];
        }
    }
}

constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }

template <int N1_, int N2_>
struct Reg {
    static constexpr int N1 = N1_, N2 = N2_, N = N1 * N2;
    static constexpr int G = cgcd(N1, N2);       // threads per column
    static constexpr int T = kRC * G;            // block size
    static constexpr int A1 = N2 / G;            // n2 values per thread
    static constexpr int A2 = N1 / G;            // k1 values per thread
    static_assert(N1 % G == 0 && N2 % G == 0, "factors must divide");
    static constexpr int E = N / G;              // complex values per thread
    // twiddles + transpose buffer (plain pass); + kept k-space tile (fused pass)
    static constexpr size_t smem_col() { return sizeof(float2) * (size_t)(N + N * kRC); }
    static constexpr size_t smem() { return sizeof(float2) * (size_t)(N + 2 * N * kRC); }
    // resident blocks of the fused x-pass: as many as 80 registers a thread (128 for
    // the several-inputs variant, which spills at 80) and the shared memory of the
    // kept k-space tile allow (3 and 2 at N = 256)
    static constexpr int XB1 = (int)(232448 / smem());
    static constexpr int xb(int regs) {
        const int r = 65536 / (T * regs);
        return (r < XB1 ? r : XB1) > 0 ? (r < XB1 ? r : XB1) : 1;
    }
};

// S[k1][n2][c]
template <class RG>
__device__ __forceinline__ int sidx(int k1, int n2, int c) {
    return (k1 * RG::N2 + n2) * kRC + c;
}

// x[N2 n1 + n2] (thread owns n2 = g + G a) -> X[k1 + N1 k2] (thread owns k1 = g + G a)
template <class RG, bool INV>
__device__ __forceinline__ void four_step_fwd(float2 (&v1)[RG::A1][RG::N1], float2 (&v2)[RG::A2][RG::N2], float2* S,
                                              const float2* tw, int c, int g) {
    constexpr int N1 = RG::N1, N2 = RG::N2, G = RG::G;
#pragma unroll
    for (int a = 0; a < RG::A1; ++a) {
        const int n2 = g + G * a;
        dft_reg<N1, INV, N2>(v1[a], tw);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            float2 v = v1[a][k1];
            if (k1 > 0) {
                float2 w = tw[n2 * k1];
                if (INV) w.y = -w.y;
                v = cmul(v, w);
            }
            S[sidx<RG>(k1, n2, c)] = v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < RG::A2; ++a) {
        const int k1 = g + G * a;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) v2[a][n2] = S[sidx<RG>(k1, n2, c)];
        dft_reg<N2, INV, N1>(v2[a], tw);
    }
    __syncthreads();  // S free again
}

// X[k1 + N1 k2] (thread owns k1) -> x[n2 + N2 n1] (thread owns n2)
template <class RG, bool INV>
__device__ __forceinline__ void four_step_inv(float2 (&v2)[RG::A2][RG::N2], float2 (&v1)[RG::A1][RG::N1], float2* S,
                                              const float2* tw, int c, int g) {
    constexpr int N1 = RG::N1, N2 = RG::N2, G = RG::G;
#pragma unroll
    for (int a = 0; a < RG::A2; ++a) {
        const int k1 = g + G * a;
        dft_reg<N2, INV, N1>(v2[a], tw);
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
            float2 v = v2[a][n2];
            if (n2 > 0 && k1 > 0) {
                float2 w = tw[n2 * k1];
                if (INV) w.y = -w.y;
                v = cmul(v, w);
            }
            S[sidx<RG>(k1, n2, c)] = v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < RG::A1; ++a) {
        const int n2 = g + G * a;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v1[a][k1] = S[sidx<RG>(k1, n2, c)];
        dft_reg<N1, INV, N2>(v1[a], tw);
    }
    __syncthreads();
}

// rows N2 n1 + n2 of the thread's n2 set
template <class RG>
__device__ __forceinline__ void load_n2(float2 (&v1)[RG::A1][RG::N1], const float2* in, int64_t base, int64_t es,
                                        bool ok, int g) {
#pragma unroll
    for (int a = 0; a < RG::A1; ++a)
#pragma unroll
        for (int n1 = 0; n1 < RG::N1; ++n1)
            v1[a][n1] = ok ? in[base + (int64_t)(RG::N2 * n1 + g + RG::G * a) * es] : make_float2(0.f, 0.f);
}

// rows k1 + N1 k2 of the thread's k1 set
template <class RG>
__device__ __forceinline__ void load_k1(float2 (&v2)[RG::A2][RG::N2], const float2* in, int64_t base, int64_t es,
                                        bool ok, int g) {
#pragma unroll
    for (int a = 0; a < RG::A2; ++a)
#pragma unroll
        for (int k2 = 0; k2 < RG::N2; ++k2)
            v2[a][k2] = ok ? in[base + (int64_t)(g + RG::G * a + RG::N1 * k2) * es] : make_float2(0.f, 0.f);
}

__device__ __forceinline__ void put(float2* d, float2 v, bool acc) { *d = acc ? cadd(*d, v) : v; }

// Plain y- or x-pass (no multiplier); in-place safe (the tile is read before any write).
template <class RG, bool INV>
__global__ void __launch_bounds__(RG::T) k_col_reg(const float2* in, float2* out, ColGeom geo,
                                                     const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    float2* s_tw = sm;
    float2* S = s_tw + RG::N;
    load_twiddles(s_tw, tw, RG::N);
    const int c = threadIdx.x % kRC, g = threadIdx.x / kRC;
    const int c0 = blockIdx.x * kRC;
    const bool ok = c0 + c < geo.ncols;
    const int64_t base = (int64_t)blockIdx.y * geo.os + c0 + c;
    float2 v1[RG::A1][RG::N1], v2[RG::A2][RG::N2];
    load_n2<RG>(v1, in, base, geo.es, ok, g);
    __syncthreads();  // twiddles
    four_step_fwd<RG, INV>(v1, v2, S, s_tw, c, g);
    if (ok)
#pragma unroll
        for (int a = 0; a < RG::A2; ++a)
#pragma unroll
            for (int k2 = 0; k2 < RG::N2; ++k2)
                out[base + (int64_t)(g + RG::G * a + RG::N1 * k2) * geo.es] = v2[a][k2];
}

// x-pass with multipliers, same contract as k_x_fused. MODE 0: one input,
// one output; 1: one input, several outputs; 2: several inputs, one output.
template <class RG, int MODE>
__global__ void __launch_bounds__(RG::T, RG::xb(MODE == 2 ? 128 : 80)) k_x_reg(XFused p, ColGeom geo,
                                                                      const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int N = RG::N;
    float2* s_tw = sm;
    float2* S = s_tw + N;
    load_twiddles(s_tw, tw, N);
    const int c = threadIdx.x % kRC, g = threadIdx.x / kRC;
    const int c0 = blockIdx.x * kRC;
    const bool ok = c0 + c < geo.ncols;
    const int kz = c0 + c;
    const int oy = blockIdx.y;
    const int ny = (2 * oy <= N) ? oy : oy - N;
    const int64_t base = (int64_t)oy * geo.os + c0 + c;
    __syncthreads();  // twiddles

    float2* Kb = S + N * kRC;  // kept k-space tile: value e of thread t at Kb[e * T + t]
    float2 v1[RG::A1][RG::N1];
    auto to_k = [&](const float2* src, float2 (&dst)[RG::A2][RG::N2]) {
        if (p.fwd) {
            load_n2<RG>(v1, src, base, geo.es, ok, g);
            four_step_fwd<RG, false>(v1, dst, S, s_tw, c, g);
        } else {
            load_k1<RG>(dst, src, base, geo.es, ok, g);
        }
    };
    auto mul_into = [&](const Mul& m, const float2 (&src)[RG::A2][RG::N2], float2 (&dst)[RG::A2][RG::N2], bool add) {
#pragma unroll
        for (int a = 0; a < RG::A2; ++a)
#pragma unroll
            for (int k2 = 0; k2 < RG::N2; ++k2) {
                const int mx = g + RG::G * a + RG::N1 * k2;
                const int nx = (2 * mx <= N) ? mx : mx - N;
                // padding columns (kz > N/2) stay zero and never index the power table
                const float2 v = ok ? apply_mul(m, src[a][k2], nx, ny, kz, N, p.ptab) : make_float2(0.f, 0.f);
                dst[a][k2] = add ? cadd(dst[a][k2], v) : v;
            }
    };
    auto emit = [&](float2 (&R)[RG::A2][RG::N2], float2* dst) {
        if (p.inv) {
            four_step_inv<RG, true>(R, v1, S, s_tw, c, g);
            if (ok)
#pragma unroll
                for (int a = 0; a < RG::A1; ++a)
#pragma unroll
                    for (int n1 = 0; n1 < RG::N1; ++n1)
                        put(dst + base + (int64_t)(g + RG::G * a + RG::N2 * n1) * geo.es, v1[a][n1], p.acc);
        } else if (ok) {
#pragma unroll
            for (int a = 0; a < RG::A2; ++a)
#pragma unroll
                for (int k2 = 0; k2 < RG::N2; ++k2)
                    put(dst + base + (int64_t)(g + RG::G * a + RG::N1 * k2) * geo.es, R[a][k2], p.acc);
        }
    };

    // i s1 R to dst1 and i s2 R to dst2 through one inverse transform (s1, s2
    // constant along the transform axis)
    auto emit2 = [&](float2 (&R)[RG::A2][RG::N2], float2* dst1, float s1, float2* dst2, float s2) {
        if (p.inv) {
            four_step_inv<RG, true>(R, v1, S, s_tw, c, g);
            if (ok)
#pragma unroll
                for (int a = 0; a < RG::A1; ++a)
#pragma unroll
                    for (int n1 = 0; n1 < RG::N1; ++n1) {
                        const int64_t o = base + (int64_t)(g + RG::G * a + RG::N2 * n1) * geo.es;
                        const float2 v = v1[a][n1];
                        put(dst1 + o, make_float2(-s1 * v.y, s1 * v.x), p.acc);
                        put(dst2 + o, make_float2(-s2 * v.y, s2 * v.x), p.acc);
                    }
        } else if (ok) {
#pragma unroll
            for (int a = 0; a < RG::A2; ++a)
#pragma unroll
                for (int k2 = 0; k2 < RG::N2; ++k2) {
                    const int64_t o = base + (int64_t)(g + RG::G * a + RG::N1 * k2) * geo.es;
                    const float2 v = R[a][k2];
                    put(dst1 + o, make_float2(-s1 * v.y, s1 * v.x), p.acc);
                    put(dst2 + o, make_float2(-s2 * v.y, s2 * v.x), p.acc);
                }
        }
    };
    float2 X[RG::A2][RG::N2];
    if constexpr (MODE == 0) {
        to_k(p.in[0], X);
        mul_into(p.mul[0], X, X, false);
        emit(X, p.out[0]);
    } else if constexpr (MODE == 1) {
        to_k(p.in[0], X);
        {
            // p.odd3: the kept tile is X f/k^2, and output o is i k_o times it
#pragma unroll
            for (int a = 0; a < RG::A2; ++a)
#pragma unroll
                for (int k2 = 0; k2 < RG::N2; ++k2) {
                    float2 v = X[a][k2];
                    if (p.odd3) {
                        const int mx = g + RG::G * a + RG::N1 * k2;
                        v = cscale(v, ok ? odd_g(p.mul[0], (2 * mx <= N) ? mx : mx - N, ny, kz, N) : 0.f);
                    }
                    Kb[(a * RG::N2 + k2) * RG::T + threadIdx.x] = v;
                }
            if (p.odd3) {
                // x component: its k_x varies along the transform axis
#pragma unroll
                for (int a = 0; a < RG::A2; ++a)
#pragma unroll
                    for (int k2 = 0; k2 < RG::N2; ++k2) {
                        const int mx = g + RG::G * a + RG::N1 * k2;
                        const float kj = odd_k(0, (2 * mx <= N) ? mx : mx - N, ny, kz, N);
                        const float2 v = Kb[(a * RG::N2 + k2) * RG::T + threadIdx.x];
                        X[a][k2] = make_float2(-kj * v.y, kj * v.x);
                    }
                emit(X, p.out[0]);
                // y and z components: k_y, k_z are constant along it, so both come
                // from one inverse transform of the kept tile
#pragma unroll
                for (int a = 0; a < RG::A2; ++a)
#pragma unroll
                    for (int k2 = 0; k2 < RG::N2; ++k2) X[a][k2] = Kb[(a * RG::N2 + k2) * RG::T + threadIdx.x];
                emit2(X, p.out[1], odd_k(1, 0, ny, kz, N), p.out[2], odd_k(2, 0, ny, kz, N));
            } else {
#pragma unroll 1
                for (int o = 0; o < p.nout; ++o) {
#pragma unroll
                    for (int a = 0; a < RG::A2; ++a)
#pragma unroll
                        for (int k2 = 0; k2 < RG::N2; ++k2) X[a][k2] = Kb[(a * RG::N2 + k2) * RG::T + threadIdx.x];
                    mul_into(p.mul[o], X, X, false);
                    emit(X, p.out[o]);
                }
            }
        }
    } else {
        // p.odd3: sum_i k_i X_i, then times i f/k^2 once
        float2 acc[RG::A2][RG::N2];
#pragma unroll 1
        for (int i = 0; i < p.nin; ++i) {
            to_k(p.in[i], X);
            if (p.odd3) {
#pragma unroll
                for (int a = 0; a < RG::A2; ++a)
#pragma unroll
                    for (int k2 = 0; k2 < RG::N2; ++k2) {
                        const int mx = g + RG::G * a + RG::N1 * k2;
                        const float2 v = cscale(X[a][k2], odd_k(i, (2 * mx <= N) ? mx : mx - N, ny, kz, N));
                        acc[a][k2] = i > 0 ? cadd(acc[a][k2], v) : v;
                    }
            } else {
                mul_into(p.mul[i], X, acc, i > 0);
            }
        }
        if (p.odd3) {
#pragma unroll
            for (int a = 0; a < RG::A2; ++a)
#pragma unroll
                for (int k2 = 0; k2 < RG::N2; ++k2) {
                    const int mx = g + RG::G * a + RG::N1 * k2;
                    const float gk = ok ? odd_g(p.mul[0], (2 * mx <= N) ? mx : mx - N, ny, kz, N) : 0.f;
                    acc[a][k2] = make_float2(-gk * acc[a][k2].y, gk * acc[a][k2].x);
                }
        }
        emit(acc, p.out[0]);
    }
}

// Tile shapes of the register path: N -> (N1, N2); other N use the shared-memory Stockham kernels.
template <class F>
bool with_reg(int N, F f) {
    switch (N) {
        case 64: f(Reg<8, 8>{}); return true;
        case 128: f(Reg<16, 8>{}); return true;
        case 192: f(Reg<8, 24>{}); return true;
        case 256: f(Reg<16, 16>{}); return true;
        case 512: f(Reg<16, 32>{}); return true;
        default: return false;
    }
}

// ----------------------------------------------------------------------------- register z passes
//
// Rows of N reals are M = N/2 complex points z_m = x_2m + i x_2m+1. A block
// stages R rows in shared memory with coalesced loads, runs the M-point
// transform of each row as the four-step order above (G threads per row,
// one transpose), and applies the real-to-complex split (or its inverse) from
// shared memory, so global reads and writes are whole rows.

template <class RG>
struct ZReg {
    static constexpr int M = RG::N, G = RG::G;
    static constexpr int R = (128 / G) < 8 ? 8 : 128 / G;  // rows per block
    static constexpr int T = R * G;
    // Row pitch of the staging buffer, which also holds the row's transpose
    // (the four-step's S aliases its row): wide enough for both, and = 8 mod 16
    // float2 so the rows of one warp fall on alternating halves of the banks.
    static constexpr int NEED = (M + 9) > RG::N1 * (RG::N2 + 1) ? (M + 9) : RG::N1 * (RG::N2 + 1);
    static constexpr int PITCH = (NEED + 7) / 16 * 16 + 8;
    static constexpr size_t smem() { return sizeof(float2) * (size_t)(M + 2 * M + R * PITCH); }
    static_assert(G <= 32 && 32 % G == 0, "a row's threads lie in one warp");
};

// four-step M-point transform of row r (natural order in A -> natural order in A).
// The G threads of a row are lanes of one warp and the transpose buffer S is
// the row's own staging memory, so warp barriers order the steps.
// TO_REGS: the result stays in v2 (element k1 + N1 k2 in v2[a][k2],
// k1 = g + G a) instead of going back to A, and there is no closing block
// barrier. (Loading the input the same way, straight from global memory with
// G-strided 8-byte elements, was slower than the staged coalesced loads.)
template <class RG, bool INV, bool TO_REGS = false>
__device__ __forceinline__ void row_fft(float2* A, const float2* tw, int g, float2 (&v1)[RG::A1][RG::N1],
                                        float2 (&v2)[RG::A2][RG::N2]) {
    constexpr int N1 = RG::N1, N2 = RG::N2, G = RG::G;
    float2* S = A;
#pragma unroll
    for (int a = 0; a < RG::A1; ++a) {
        const int n2 = g + G * a;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v1[a][n1] = A[N2 * n1 + n2];
    }
    __syncwarp();  // the row is in registers before S overwrites it
#pragma unroll
    for (int a = 0; a < RG::A1; ++a) {
        const int n2 = g + G * a;
        dft_reg<N1, INV, N2>(v1[a], tw);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            float2 v = v1[a][k1];
            if (k1 > 0) {
                float2 w = tw[n2 * k1];
                if (INV) w.y = -w.y;
                v = cmul(v, w);
            }
            S[k1 * (N2 + 1) + n2] = v;
        }
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < RG::A2; ++a) {
        const int k1 = g + G * a;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) v2[a][n2] = S[k1 * (N2 + 1) + n2];
    }
    if (!TO_REGS) __syncwarp();  // S read before the result overwrites it
#pragma unroll
    for (int a = 0; a < RG::A2; ++a) {
        const int k1 = g + G * a;
        dft_reg<N2, INV, N1>(v2[a], tw);
        if (!TO_REGS)
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) A[k1 + N1 * k2] = v2[a][k2];
    }
    if (!TO_REGS) __syncthreads();
}

template <class RG>
__global__ void __launch_bounds__(ZReg<RG>::T) k_z_r2c_reg(const float* __restrict__ in, float2* __restrict__ out,
                                                             int64_t nrows, const float2* __restrict__ twM,
                                                             const float2* __restrict__ twN) {
    using Z = ZReg<RG>;
    constexpr int M = Z::M, N = 2 * M, P = M + 1;
    extern __shared__ float2 sm[];
    float2* s_twM = sm;
    float2* s_twN = s_twM + M;
    float2* A = s_twN + N;                    // [R][PITCH]
    const int tid = threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.x * Z::R;
    const int rows = (int)min((int64_t)Z::R, nrows - row0);
    for (int t = tid; t < M; t += Z::T) s_twM[t] = twM[t];
    for (int t = tid; t < N; t += Z::T) s_twN[t] = twN[t];
    const float2* src = reinterpret_cast<const float2*>(in + row0 * N);
    {
        // every load of the thread in flight before the first shared-memory store
        constexpr int LD = (Z::R * M + Z::T - 1) / Z::T;
        float2 v[LD];
#pragma unroll
        for (int q = 0; q < LD; ++q) {
            const int t = tid + q * Z::T, r = t / M;
            v[q] = (t < Z::R * M && r < rows) ? src[t] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < LD; ++q) {
            const int t = tid + q * Z::T, r = t / M, m = t - r * M;
            if (t < Z::R * M) A[r * Z::PITCH + m] = v[q];
        }
    }
    __syncthreads();
    {
        const int r = tid / Z::G, g = tid - r * Z::G;
        float2 v1[RG::A1][RG::N1], v2[RG::A2][RG::N2];
        row_fft<RG, false>(A + r * Z::PITCH, s_twM, g, v1, v2);
    }
    // X_k = E_k + exp(-2 pi i k / N) O_k from Z_k and conj(Z_(M-k)); one thread per
    // pair (k, M - k), which both come from the same two values (k = 0 also gives X_M)
    auto split = [&](float2 zk, float2 zc, int kk) {
        zc.y = -zc.y;
        const float2 e = cscale(cadd(zk, zc), 0.5f);
        const float2 dd = csub(zk, zc);
        const float2 o = make_float2(0.5f * dd.y, -0.5f * dd.x);  // -i/2 (zk - zc)
        return cadd(e, cmul(s_twN[kk], o));
    };
    for (int t = tid; t < Z::R * (M / 2 + 1); t += Z::T) {
        const int rr = t / (M / 2 + 1), k = t - rr * (M / 2 + 1);
        if (rr >= rows) continue;
        const float2* Zr = A + rr * Z::PITCH;
        const float2 za = Zr[k], zb = Zr[k == 0 ? 0 : M - k];  // Z_k, Z_(M-k)
        float2* orow = out + (row0 + rr) * P;
        orow[k] = split(za, zb, k);
        if (k == 0)
            orow[M] = split(za, za, M);
        else if (M - k != k)
            orow[M - k] = split(zb, za, M - k);
    }
}

template <class RG>
__global__ void __launch_bounds__(ZReg<RG>::T) k_z_c2r_reg(const float2* __restrict__ in, float* __restrict__ out,
                                                             int64_t nrows, float scale, const float2* __restrict__ twM,
                                                             const float2* __restrict__ twN) {
    using Z = ZReg<RG>;
    constexpr int M = Z::M, N = 2 * M, P = M + 1;
    extern __shared__ float2 sm[];
    float2* s_twM = sm;
    float2* s_twN = s_twM + M;
    float2* A = s_twN + N;                    // [R][PITCH]: the P inputs, then z
    const int tid = threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.x * Z::R;
    const int rows = (int)min((int64_t)Z::R, nrows - row0);
    for (int t = tid; t < M; t += Z::T) s_twM[t] = twM[t];
    for (int t = tid; t < N; t += Z::T) s_twN[t] = twN[t];
    const float2* src = in + row0 * P;
    {
        constexpr int LD = (Z::R * P + Z::T - 1) / Z::T;
        float2 v[LD];
#pragma unroll
        for (int q = 0; q < LD; ++q) {
            const int t = tid + q * Z::T, r = t / P;
            v[q] = (t < Z::R * P && r < rows) ? src[t] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < LD; ++q) {
            const int t = tid + q * Z::T, r = t / P, k = t - r * P;
            if (t < Z::R * P) A[r * Z::PITCH + k] = v[q];
        }
    }
    __syncthreads();
    // z_k = E_k + i O_k with E, O from X_k and conj(X_(M-k)); the pairs (k, M-k)
    // are updated by one thread so the row can be rewritten in place
    for (int t = tid; t < Z::R * (M / 2 + 1); t += Z::T) {
        const int rr = t / (M / 2 + 1), k = t - rr * (M / 2 + 1);
        float2* Xr = A + rr * Z::PITCH;
        const int kc = M - k;
        float2 xk = Xr[k], xc = Xr[kc];
        if (k == 0) {  // X_0 and X_M: imaginary parts carry nothing for a real signal
            xk.y = 0.f;
            xc.y = 0.f;
        }
        float2 zk, zc;
        {
            float2 c = xc;
            c.y = -c.y;
            float2 e = cscale(cadd(xk, c), 0.5f);
            float2 w = s_twN[k];
            w.y = -w.y;  // exp(+2 pi i k / N)
            float2 o = cmul(cscale(csub(xk, c), 0.5f), w);
            zk = make_float2(e.x - o.y, e.y + o.x);  // e + i o
        }
        if (kc != k && kc < M) {
            float2 c = xk;
            c.y = -c.y;
            float2 e = cscale(cadd(xc, c), 0.5f);
            float2 w = s_twN[kc];
            w.y = -w.y;
            float2 o = cmul(cscale(csub(xc, c), 0.5f), w);
            zc = make_float2(e.x - o.y, e.y + o.x);
            Xr[kc] = zc;
        }
        Xr[k] = zk;
    }
    __syncthreads();
    const int r = tid / Z::G, g = tid - r * Z::G;
    float2 v1[RG::A1][RG::N1], v2[RG::A2][RG::N2];
    row_fft<RG, true, true>(A + r * Z::PITCH, s_twM, g, v1, v2);
    // the row from the four-step's registers straight to global memory
    if (r < rows) {
        float2* drow = reinterpret_cast<float2*>(out + (row0 + r) * N);
        const float sc = scale * 2.0f / (float)N;
#pragma unroll
        for (int a = 0; a < RG::A2; ++a)
#pragma unroll
            for (int k2 = 0; k2 < RG::N2; ++k2) drow[g + Z::G * a + RG::N1 * k2] = cscale(v2[a][k2], sc);
    }
}

// Row transform shapes: N -> M = N/2 = N1 N2.
template <class F>
bool with_zreg(int N, F f) {
    switch (N) {
        case 64: f(Reg<8, 4>{}); return true;
        case 128: f(Reg<8, 8>{}); return true;
        case 192: f(Reg<8, 12>{}); return true;
        case 256: f(Reg<16, 8>{}); return true;
        case 384: f(Reg<8, 24>{}); return true;
        case 512: f(Reg<16, 16>{}); return true;
        default: return false;
    }
}

size_t smem_z(int N, bool c2r) {
    int M = N / 2, ld = M + 1;
    return sizeof(float2) * (size_t)(M + N + (c2r ? 3 : 2) * kRows * ld);
}
size_t smem_col(int N, int nbuf) { return sizeof(float2) * (size_t)(N + nbuf * N * kCols); }

ColGeom geom_y(const pmr_ctx* c) { return ColGeom{c->N, c->P, (int64_t)c->P, (int64_t)c->N * c->P}; }
ColGeom geom_x(const pmr_ctx* c) { return ColGeom{c->N, c->P, (int64_t)c->N * c->P, (int64_t)c->P}; }

int launch_z_r2c(pmr_ctx* c, const float* in, float2* out) {
    int64_t nrows = (int64_t)c->N * c->N;
    bool done = with_zreg(c->N, [&](auto rg) {
        using Z = ZReg<decltype(rg)>;
        k_z_r2c_reg<decltype(rg)><<<nblocks(nrows, Z::R), Z::T, Z::smem(), c->stream>>>(in, out, nrows, c->plan.twM,
                                                                                       c->plan.twN);
    });
    if (!done)
        k_z_r2c<<<nblocks(nrows, kRows), kThreads, smem_z(c->N, false), c->stream>>>(in, out, nrows, c->N, c->plan.rM,
                                                                                    c->plan.twM, c->plan.twN);
    return check_launch(c, "z_r2c");
}

int launch_z_c2r(pmr_ctx* c, const float2* in, float* out) {
    int64_t nrows = (int64_t)c->N * c->N;
    float scale = (float)(1.0 / ((double)c->N * c->N));
    bool done = with_zreg(c->N, [&](auto rg) {
        using Z = ZReg<decltype(rg)>;
        k_z_c2r_reg<decltype(rg)><<<nblocks(nrows, Z::R), Z::T, Z::smem(), c->stream>>>(in, out, nrows, scale,
                                                                                       c->plan.twM, c->plan.twN);
    });
    if (!done)
        k_z_c2r<<<nblocks(nrows, kRows), kThreads, smem_z(c->N, true), c->stream>>>(in, out, nrows, c->N, scale,
                                                                                   c->plan.rM, c->plan.twM, c->plan.twN);
    return check_launch(c, "z_c2r");
}

int launch_col(pmr_ctx* c, const float2* in, float2* out, ColGeom g, bool inv) {
    bool done = with_reg(c->N, [&](auto rg) {
        using RG = decltype(rg);
        dim3 grid(nblocks(g.ncols, kRC), c->N);
        if (inv) k_col_reg<RG, true><<<grid, RG::T, RG::smem_col(), c->stream>>>(in, out, g, c->plan.twN);
        else k_col_reg<RG, false><<<grid, RG::T, RG::smem_col(), c->stream>>>(in, out, g, c->plan.twN);
    });
    if (!done) {
        dim3 grid(nblocks(g.ncols, kCols), c->N);
        if (inv) k_col<true><<<grid, kThreads, smem_col(c->N, 2), c->stream>>>(in, out, g, c->plan.rN, c->plan.twN);
        else k_col<false><<<grid, kThreads, smem_col(c->N, 2), c->stream>>>(in, out, g, c->plan.rN, c->plan.twN);
    }
    return check_launch(c, "col_pass");
}

int launch_x_fused(pmr_ctx* c, const XFused& p_in) {
    XFused p = p_in;
    const int width3 = p.nin > 1 ? p.nin : p.nout;
    p.odd3 = width3 == 3;
    for (int o = 0; o < 3 && p.odd3; ++o)
        p.odd3 = p.mul[o].type == MUL_ODD && p.mul[o].j == o && p.mul[o].scale == p.mul[0].scale &&
                 p.mul[o].weighted == p.mul[0].weighted;
    bool done = with_reg(c->N, [&](auto rg) {
        using RG = decltype(rg);
        dim3 grid(nblocks(c->P, kRC), c->N);
        if (p.nin > 1) k_x_reg<RG, 2><<<grid, RG::T, RG::smem(), c->stream>>>(p, geom_x(c), c->plan.twN);
        else if (p.nout > 1) k_x_reg<RG, 1><<<grid, RG::T, RG::smem(), c->stream>>>(p, geom_x(c), c->plan.twN);
        else k_x_reg<RG, 0><<<grid, RG::T, RG::smem(), c->stream>>>(p, geom_x(c), c->plan.twN);
    });
    if (!done) {
        dim3 grid(nblocks(c->P, kCols), c->N);
        k_x_fused<<<grid, kThreads, smem_col(c->N, 3), c->stream>>>(p, geom_x(c), c->plan.rN, c->plan.twN);
    }
    // distinct names per variant: their algorithmic bytes differ
    static const char* names[2][2][4] = {
        {{"x_mul_1", "x_mul_1", "x_mul_2", "x_mul_3"}, {"x_inv_1", "x_inv_1", "x_inv_2", "x_inv_3"}},
        {{"x_fwd_1", "x_fwd_1", "x_fwd_2", "x_fwd_3"}, {"x_conv_1", "x_conv_1", "x_conv_2", "x_conv_3"}}};
    const int width = p.nin > 1 ? p.nin : p.nout;  // inputs (nin > 1) or outputs
    const char* nm = names[p.fwd ? 1 : 0][p.inv ? 1 : 0][width];
    return check_launch(c, p.nin > 1 ? (p.inv ? "x_conv_in3" : "x_fwd_in3") : nm);
}

XFused make_x(const float2* const* in, int nin, float2* const* out, int nout, const Mul* mul, int nmul, bool fwd,
              bool inv, const pmr_ctx* c) {
    XFused p{};
    for (int i = 0; i < nin; ++i) p.in[i] = in[i];
    for (int i = 0; i < nout; ++i) p.out[i] = out[i];
    for (int i = 0; i < nmul; ++i) p.mul[i] = mul[i];
    p.nin = nin;
    p.nout = nout;
    p.fwd = fwd;
    p.inv = inv;
    p.ptab = c->power_tab;
    return p;
}

}  // namespace

namespace {
// A kernel's dynamic shared-memory limit is process-wide while contexts of
// different mesh sizes may run at once: the limit only ever grows.
int raise_smem_limit(pmr_ctx* c, const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<const void*, size_t> set;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = set[fn];
    if (bytes <= cur) return PMR_OK;
    PMR_TRY(check_cuda(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
                       "smem attr"));
    cur = bytes;
    return PMR_OK;
}
}  // namespace

int fft_init(pmr_ctx* c) {
    const int N = c->N, M = N / 2;
    c->plan.N = N;
    c->plan.M = M;
    c->plan.P = M + 1;
    c->plan.rN = make_radix(N);
    c->plan.rM = make_radix(M);
    std::vector<float2> tN(N), tM(M);
    for (int t = 0; t < N; ++t) {
        double ang = -2.0 * M_PI * t / N;
        tN[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    for (int t = 0; t < M; ++t) {
        double ang = -2.0 * M_PI * t / M;
        tM[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    PMR_TRY(check_cuda(c, cudaMalloc(&c->plan.twN, sizeof(float2) * N), "twiddles"));
    PMR_TRY(check_cuda(c, cudaMalloc(&c->plan.twM, sizeof(float2) * M), "twiddles"));
    PMR_TRY(check_cuda(c, cudaMemcpy(c->plan.twN, tN.data(), sizeof(float2) * N, cudaMemcpyHostToDevice), "twiddles"));
    PMR_TRY(check_cuda(c, cudaMemcpy(c->plan.twM, tM.data(), sizeof(float2) * M, cudaMemcpyHostToDevice), "twiddles"));
    PMR_TRY(raise_smem_limit(c, (const void*)k_x_fused, smem_col(N, 3)));
    PMR_TRY(raise_smem_limit(c, (const void*)k_col<true>, smem_col(N, 2)));
    PMR_TRY(raise_smem_limit(c, (const void*)k_col<false>, smem_col(N, 2)));
    PMR_TRY(raise_smem_limit(c, (const void*)k_z_r2c, smem_z(N, false)));
    PMR_TRY(raise_smem_limit(c, (const void*)k_z_c2r, smem_z(N, true)));
    int rc = PMR_OK;
    with_zreg(N, [&](auto rg) {
        using Z = ZReg<decltype(rg)>;
        for (const void* fn : {(const void*)k_z_r2c_reg<decltype(rg)>, (const void*)k_z_c2r_reg<decltype(rg)>})
            if (rc == PMR_OK) rc = raise_smem_limit(c, fn, Z::smem());
    });
    with_reg(N, [&](auto rg) {
        using RG = decltype(rg);
        for (const void* fn : {(const void*)k_col_reg<RG, true>, (const void*)k_col_reg<RG, false>,
                               (const void*)k_x_reg<RG, 0>, (const void*)k_x_reg<RG, 1>, (const void*)k_x_reg<RG, 2>})
            if (rc == PMR_OK) rc = raise_smem_limit(c, fn, RG::smem());
    });
    PMR_TRY(rc);
    return PMR_OK;
}

void fft_free(pmr_ctx* c) {
    cudaFree(c->plan.twN);
    cudaFree(c->plan.twM);
    c->plan.twN = c->plan.twM = nullptr;
}

int fft_r2c(pmr_ctx* c, const float* in, float2* out) {
    PMR_TRY(launch_z_r2c(c, in, out));
    PMR_TRY(launch_col(c, out, out, geom_y(c), false));
    return launch_col(c, out, out, geom_x(c), false);
}

int fft_c2r(pmr_ctx* c, const float2* in, float* out, float2* work) {
    PMR_TRY(launch_col(c, in, work, geom_x(c), true));
    PMR_TRY(launch_col(c, work, work, geom_y(c), true));
    return launch_z_c2r(c, work, out);
}

int conv_1toN(pmr_ctx* c, const float* in, float* const* out, const Mul* mul, int nout) {
    float2* outs[3] = {c->c3, c->c3 + c->NH, c->c3 + 2 * c->NH};
    PMR_TRY(launch_z_r2c(c, in, c->cA));
    PMR_TRY(launch_col(c, c->cA, c->cA, geom_y(c), false));
    const float2* ins[1] = {c->cA};
    PMR_TRY(launch_x_fused(c, make_x(ins, 1, outs, nout, mul, nout, true, true, c)));
    // last-written output first: more of it is still in L2
    for (int j = nout - 1; j >= 0; --j) {
        PMR_TRY(launch_col(c, outs[j], outs[j], geom_y(c), true));
        PMR_TRY(launch_z_c2r(c, outs[j], out[j]));
    }
    return PMR_OK;
}

int conv_Nto1(pmr_ctx* c, const float* const* in, const Mul* mul, int nin, float* out) {
    float2* ks[3] = {c->c3, c->c3 + c->NH, c->c3 + 2 * c->NH};
    // input 0 last: the fused pass reads it first, so more of it is still in L2
    for (int i = nin - 1; i >= 0; --i) {
        PMR_TRY(launch_z_r2c(c, in[i], ks[i]));
        PMR_TRY(launch_col(c, ks[i], ks[i], geom_y(c), false));
    }
    const float2* ins[3] = {ks[0], ks[1], ks[2]};
    float2* outs[1] = {c->cA};
    PMR_TRY(launch_x_fused(c, make_x(ins, nin, outs, 1, mul, nin, true, true, c)));
    PMR_TRY(launch_col(c, c->cA, c->cA, geom_y(c), true));
    return launch_z_c2r(c, c->cA, out);
}

int k_to_real(pmr_ctx* c, const float2* in, float* const* out, const Mul* mul, int nout) {
    float2* outs[3] = {c->c3, c->c3 + c->NH, c->c3 + 2 * c->NH};
    const float2* ins[1] = {in};
    PMR_TRY(launch_x_fused(c, make_x(ins, 1, outs, nout, mul, nout, false, true, c)));
    for (int j = 0; j < nout; ++j) {
        PMR_TRY(launch_col(c, outs[j], outs[j], geom_y(c), true));
        PMR_TRY(launch_z_c2r(c, outs[j], out[j]));
    }
    return PMR_OK;
}

int real_to_k(pmr_ctx* c, const float* const* in, const Mul* mul, int nin, float2* out) {
    float2* ks[3] = {c->c3, c->c3 + c->NH, c->c3 + 2 * c->NH};
    for (int i = 0; i < nin; ++i) {
        PMR_TRY(launch_z_r2c(c, in[i], ks[i]));
        PMR_TRY(launch_col(c, ks[i], ks[i], geom_y(c), false));
    }
    const float2* ins[3] = {ks[0], ks[1], ks[2]};
    float2* outs[1] = {out};
    return launch_x_fused(c, make_x(ins, nin, outs, 1, mul, nin, true, false, c));
}

int real_to_k_add(pmr_ctx* c, const float* const* in, const Mul* mul, int nin, float2* out) {
    float2* ks[3] = {c->c3, c->c3 + c->NH, c->c3 + 2 * c->NH};
    for (int i = 0; i < nin; ++i) {
        PMR_TRY(launch_z_r2c(c, in[i], ks[i]));
        PMR_TRY(launch_col(c, ks[i], ks[i], geom_y(c), false));
    }
    const float2* ins[3] = {ks[0], ks[1], ks[2]};
    float2* outs[1] = {out};
    XFused p = make_x(ins, nin, outs, 1, mul, nin, true, false, c);
    p.acc = 1;
    return launch_x_fused(c, p);
}

}  // namespace pmr

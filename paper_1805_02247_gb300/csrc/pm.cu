// Particle-mesh kernels: cell keys and a deterministic counting sort, CIC
// paint as a cell-sorted segmented gather (no float atomics, fixed summation
// order), CIC readout and its position gradient, the fused readout + kick +
// drift step, Zel'dovich initial conditions, and the adjoints (Sec. 3 forward
// model; Sec. 5.2 gradients written by hand).
//
// Particles carry a float32 displacement from their Lagrangian lattice point q
// (x = q + disp), so the cell index q + floor(disp) and the CIC fraction
// disp - floor(disp) keep full float32 precision at any mesh size. The
// explicit-position form (absolute x, wrapped by fmod) serves the
// single-step entry points.
#include "common.cuh"

namespace pmr {
namespace {

constexpr int kT = 256;

struct Cell {
    int i[3];    // cell of the lower corner, in [0, N)
    float d[3];  // fractional offset in [0, 1)
};

// Explicit positions: w = fmod(u, N) (exact), + N if negative, 0 if it rounds to N.
__device__ __forceinline__ float wrap_pos(float u, float n) {
    float w = fmodf(u, n);
    if (w < 0.f) w += n;
    if (w >= n) w = 0.f;
    return w;
}

// lattice point of particle i = (ix N + iy) N + iz (N^3 < 2^31)
__device__ __forceinline__ void lattice_of(uint32_t i, const FastDiv& fN, int q[3]) {
    const uint32_t t = fN.div(i);
    q[2] = (int)(i - t * fN.d);
    q[0] = (int)fN.div(t);
    q[1] = (int)(t - (uint32_t)q[0] * fN.d);
}

__device__ __forceinline__ Cell cell_of(const float* __restrict__ pos, int64_t np, int64_t i, bool lattice, int N,
                                        const FastDiv& fN) {
    Cell c;
    if (lattice) {
        int q[3];
        lattice_of((uint32_t)i, fN, q);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float u = pos[a * np + i];
            float f = floorf(u);
            c.d[a] = u - f;
            int ii = (q[a] + (int)f) % N;
            c.i[a] = ii < 0 ? ii + N : ii;
        }
    } else {
        const float n = (float)N;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float w = wrap_pos(pos[a * np + i], n);
            float f = floorf(w);
            c.i[a] = (int)f;
            c.d[a] = w - f;
        }
    }
    return c;
}

__device__ __forceinline__ uint32_t key_of(const Cell& c, int N) {
    return ((uint32_t)c.i[0] * N + c.i[1]) * N + c.i[2];
}

__device__ __forceinline__ int64_t corner(const Cell& c, int o, int N) {
    int x = c.i[0] + ((o >> 2) & 1), y = c.i[1] + ((o >> 1) & 1), z = c.i[2] + (o & 1);
    if (x == N) x = 0;
    if (y == N) y = 0;
    if (z == N) z = 0;
    return ((int64_t)x * N + y) * N + z;
}

__device__ __forceinline__ float wgt(const Cell& c, int o) {
    float wx = ((o >> 2) & 1) ? c.d[0] : 1.f - c.d[0];
    float wy = ((o >> 1) & 1) ? c.d[1] : 1.f - c.d[1];
    float wz = (o & 1) ? c.d[2] : 1.f - c.d[2];
    return wx * wy * wz;
}

// d/dx_a of the corner weight
__device__ __forceinline__ void dwgt(const Cell& c, int o, float g[3]) {
    float w[3], s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int bit = (o >> (2 - a)) & 1;
        w[a] = bit ? c.d[a] : 1.f - c.d[a];
        s[a] = bit ? 1.f : -1.f;
    }
    g[0] = s[0] * w[1] * w[2];
    g[1] = w[0] * s[1] * w[2];
    g[2] = w[0] * w[1] * s[2];
}

// ----------------------------------------------------------------------------- sort

__global__ void k_keys(const float* __restrict__ pos, int64_t np, bool lattice, int N, FastDiv fN, uint32_t* __restrict__ keys,
                       uint32_t* __restrict__ counts, uint32_t* __restrict__ rank) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    uint32_t k = key_of(cell_of(pos, np, i, lattice, N, fN), N);
    keys[i] = k;
    // the particle's slot in its cell (arbitrary among the cell's particles;
    // k_seg_fix restores ascending particle index)
    rank[i] = atomicAdd(&counts[k], 1u);
}

// Exclusive scan of the cell counts, reduce-then-scan: k_scan_reduce sums each
// block's kScanBlock counts, k_scan_part scans the block sums (one block),
// k_scan_apply scans each block from its offset.
constexpr int kScanT = 256, kScanPerT = 16, kScanBlock = kScanT * kScanPerT;

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

__global__ void __launch_bounds__(kScanT) k_scan_reduce(const uint32_t* __restrict__ in, int64_t n,
                                                        uint32_t* __restrict__ part) {
    __shared__ uint32_t wsum[kScanT / 32];
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPerT; ++k) {
        const int64_t i = b0 + k * kScanT + threadIdx.x;
        if (i < n) s += in[i];
    }
    s = warp_sum_u32(s);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = threadIdx.x < kScanT / 32 ? wsum[threadIdx.x] : 0u;
        t = warp_sum_u32(t);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// Phase 2: exclusive scan of the block totals by one block (serial chunks).
constexpr int kScanPartT = 1024;
__global__ void __launch_bounds__(kScanPartT) k_scan_part(uint32_t* __restrict__ part, int nb,
                                                         uint32_t* __restrict__ total_out) {
    __shared__ uint32_t carry;
    __shared__ uint32_t wsum[kScanPartT / 32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b0 = 0; b0 < nb; b0 += kScanPartT) {
        int idx = b0 + threadIdx.x;
        uint32_t v = idx < nb ? part[idx] : 0u, inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += t;
        }
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            uint32_t t = (lane < kScanPartT / 32) ? wsum[lane] : 0u, ti = t;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                uint32_t u = __shfl_up_sync(0xffffffffu, ti, d);
                if (lane >= d) ti += u;
            }
            if (lane < kScanPartT / 32) wsum[lane] = ti - t;
        }
        __syncthreads();
        uint32_t ex = carry + wsum[wid] + inc - v;
        if (idx < nb) part[idx] = ex;
        __syncthreads();
        if (threadIdx.x == kScanPartT - 1) carry = ex + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

// shared-memory index with one padding word per 32, so a thread's run of
// kScanPerT consecutive elements and a warp's run of 32 are both conflict-free
__device__ __forceinline__ int scan_sidx(int e) { return e + (e >> 5); }

__global__ void __launch_bounds__(kScanT) k_scan_apply(const uint32_t* __restrict__ in, int64_t n,
                                                       const uint32_t* __restrict__ part, uint32_t* __restrict__ out) {
    __shared__ uint32_t tile[kScanBlock + kScanBlock / 32];
    __shared__ uint32_t wtot[kScanT / 32];
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k < kScanPerT; ++k) {
        const int e = k * kScanT + tid;
        tile[scan_sidx(e)] = b0 + e < n ? in[b0 + e] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanPerT], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPerT; ++k) {
        v[k] = tile[scan_sidx(tid * kScanPerT + k)];
        s += v[k];
    }
    uint32_t inc = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += t;
    }
    if (lane == 31) wtot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < kScanT / 32 ? wtot[lane] : 0u, ti = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, ti, d);
            if (lane >= d) ti += u;
        }
        if (lane < kScanT / 32) wtot[lane] = ti - t;
    }
    __syncthreads();
    uint32_t run = part[blockIdx.x] + wtot[wid] + inc - s;
#pragma unroll
    for (int k = 0; k < kScanPerT; ++k) {
        tile[scan_sidx(tid * kScanPerT + k)] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanPerT; ++k) {
        const int e = k * kScanT + tid;
        if (b0 + e < n) out[b0 + e] = tile[scan_sidx(e)];
    }
}

__global__ void k_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ rank, int64_t np,
                          const uint32_t* __restrict__ start, uint32_t* __restrict__ perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    perm[start[keys[i]] + rank[i]] = (uint32_t)i;
}

// out[m][j] = in[m][perm[j]]: per-particle values into the order of a sort
__global__ void k_permute3(const uint32_t* __restrict__ perm, const float* __restrict__ in, int64_t np,
                           float* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const int64_t i = perm[j];
    out[j] = in[i];
    out[np + j] = in[np + i];
    out[2 * np + j] = in[2 * np + i];
}

// Ascending particle index inside every cell segment (the scatter leaves it
// arbitrary), then, with sfrac, every particle's fractional CIC offsets in the
// sorted order: sfrac[a][j] of particle perm[j] (the float32 values cell_of
// gives). A block owns kFixCells consecutive cells, whose particles are one
// contiguous run of perm: the run is staged in shared memory, segments of up to
// kSegThread particles are insertion-sorted by one thread each, up to
// kSegWarp by one warp (warp_seg_sort in registers up to 32, seg_sort<true>
// in shared memory beyond), longer ones (crowded cells of a clustered field)
// by the whole block with seg_sort<false>, and
// the run is written back with coalesced stores. A run longer than kFixCap is
// listed in ovf for k_seg_fix_big, which does the same in global memory.
constexpr int kFixCells = 512, kFixT = 256, kFixCap = 5120, kSegThread = 8, kSegWarp = 512;

// Sorts a[0, len) ascending with every thread of the block, or with the 32
// lanes of the calling warp when WARP (a bitonic network over the next power of
// two P >= len, in the form whose every compare-exchange puts the smaller value
// at the lower index: the first step of each merge pairs mirrored positions.
// Positions >= len act as +infinity and are never touched.) All threads of the
// block (of the warp) must call it; it ends with a block (warp) barrier.
template <bool WARP>
__device__ void seg_sort(uint32_t* a, int len) {
    int P = 1;
    while (P < len) P <<= 1;
    const int t0 = WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
    const int dt = WARP ? 32 : (int)blockDim.x;
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = t0; t < (P >> 1); t += dt) {
                int lo, hi;
                if (j == (k >> 1)) {  // mirrored pairs within blocks of k
                    const int blk = t / j, o = t - blk * j;
                    lo = blk * k + o;
                    hi = blk * k + k - 1 - o;
                } else {  // half-cleaner at distance j
                    lo = (t / j) * 2 * j + (t % j);
                    hi = lo + j;
                }
                if (hi < len) {
                    const uint32_t x = a[lo], y = a[hi];
                    if (x > y) {
                        a[lo] = y;
                        a[hi] = x;
                    }
                }
            }
            if (WARP)
                __syncwarp();
            else
                __syncthreads();
        }
    }
}

__device__ __forceinline__ void write_sorted(uint32_t i, int64_t j, const float* __restrict__ pos, int64_t np,
                                             bool lattice, int N, const FastDiv& fN, uint32_t* __restrict__ perm,
                                             float* __restrict__ sfrac) {
    perm[j] = i;
    if (sfrac) {
        const Cell cl = cell_of(pos, np, i, lattice, N, fN);
        sfrac[j] = cl.d[0];
        sfrac[np + j] = cl.d[1];
        sfrac[2 * np + j] = cl.d[2];
    }
}

// Sorts a[0, len), len <= 32, ascending with the 32 lanes of a warp: a bitonic
// network on one value per lane (UINT_MAX padding) through shuffles.
__device__ __forceinline__ void warp_seg_sort(uint32_t* a, int len) {
    const int lane = threadIdx.x & 31;
    uint32_t v = lane < len ? a[lane] : 0xffffffffu;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool up = (lane & k) == 0, lo = (lane & j) == 0;
            v = (lo == up) ? min(v, o) : max(v, o);
        }
    __syncwarp();
    if (lane < len) a[lane] = v;
}

__global__ void __launch_bounds__(kFixT) k_seg_fix(const uint32_t* __restrict__ start, uint32_t* __restrict__ perm,
                                                   int64_t ncell, const float* __restrict__ pos, int64_t np,
                                                   bool lattice, int N, FastDiv fN, float* __restrict__ sfrac,
                                                   uint32_t* __restrict__ ovf, uint32_t* __restrict__ novf) {
    __shared__ uint32_t buf[kFixCap];
    __shared__ uint32_t sst[kFixCells + 1];
    __shared__ uint32_t longs[kFixCells];
    __shared__ uint32_t meds[kFixCells];
    __shared__ int nlong, nmed;
    const int tid = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * kFixCells;
    const int nc = (int)min((int64_t)kFixCells, ncell - c0);
    for (int t = tid; t <= nc; t += kFixT) sst[t] = start[c0 + t];
    if (tid == 0) nlong = nmed = 0;
    __syncthreads();
    const uint32_t s0 = sst[0];
    const int n = (int)(sst[nc] - s0);
    if (n > kFixCap) {
        if (tid == 0) ovf[atomicAdd(novf, 1u)] = blockIdx.x;
        return;
    }
    for (int j = tid; j < n; j += kFixT) buf[j] = perm[s0 + j];
    __syncthreads();
    for (int cl = tid; cl < nc; cl += kFixT) {
        const int a = (int)(sst[cl] - s0), e = (int)(sst[cl + 1] - s0);
        if (e - a <= 1) continue;
        if (e - a > kSegWarp) {
            longs[atomicAdd(&nlong, 1)] = (uint32_t)cl;
            continue;
        }
        if (e - a > kSegThread) {  // one warp per segment, below
            meds[atomicAdd(&nmed, 1)] = (uint32_t)cl;
            continue;
        }
        for (int p = a + 1; p < e; ++p) {
            const uint32_t v = buf[p];
            int q = p - 1;
            while (q >= a && buf[q] > v) {
                buf[q + 1] = buf[q];
                --q;
            }
            buf[q + 1] = v;
        }
    }
    __syncthreads();
    for (int mi = tid >> 5; mi < nmed; mi += kFixT / 32) {
        const int cl = (int)meds[mi];
        const int a = (int)(sst[cl] - s0), len = (int)(sst[cl + 1] - s0) - a;
        if (len <= 32)
            warp_seg_sort(buf + a, len);
        else
            seg_sort<true>(buf + a, len);
    }
    __syncthreads();
    const int nl = nlong;
    for (int li = 0; li < nl; ++li) {
        const int cl = (int)longs[li];
        const int a = (int)(sst[cl] - s0), e = (int)(sst[cl + 1] - s0);
        seg_sort<false>(buf + a, e - a);
    }
    for (int j = tid; j < n; j += 2 * kFixT) {
        const int j2 = j + kFixT;
        const uint32_t i1 = buf[j], i2 = buf[j2 < n ? j2 : j];
        const Cell c1 = cell_of(pos, np, i1, lattice, N, fN);
        const Cell c2 = cell_of(pos, np, i2, lattice, N, fN);
        perm[s0 + j] = i1;
        if (sfrac) {
            sfrac[s0 + j] = c1.d[0];
            sfrac[np + s0 + j] = c1.d[1];
            sfrac[2 * np + s0 + j] = c1.d[2];
        }
        if (j2 < n) {
            perm[s0 + j2] = i2;
            if (sfrac) {
                sfrac[s0 + j2] = c2.d[0];
                sfrac[np + s0 + j2] = c2.d[1];
                sfrac[2 * np + s0 + j2] = c2.d[2];
            }
        }
    }
}

// The runs k_seg_fix could not stage: the same steps on global memory, one
// block per listed run.
__global__ void __launch_bounds__(kFixT) k_seg_fix_big(const uint32_t* __restrict__ start, uint32_t* __restrict__ perm,
                                                       int64_t ncell, const float* __restrict__ pos, int64_t np,
                                                       bool lattice, int N, FastDiv fN, float* __restrict__ sfrac,
                                                       const uint32_t* __restrict__ ovf,
                                                       const uint32_t* __restrict__ novf) {
    const uint32_t no = *novf;
    const int tid = threadIdx.x;
    for (uint32_t bi = blockIdx.x; bi < no; bi += gridDim.x) {
        const int64_t c0 = (int64_t)ovf[bi] * kFixCells;
        const int nc = (int)min((int64_t)kFixCells, ncell - c0);
        for (int cl = tid; cl < nc; cl += kFixT) {
            const uint32_t a = start[c0 + cl], e = start[c0 + cl + 1];
            if (e - a <= 1 || e - a > (uint32_t)kSegThread) continue;
            for (uint32_t p = a + 1; p < e; ++p) {
                const uint32_t v = perm[p];
                uint32_t q = p;
                while (q > a && perm[q - 1] > v) {
                    perm[q] = perm[q - 1];
                    --q;
                }
                perm[q] = v;
            }
        }
        for (int cl = tid >> 5; cl < nc; cl += kFixT / 32) {
            const uint32_t a = start[c0 + cl], e = start[c0 + cl + 1];
            if (e - a <= (uint32_t)kSegThread || e - a > (uint32_t)kSegWarp) continue;
            if (e - a <= 32u)
                warp_seg_sort(perm + a, (int)(e - a));
            else
                seg_sort<true>(perm + a, (int)(e - a));
        }
        __syncthreads();
        for (int cl = 0; cl < nc; ++cl) {
            const uint32_t a = start[c0 + cl], e = start[c0 + cl + 1];
            if (e - a > (uint32_t)kSegWarp) seg_sort<false>(perm + a, (int)(e - a));
        }
        const uint32_t s0 = start[c0], s1 = start[c0 + nc];
        for (uint32_t j = s0 + tid; j < s1; j += kFixT) write_sorted(perm[j], j, pos, np, lattice, N, fN, perm, sfrac);
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------- paint / readout

// CIC paint as a gather over the cell-sorted particles (Sec. 2: the CIC
// density): rho_m(c) = scale * sum over the 8 corners o of the sums S_o of
// mass_m(j) W_o(x_j) over the sorted particles j of bin c - o, + offset, in a
// fixed order, so the result does not depend on scheduling.
// A block owns X x Y x 32 cells (32 = the warp: lane l is the cell and bin
// z0 + l); its bins are the rows (x, y) of the tile grown by one on the low x
// and y sides. Warp w walks the rows of x = x0 - 1 + w along y, each lane
// summing its bin's 8 corner terms over the bin's particles (the loads of a
// warp fall in one contiguous run of the sorted arrays), and folds in
// registers first z, T_(ox,oy)(z) = S_(ox,oy,0)(z) + S_(ox,oy,1)(z - 1) (the
// bins z0 - 1 of the warp's rows, lane 0's left neighbours, are summed first,
// one row per lane), then y, U_ox(x, y) = T_(ox,0)(x, y) + T_(ox,1)(x, y - 1) (the
// previous row's T_(ox,1) carried in registers), so a row leaves 2 values per
// cell in shared memory. Each cell then adds the 2 rows that hold it:
// rho = U_0(x, y) + U_1(x - 1, y).
// MMODE 0: unit masses; 1: mass[perm[j]]; 2: masses in sorted order, mass[m][j].
template <int NM>
struct WTile {
    static constexpr int X = 8, Y = NM == 1 ? 16 : 8;
    static constexpr int RX = X + 1, RY = Y + 1, NR = RX * RY;
    static constexpr int W = RX;  // warps per block: one per x-row of bins
    // U values [2 (ox)][NM][X][Y][32] (U_0 of bin rows 1..X, U_1 of rows 0..X-1: the
    // ones the x fold reads), then the halo bins' S_(ox,oy,1) [4][NM][NR]
    static constexpr size_t smem = sizeof(float) * (2 * NM * X * Y * 32 + 4 * NM * NR);
};

template <int NM, int MMODE>
__global__ void __launch_bounds__(WTile<NM>::W * 32, NM == 1 ? 4 : 3) k_paint_wtile(const uint32_t* __restrict__ start,
                                                                     const uint32_t* __restrict__ perm,
                                                                     const float* __restrict__ sfrac,
                                                                     const float* __restrict__ mass, int64_t np, int N,
                                                                     float scale, float offset, float* r0, float* r1,
                                                                     float* r2) {
    using WT = WTile<NM>;
    extern __shared__ float Us[];  // [2 (ox)][NM][X][Y][32]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int z0 = blockIdx.x * 32, y0 = blockIdx.y * WT::Y, x0 = blockIdx.z * WT::X;
    const int z = z0 + lane;
    const bool zin = z < N;
    const int zh = z0 == 0 ? N - 1 : z0 - 1;  // the bin left of lane 0
    const float* __restrict__ sf1 = sfrac + np;
    const float* __restrict__ sf2 = sfrac + 2 * np;

    auto row_base = [&](int r) -> int64_t {
        const int bx = r / WT::RY, by = r - bx * WT::RY;
        int gx = x0 - 1 + bx, gy = y0 - 1 + by;
        gx = gx < 0 ? gx + N : (gx >= N ? gx - N : gx);
        gy = gy < 0 ? gy + N : (gy >= N ? gy - N : gy);
        return ((int64_t)gx * N + gy) * N;
    };
    // particle j's fractional offsets and masses
    auto load = [&](uint32_t j, float& dx, float& dy, float& dz, float (&mv)[NM]) {
        dx = sfrac[j];
        dy = sf1[j];
        dz = sf2[j];
#pragma unroll
        for (int m = 0; m < NM; ++m) mv[m] = 1.f;
        if (MMODE == 1) mv[0] = mass[perm[j]];
        if (MMODE == 2)
#pragma unroll
            for (int m = 0; m < NM; ++m) mv[m] = mass[m * np + j];
    };
    // one particle's corner terms (oz = 1 only when ONLY1)
    auto acc_v = [&](float dx, float dy, float dz, const float (&mv)[NM], float (&S)[2][2][2][NM], bool only1) {
        const float ux = 1.f - dx, uy = 1.f - dy, uz = 1.f - dz;
        const float a[2][2] = {{ux * uy, ux * dy}, {dx * uy, dx * dy}};
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const float wz0 = MMODE ? uz * mv[m] : uz, wz1 = MMODE ? dz * mv[m] : dz;
#pragma unroll
            for (int ox = 0; ox < 2; ++ox)
#pragma unroll
                for (int oy = 0; oy < 2; ++oy) {
                    if (!only1) S[ox][oy][0][m] = fmaf(a[ox][oy], wz0, S[ox][oy][0][m]);
                    S[ox][oy][1][m] = fmaf(a[ox][oy], wz1, S[ox][oy][1][m]);
                }
        }
    };
    auto acc = [&](uint32_t j, float (&S)[2][2][2][NM], bool only1) {
        float dx, dy, dz, mv[NM];
        load(j, dx, dy, dz, mv);
        acc_v(dx, dy, dz, mv, S, only1);
    };

    // warp w walks the bins of x-row w along y; the next row's bin bounds are
    // loaded before this row's particles
    const int bx = w;
    // the warp's rows (x0 - 1 + bx, y0 - 1 + by): the x part of the base is fixed,
    // y advances by one per row (periodic)
    int gxw = x0 - 1 + bx;
    gxw = gxw < 0 ? gxw + N : (gxw >= N ? gxw - N : gxw);
    const int64_t xbase = (int64_t)gxw * N * N + z;
    int gy_n = y0 - 1 < 0 ? y0 - 1 + N : y0 - 1;
    uint32_t s_n = 0, e_n = 0;
    if (zin) {
        const int64_t rb = xbase + (int64_t)gy_n * N;
        s_n = start[rb];
        e_n = start[rb + 1];
    }
    // first the halo bin z0 - 1 of each of the warp's rows (lane 0's left
    // neighbour there), one row per lane; only this warp reads them
    float* Hs = Us + 2 * NM * WT::X * WT::Y * 32;  // [4 (ox,oy)][NM][NR]
    static_assert(WTile<NM>::RY <= 32, "one halo row per lane");
    if (lane < WT::RY) {
        const int r = bx * WT::RY + lane;
        const int64_t rb = row_base(r);
        float H[2][2][2][NM] = {};
        const uint32_t hs = start[rb + zh], he = start[rb + zh + 1];
#pragma unroll 1
        for (uint32_t j = hs; j < he; ++j) acc(j, H, true);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int m = 0; m < NM; ++m) Hs[(q * NM + m) * WT::NR + r] = H[q >> 1][q & 1][1][m];
    }
    __syncwarp();
    float C[2][NM];   // T_(ox,1) of the previous row
    for (int by = 0; by < WT::RY; ++by) {
        const int r = bx * WT::RY + by;
        const uint32_t s = s_n, e = e_n;
        gy_n = gy_n + 1 == N ? 0 : gy_n + 1;
        if (by + 1 < WT::RY && zin) {
            const int64_t rb = xbase + (int64_t)gy_n * N;
            s_n = start[rb];
            e_n = start[rb + 1];
        }
        float S[2][2][2][NM] = {};
        // bins hold about one particle: no unrolled body to skip past
#pragma unroll 1
        for (uint32_t j = s; j < e; ++j) acc(j, S, false);
#pragma unroll
        for (int ox = 0; ox < 2; ++ox)
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                float T[2];
#pragma unroll
                for (int oy = 0; oy < 2; ++oy) {
                    float left = __shfl_up_sync(0xffffffffu, S[ox][oy][1][m], 1);
                    if (lane == 0) left = Hs[((ox * 2 + oy) * NM + m) * WT::NR + r];
                    T[oy] = S[ox][oy][0][m] + left;
                }
                const int ux = bx - 1 + ox;  // U_0 of row bx at slot bx - 1, U_1 at slot bx
                if (by > 0 && ux >= 0 && ux < WT::X)
                    Us[(((ox * NM + m) * WT::X + ux) * WT::Y + by - 1) * 32 + lane] = T[0] + C[ox][m];
                C[ox][m] = T[1];
            }
    }
    __syncthreads();
    for (int q = w; q < WT::X * WT::Y; q += WT::W) {
        const int lx = q / WT::Y, ly = q - lx * WT::Y;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= N || gy >= N || !zin) continue;
        const int64_t c = ((int64_t)gx * N + gy) * N + z;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const float u0 = Us[(((0 * NM + m) * WT::X + lx) * WT::Y + ly) * 32 + lane];
            const float u1 = Us[(((1 * NM + m) * WT::X + lx) * WT::Y + ly) * 32 + lane];
            float* out = m == 0 ? r0 : (m == 1 ? r1 : r2);
            out[c] = (u0 + u1) * scale + offset;
        }
    }
}

__global__ void k_readout(const float* __restrict__ f, const float* __restrict__ pos, int64_t np, bool lattice, int N, FastDiv fN,
                          float* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    Cell cl = cell_of(pos, np, i, lattice, N, fN);
    float acc = 0.f;
#pragma unroll
    for (int o = 0; o < 8; ++o) acc += wgt(cl, o) * f[corner(cl, o, N)];
    out[i] = acc;
}

__global__ void k_readout_grad(const float* __restrict__ f, const float* __restrict__ pos, int64_t np, bool lattice,
                               int N, FastDiv fN, float scale, bool accumulate, float* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    Cell cl = cell_of(pos, np, i, lattice, N, fN);
    float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        float dw[3];
        dwgt(cl, o, dw);
        const float v = f[corner(cl, o, N)];
        g[0] += dw[0] * v;
        g[1] += dw[1] * v;
        g[2] += dw[2] * v;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float r = scale * g[a];
        out[a * np + i] = accumulate ? out[a * np + i] + r : r;
    }
}

// ----------------------------------------------------------------------------- stepping

// Forward step: p += kick * R(x) (force read out at x), disp' = disp + drift * p.
// Each thread takes KP particles, blockDim apart, with every load of all of
// them issued before their arithmetic (more memory requests in flight).
constexpr int KP = 2;
__global__ void k_kick_drift(const float* __restrict__ F, const float* __restrict__ din, float* __restrict__ dout,
                             float* __restrict__ mom, int64_t np, int N, FastDiv fN, float kick, float drift) {
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * KP + threadIdx.x;
    Cell cl[KP];
    float r[KP][3], p[KP][3], d[KP][3];
#pragma unroll
    for (int u = 0; u < KP; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        if (i < np) {
            cl[u] = cell_of(din, np, i, true, N, fN);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                p[u][a] = mom[a * np + i];
                d[u][a] = din[a * np + i];
            }
        }
    }
#pragma unroll
    for (int u = 0; u < KP; ++u) {
        r[u][0] = r[u][1] = r[u][2] = 0.f;
        if (i0 + (int64_t)u * blockDim.x < np) {
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int64_t idx = corner(cl[u], o, N);
                const float w = wgt(cl[u], o);
                r[u][0] += w * F[idx];
                r[u][1] += w * F[np + idx];
                r[u][2] += w * F[2 * np + idx];
            }
        }
    }
#pragma unroll
    for (int u = 0; u < KP; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        if (i >= np) continue;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float pa = p[u][a] + kick * r[u][a];
            mom[a * np + i] = pa;
            dout[a * np + i] = d[u][a] + drift * pa;
        }
    }
}

// Two adjoint updates in one pass over the particles: the end of step s
// (the readout gradient of G at x_s added to lam_x) and the start of step
// s - 1, the adjoint of its drift then the direct (weight-gradient) part of
// its kick: lam_p += drift lam_x; lam_x += kick sum_j lam_p_j grad_x R_j(x)
// with R the readout of F = F(x_{s-1}). lam_x is read and written once.
// INIT: the first pass of the adjoint, whose lam_x is the readout gradient of
// the final density's gradient G alone and whose lam_p starts at zero.
template <bool INIT>
__global__ void k_adj_readout_direct(const float* __restrict__ G, const float* __restrict__ disp_s,
                                     const float* __restrict__ F, const float* __restrict__ disp_p,
                                     float* __restrict__ lam_x, float* __restrict__ lam_p, int64_t np, int N,
                                     FastDiv fN, float kick, float drift) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float lx[3], lp[3];
    {
        const Cell cl = cell_of(disp_s, np, i, true, N, fN);
        float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            float dw[3];
            dwgt(cl, o, dw);
            const float v = G[corner(cl, o, N)];
            g[0] += dw[0] * v;
            g[1] += dw[1] * v;
            g[2] += dw[2] * v;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) lx[a] = INIT ? g[a] : lam_x[a * np + i] + g[a];
    }
    const Cell cl = cell_of(disp_p, np, i, true, N, fN);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lp[a] = INIT ? drift * lx[a] : lam_p[a * np + i] + drift * lx[a];
        lam_p[a * np + i] = lp[a];
    }
    float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        float dw[3];
        dwgt(cl, o, dw);
        const int64_t idx = corner(cl, o, N);
        const float v = lp[0] * F[idx] + lp[1] * F[np + idx] + lp[2] * F[2 * np + idx];
        g[0] += dw[0] * v;
        g[1] += dw[1] * v;
        g[2] += dw[2] * v;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) lam_x[a * np + i] = lx[a] + kick * g[a];
}

// disp = D0 psi, p = Gp0 psi (psi already in disp)
__global__ void k_za_finish(float* __restrict__ disp, float* __restrict__ mom, int64_t n, float D0, float Gp0) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float psi = disp[i];
    disp[i] = D0 * psi;
    mom[i] = Gp0 * psi;
}

// lam_psi = D0 lam_x + Gp0 lam_p
__global__ void k_za_adj_combine(const float* __restrict__ lx, const float* __restrict__ lp, float* __restrict__ out,
                                 int64_t n, float D0, float Gp0) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = D0 * lx[i] + Gp0 * lp[i];
}

// ----------------------------------------------------------------------------- second-order LPT

// S = phi_xx phi_yy + phi_xx phi_zz + phi_yy phi_zz - phi_xy^2 - phi_xz^2 - phi_yz^2
__global__ void k_lpt2_source(const float* __restrict__ H, int64_t n, float* __restrict__ S) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float xx = H[i], yy = H[n + i], zz = H[2 * n + i];
    const float xy = H[3 * n + i], xz = H[4 * n + i], yz = H[5 * n + i];
    S[i] = xx * yy + xx * zz + yy * zz - xy * xy - xz * xz - yz * yz;
}

// disp holds psi1 on entry: disp = D1 psi1 + D2 psi2, mom = Gp psi1 + Gp2 psi2
__global__ void k_lpt2_finish(float* __restrict__ disp, const float* __restrict__ psi2, float* __restrict__ mom,
                              int64_t n, float D1, float D2, float Gp, float Gp2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = disp[i], b = psi2[i];
    disp[i] = D1 * a + D2 * b;
    mom[i] = Gp * a + Gp2 * b;
}

// adjoint of the source: dS/dphi_ii = sum of the other two diagonal entries,
// dS/dphi_ij = -2 phi_ij (i < j); G = sigma * dS/dH
__global__ void k_lpt2_hess_grad(const float* __restrict__ sigma, const float* __restrict__ H, int64_t n,
                                 float* __restrict__ G) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float sg = sigma[i];
    const float xx = H[i], yy = H[n + i], zz = H[2 * n + i];
    G[i] = sg * (yy + zz);
    G[n + i] = sg * (xx + zz);
    G[2 * n + i] = sg * (xx + yy);
    G[3 * n + i] = -2.f * sg * H[3 * n + i];
    G[4 * n + i] = -2.f * sg * H[4 * n + i];
    G[5 * n + i] = -2.f * sg * H[5 * n + i];
}

}  // namespace

// ============================================================================= host wrappers

int cell_sort_into(pmr_ctx* c, const float* pos, int64_t np, bool lattice, uint32_t* keys_out, uint32_t* perm,
                   uint32_t* start, float* sfrac) {
    const int N = c->N;
    const int64_t N3 = c->N3;
    const FastDiv fN((uint32_t)N);
    uint32_t* keys = keys_out ? keys_out : c->keys;
    uint32_t* rank = c->sort_tmp;  // slot of each particle in its cell, until the scatter
    PMR_TRY(check_cuda(c, cudaMemsetAsync(c->counts, 0, sizeof(uint32_t) * N3, c->stream), "memset"));
    PMR_TRY(check_cuda(c, cudaMemsetAsync(c->long_count, 0, sizeof(uint32_t), c->stream), "memset"));
    if (np > 0) {
        k_keys<<<nblocks(np, kT), kT, 0, c->stream>>>(pos, np, lattice, N, fN, keys, c->counts, rank);
        PMR_TRY(check_launch(c, "keys"));
    }
    const int nb = (int)((N3 + kScanBlock - 1) / kScanBlock);
    k_scan_reduce<<<nb, kScanT, 0, c->stream>>>(c->counts, N3, c->scan_part);
    PMR_TRY(check_launch(c, "scan_reduce"));
    k_scan_part<<<1, kScanPartT, 0, c->stream>>>(c->scan_part, nb, start + N3);
    PMR_TRY(check_launch(c, "scan_part"));
    k_scan_apply<<<nb, kScanT, 0, c->stream>>>(c->counts, N3, c->scan_part, start);
    PMR_TRY(check_launch(c, "scan_apply"));
    if (np == 0) return PMR_OK;
    k_scatter<<<nblocks(np, kT), kT, 0, c->stream>>>(keys, rank, np, start, perm);
    PMR_TRY(check_launch(c, "scatter"));
    k_seg_fix<<<nblocks(N3, kFixCells), kFixT, 0, c->stream>>>(start, perm, N3, pos, np, lattice, N, fN, sfrac,
                                                               c->long_list, c->long_count);
    PMR_TRY(check_launch(c, "seg_fix"));
    k_seg_fix_big<<<256, kFixT, 0, c->stream>>>(start, perm, N3, pos, np, lattice, N, fN, sfrac, c->long_list,
                                               c->long_count);
    return check_launch(c, "seg_fix_big");
}

int cell_sort(pmr_ctx* c, const float* pos, int64_t np, bool lattice, uint32_t* keys_out) {
    return cell_sort_into(c, pos, np, lattice, keys_out, c->perm, c->cell_start, c->sfrac);
}

template <int NM, int MMODE>
int launch_paint_wtile(pmr_ctx* c, const uint32_t* perm, const uint32_t* start, const float* sfrac, const float* mass,
                       int64_t np, float scale, float offset, float* const* rho) {
    using WT = WTile<NM>;
    // one mass fits the default 48 KB of dynamic shared memory, so the
    // allocation-free paint (which has no context and so no set-up call)
    // needs no attribute; pm_init raises the limit for three masses
    static_assert(WTile<1>::smem <= 48 * 1024, "one-mass paint within the default shared-memory limit");
    const int N = c->N;
    const dim3 grid((N + 31) / 32, (N + WT::Y - 1) / WT::Y, (N + WT::X - 1) / WT::X);
    k_paint_wtile<NM, MMODE><<<grid, WT::W * 32, WT::smem, c->stream>>>(
        start, perm, sfrac, mass, np, N, scale, offset, rho[0], NM > 1 ? rho[1] : nullptr, NM > 2 ? rho[2] : nullptr);
    return check_launch(c, NM == 1 ? "paint" : "paint3");
}

// Every paint reads the fractional offsets its sort wrote (sfrac).
int paint_with(pmr_ctx* c, const float* pos, int64_t np, bool lattice, const uint32_t* perm, const uint32_t* start,
               const float* sfrac, const float* mass, int nmass, float scale, float offset, float* const* rho) {
    (void)pos;
    (void)lattice;
    if (!sfrac || nmass != 1) return fail(c, PMR_EINVAL, "paint: one mass and the sort's offsets are required");
    return mass ? launch_paint_wtile<1, 1>(c, perm, start, sfrac, mass, np, scale, offset, rho)
                : launch_paint_wtile<1, 0>(c, perm, start, sfrac, nullptr, np, scale, offset, rho);
}

// Three-mass paint of the lattice particles with their masses first moved into
// the sort's order, so the paint's bin loop reads offsets and masses as
// independent, coalesced loads. Scratch: c->F (the kept per-step forces live
// in c->F_all).
int paint3_sorted(pmr_ctx* c, const uint32_t* perm, const uint32_t* start, const float* sfrac, const float* mass,
                  float scale, float* const* rho) {
    const int64_t np = c->N3;
    float* smass = c->F;
    k_permute3<<<nblocks(np, kT), kT, 0, c->stream>>>(perm, mass, np, smass);
    PMR_TRY(check_launch(c, "permute3"));
    return launch_paint_wtile<3, 2>(c, perm, start, sfrac, smass, np, scale, 0.0f, rho);
}

int pm_init(pmr_ctx* c) {
    return check_cuda(c,
                      cudaFuncSetAttribute(k_paint_wtile<3, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)WTile<3>::smem),
                      "paint smem attr");
}

int paint(pmr_ctx* c, const float* pos, int64_t np, bool lattice, const float* mass, int nmass, float scale,
          float offset, float* const* rho) {
    return paint_with(c, pos, np, lattice, c->perm, c->cell_start, c->sfrac, mass, nmass, scale, offset, rho);
}

int readout(pmr_ctx* c, const float* field, const float* pos, int64_t np, bool lattice, float* out) {
    k_readout<<<nblocks(np, kT), kT, 0, c->stream>>>(field, pos, np, lattice, c->N, FastDiv((uint32_t)c->N), out);
    return check_launch(c, "readout");
}

int readout_grad(pmr_ctx* c, const float* field, const float* pos, int64_t np, bool lattice, float scale,
                 bool accumulate, float* out) {
    k_readout_grad<<<nblocks(np, kT), kT, 0, c->stream>>>(field, pos, np, lattice, c->N, FastDiv((uint32_t)c->N), scale, accumulate, out);
    return check_launch(c, "readout_grad");
}

int density_from(pmr_ctx* c, const float* disp, float* delta) {
    PMR_TRY(cell_sort(c, disp, c->N3, true, nullptr));
    float* outs[1] = {delta};
    // unit-mass particles, one per cell: rho_bar = 1
    return paint(c, disp, c->N3, true, nullptr, 1, 1.0f, -1.0f, outs);
}

int density_slot(pmr_ctx* c, int s, const float* disp, float* delta, bool sort) {
    uint32_t* perm = c->perm_all + (int64_t)s * c->N3;
    uint32_t* start = c->start_all + (int64_t)s * (c->N3 + 1);
    float* sfrac = c->sfrac_all + (int64_t)s * 3 * c->N3;
    if (sort) PMR_TRY(cell_sort_into(c, disp, c->N3, true, nullptr, perm, start, sfrac));
    float* outs[1] = {delta};
    return paint_with(c, disp, c->N3, true, perm, start, sfrac, nullptr, 1, 1.0f, -1.0f, outs);
}

int za_ics(pmr_ctx* c, const float2* s_k, float* disp, float* mom) {
    Mul mul[3];
    for (int j = 0; j < 3; ++j) mul[j] = Mul{MUL_ODD, j, 1.0f, 0.f, 0};
    float* outs[3] = {disp, disp + c->N3, disp + 2 * c->N3};
    PMR_TRY(k_to_real(c, s_k, outs, mul, 3));
    k_za_finish<<<nblocks(3 * c->N3, kT), kT, 0, c->stream>>>(disp, mom, 3 * c->N3, (float)c->D0, (float)c->Gp0);
    return check_launch(c, "za_finish");
}

namespace {
// phi_ij of the first-order potential (lap phi = delta = irfft(s)) into lpt_H
int lpt2_hessian(pmr_ctx* c, const float2* s_k) {
    static const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int h = 0; h < 2; ++h) {
        Mul mul[3];
        float* outs[3];
        for (int t = 0; t < 3; ++t) {
            const int* pr = pairs[3 * h + t];
            mul[t] = Mul{MUL_HESS, pr[0], 1.0f, 0.f, 0, pr[1]};
            outs[t] = c->lpt_H + (int64_t)(3 * h + t) * c->N3;
        }
        PMR_TRY(k_to_real(c, s_k, outs, mul, 3));
    }
    return PMR_OK;
}
}  // namespace

// Sec. 3 initial conditions of order cfg.lpt_order; the Hessian of the
// first-order potential stays in lpt_H for the adjoint.
int lpt_ics(pmr_ctx* c, const float2* s_k, float* disp, float* mom) {
    if (c->cfg.lpt_order != 2) return za_ics(c, s_k, disp, mom);
    const int64_t N3 = c->N3;
    Mul mul[3];
    for (int j = 0; j < 3; ++j) mul[j] = Mul{MUL_ODD, j, 1.0f, 0.f, 0};
    float* psi1[3] = {disp, disp + N3, disp + 2 * N3};
    PMR_TRY(k_to_real(c, s_k, psi1, mul, 3));
    PMR_TRY(lpt2_hessian(c, s_k));
    k_lpt2_source<<<nblocks(N3, kT), kT, 0, c->stream>>>(c->lpt_H, N3, c->delta);
    PMR_TRY(check_launch(c, "lpt2_source"));
    // psi2 = grad phi2, lap phi2 = S: psi2_k = -i k S_k / k^2
    for (int j = 0; j < 3; ++j) mul[j] = Mul{MUL_ODD, j, -1.0f, 0.f, 0};
    float* psi2[3] = {c->F, c->F + N3, c->F + 2 * N3};
    PMR_TRY(conv_1toN(c, c->delta, psi2, mul, 3));
    k_lpt2_finish<<<nblocks(3 * N3, kT), kT, 0, c->stream>>>(disp, c->F, mom, 3 * N3, (float)c->D0, (float)c->D2_0,
                                                              (float)c->Gp0, (float)c->Gp2_0);
    return check_launch(c, "lpt2_finish");
}

// Adjoint of lpt_ics at s_k (grad overwritten). have_H: lpt_H already holds
// the Hessian of s_k (it does after lpt_ics on the same s_k).
int lpt_adjoint(pmr_ctx* c, const float2* s_k, const float* lam_x, const float* lam_p, float2* grad, bool have_H) {
    PMR_TRY(za_adjoint(c, lam_x, lam_p, grad));
    if (c->cfg.lpt_order != 2) return PMR_OK;
    const int64_t N3 = c->N3;
    if (!have_H) PMR_TRY(lpt2_hessian(c, s_k));
    // mu = D2 lam_x + Gp2 lam_p; sigma = sum_j irfft(conj(-i k_j / k^2) rfft(mu_j))
    k_za_adj_combine<<<nblocks(3 * N3, kT), kT, 0, c->stream>>>(lam_x, lam_p, c->F, 3 * N3, (float)c->D2_0,
                                                                 (float)c->Gp2_0);
    PMR_TRY(check_launch(c, "lpt2_adj_combine"));
    Mul mul[3];
    for (int j = 0; j < 3; ++j) mul[j] = Mul{MUL_ODD, j, 1.0f, 0.f, 0};
    const float* mu[3] = {c->F, c->F + N3, c->F + 2 * N3};
    PMR_TRY(conv_Nto1(c, mu, mul, 3, c->delta));
    k_lpt2_hess_grad<<<nblocks(N3, kT), kT, 0, c->stream>>>(c->delta, c->lpt_H, N3, c->lpt_G);
    PMR_TRY(check_launch(c, "lpt2_hess_grad"));
    // grad += sum_ij (k_i k_j / k^2) (w / N^3) rfft(G_ij)
    static const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    const float inv_n3 = (float)(1.0 / (double)N3);
    for (int h = 0; h < 2; ++h) {
        Mul hm[3];
        const float* gin[3];
        for (int t = 0; t < 3; ++t) {
            const int* pr = pairs[3 * h + t];
            hm[t] = Mul{MUL_HESS, pr[0], inv_n3, 0.f, 1, pr[1]};
            gin[t] = c->lpt_G + (int64_t)(3 * h + t) * N3;
        }
        PMR_TRY(real_to_k_add(c, gin, hm, 3, grad));
    }
    return PMR_OK;
}

int kick_drift(pmr_ctx* c, const float* F, const float* din, float* dout, float* mom, float kick, float drift) {
    k_kick_drift<<<nblocks(c->N3, kT * KP), kT, 0, c->stream>>>(F, din, dout, mom, c->N3, c->N, FastDiv((uint32_t)c->N), kick, drift);
    return check_launch(c, "kick_drift");
}


// grad_s = sum_j conj(i k_j / k^2) (w / N^3) rfft(D0 lam_x_j + Gp0 lam_p_j)
int za_adjoint(pmr_ctx* c, const float* lam_x, const float* lam_p, float2* grad) {
    float* tmp = c->F;  // 3 meshes of scratch
    k_za_adj_combine<<<nblocks(3 * c->N3, kT), kT, 0, c->stream>>>(lam_x, lam_p, tmp, 3 * c->N3, (float)c->D0,
                                                                     (float)c->Gp0);
    PMR_TRY(check_launch(c, "za_adj_combine"));
    Mul mul[3];
    const float inv_n3 = (float)(1.0 / (double)c->N3);
    for (int j = 0; j < 3; ++j) mul[j] = Mul{MUL_ODD, j, -inv_n3, 0.f, 1};
    const float* ins[3] = {tmp, tmp + c->N3, tmp + 2 * c->N3};
    return real_to_k(c, ins, mul, 3, grad);
}

int pm_forward_impl(pmr_ctx* c, const float2* s_k) {
    const int64_t N3 = c->N3;
    c->have_forward = false;  // the stored trajectory is being replaced
    PMR_TRY(lpt_ics(c, s_k, c->disp, c->mom));
    const float om15 = (float)(1.5 * c->cfg.omega_m);
    Mul fm[3];
    for (int j = 0; j < 3; ++j) fm[j] = Mul{MUL_ODD, j, om15, 0.f, 0};
    for (int s = 0; s < c->cfg.nsteps; ++s) {
        const float* din = c->disp + (int64_t)s * 3 * N3;
        float* dout = c->disp + (int64_t)(s + 1) * 3 * N3;
        float* F = c->F_all + (int64_t)s * 3 * N3;  // kept for the adjoint
        float* Fj[3] = {F, F + N3, F + 2 * N3};
        PMR_TRY(density_slot(c, s, din, c->delta, true));
        PMR_TRY(conv_1toN(c, c->delta, Fj, fm, 3));
        PMR_TRY(kick_drift(c, F, din, dout, c->mom, (float)c->kick[s], (float)c->drift[s]));
    }
    c->have_forward = true;
    c->fwd_id++;
    return PMR_OK;
}

// Reverse sweep. On entry lam_x holds dL/dx at the final positions and lam_p = 0.
// gfin: the loss gradient with respect to the final density (N^3); the
// adjoint starts with lam_x = its readout gradient at x_nsteps and lam_p = 0.
int pm_adjoint_impl(pmr_ctx* c, const float* gfin, float2* grad) {
    const int64_t N3 = c->N3;
    const float om15 = (float)(1.5 * c->cfg.omega_m);
    Mul fmT[3];
    for (int j = 0; j < 3; ++j) fmT[j] = Mul{MUL_ODD, j, -om15, 0.f, 0};  // conj of an imaginary multiplier
    float* Gj[3] = {c->gfeat, c->gfeat + N3, c->gfeat + 2 * N3};
    // Step s of the adjoint: direct kick term with the force F(x_s) the forward
    // sweep kept; three-mass paint (on the forward sweep's sort) and its force
    // transpose into G; readout gradient of G at x_s. The readout of step s and
    // the direct term of step s - 1 share one particle pass (as do the final
    // density's readout and the direct term of the last step).
    const int S = c->cfg.nsteps;
    const FastDiv fN((uint32_t)c->N);
    auto force_at = [&](int s) -> const float* { return c->F_all + (int64_t)s * 3 * N3; };
    if (S == 0) {
        PMR_TRY(readout_grad(c, gfin, c->disp, N3, true, 1.0f, false, c->lam_x));
        PMR_TRY(check_cuda(c, cudaMemsetAsync(c->lam_p, 0, sizeof(float) * 3 * N3, c->stream), "memset"));
    } else {
        k_adj_readout_direct<true><<<nblocks(N3, kT), kT, 0, c->stream>>>(
            gfin, c->disp + (int64_t)S * 3 * N3, force_at(S - 1), c->disp + (int64_t)(S - 1) * 3 * N3, c->lam_x,
            c->lam_p, N3, c->N, fN, (float)c->kick[S - 1], (float)c->drift[S - 1]);
        PMR_TRY(check_launch(c, "adj_readout_direct"));
    }
    for (int s = S - 1; s >= 0; --s) {
        const float* d = c->disp + (int64_t)s * 3 * N3;
        PMR_TRY(paint3_sorted(c, c->perm_all + (int64_t)s * N3, c->start_all + (int64_t)s * (N3 + 1),
                              c->sfrac_all + (int64_t)s * 3 * N3, c->lam_p, (float)c->kick[s], Gj));
        const float* gins[3] = {Gj[0], Gj[1], Gj[2]};
        PMR_TRY(conv_Nto1(c, gins, fmT, 3, c->gm));
        if (s == 0) {
            PMR_TRY(readout_grad(c, c->gm, d, N3, true, 1.0f, true, c->lam_x));
            break;
        }
        k_adj_readout_direct<false><<<nblocks(N3, kT), kT, 0, c->stream>>>(
            c->gm, d, force_at(s - 1), c->disp + (int64_t)(s - 1) * 3 * N3, c->lam_x, c->lam_p, N3, c->N, fN,
            (float)c->kick[s - 1], (float)c->drift[s - 1]);
        PMR_TRY(check_launch(c, "adj_readout_direct"));
    }
    return lpt_adjoint(c, nullptr, c->lam_x, c->lam_p, grad, true);  // Hessian kept by pm_forward
}

}  // namespace pmr

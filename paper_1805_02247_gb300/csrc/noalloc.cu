// Deterministic CIC paint for callers that cannot allocate device memory.
//
// pmr_paint() needs a context, and creating one calls cudaMalloc. Some callers
// cannot do that: code running while a CUDA graph is being captured (an
// allocation there is illegal or breaks the capture), plug-ins of frameworks
// that own every device allocation through their own pool and forbid raw
// cudaMalloc, and real-time loops that must not synchronise the device (which
// cudaMalloc/cudaFree may do). pmr_paint_noalloc() gives them the same paint
// with its sorting scratch taken from one fixed array in device memory that
// exists as soon as this library is loaded on a GPU.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int64_t kMaxCells = int64_t(1) << 18;      // 64^3
constexpr int64_t kMaxParticles = int64_t(1) << 18;  // one per cell at 64^3
constexpr size_t kAlign = 256;

constexpr size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// Scratch regions (bytes), each 256-byte aligned.
constexpr size_t kKeys = up(4 * kMaxParticles);
constexpr size_t kPerm = up(4 * kMaxParticles);
constexpr size_t kTmp = up(4 * kMaxParticles);
constexpr size_t kStart = up(4 * (kMaxCells + 1));
constexpr size_t kCounts = up(4 * kMaxCells);
constexpr size_t kLong = up(4 * kMaxCells);
constexpr size_t kPart = up(4 * ((kMaxCells + 1023) / 1024));
constexpr size_t kLongCount = up(16);
constexpr size_t kFrac = up(4 * 3 * kMaxParticles);  // sorted fractional offsets, as pmr_paint uses them
constexpr size_t kScratchBytes = kKeys + kPerm + kTmp + kStart + kCounts + kLong + kPart + kLongCount + kFrac;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_paint_scratch[kScratchBytes];

// The array's name in host code is only a host-side stand-in; its device
// address is looked up once per device with that device current.
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_address(unsigned char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return pmr::fail(nullptr, PMR_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return pmr::fail(nullptr, PMR_EINVAL, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_paint_scratch);
        if (e != cudaSuccess || !p)
            return pmr::fail(nullptr, PMR_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return PMR_OK;
}

}  // namespace

extern "C" int pmr_paint_noalloc(int N, const float* x, int64_t np, const float* mass, float* rho, void* stream) {
    // The paint's tiles wrap their halo rows once, which needs N >= 8 (the
    // smallest mesh pmr_create accepts); the fixed array holds N <= 64.
    if (N < 8 || (int64_t)N * N * N > kMaxCells)
        return pmr::fail(nullptr, PMR_EINVAL, "pmr_paint_noalloc: N must be in [8, 64] (N^3 <= 262144)");
    if (np < 0 || np > (int64_t)N * N * N)
        return pmr::fail(nullptr, PMR_EINVAL, "pmr_paint_noalloc: np must be in [0, N^3]");
    if (!rho || (np > 0 && !x)) return pmr::fail(nullptr, PMR_EINVAL, "pmr_paint_noalloc: NULL argument");
    unsigned char* base = nullptr;
    PMR_TRY(scratch_address(&base));

    // A context on the host stack whose sort buffers point into the fixed
    // array; it owns no device memory and is never destroyed with pmr_destroy.
    pmr_ctx c;
    c.stream = (cudaStream_t)stream;
    c.N = N;
    c.N3 = (int64_t)N * N * N;
    unsigned char* p = base;
    c.keys = reinterpret_cast<uint32_t*>(p); p += kKeys;
    c.perm = reinterpret_cast<uint32_t*>(p); p += kPerm;
    c.sort_tmp = reinterpret_cast<uint32_t*>(p); p += kTmp;
    c.cell_start = reinterpret_cast<uint32_t*>(p); p += kStart;
    c.counts = reinterpret_cast<uint32_t*>(p); p += kCounts;
    c.long_list = reinterpret_cast<uint32_t*>(p); p += kLong;
    c.scan_part = reinterpret_cast<uint32_t*>(p); p += kPart;
    c.long_count = reinterpret_cast<uint32_t*>(p); p += kLongCount;
    c.sfrac = reinterpret_cast<float*>(p);

    // cell_sort clears the histogram and the long-segment counter itself;
    // every other region is fully written before it is read.
    int rc = pmr::cell_sort(&c, x, np, false, nullptr);
    if (rc == PMR_OK) {
        float* outs[1] = {rho};
        rc = pmr::paint(&c, x, np, false, mass, 1, 1.0f, 0.0f, outs);
    }
    if (rc != PMR_OK) return pmr::fail(nullptr, rc, "pmr_paint_noalloc: " + c.err);
    return PMR_OK;
}

// Allocation-free Morton keys + sort: nbody_sort_keys_noalloc.
//
// For callers that cannot call cudaMalloc: runtimes that own a fixed device-memory budget (an
// embedding application with its own pool), real-time loops that must not block in the
// allocator, and plugins whose host application forbids allocation after start-up.  The working
// memory that nbody_build_tree keeps in its context (alternate key and id buffers, digit
// histograms, box partials) lives here in one file-scope device array instead, which every GPU
// that loads the library holds until the process exits.
#include <mutex>

#include "nbody_internal.cuh"

using namespace nb;

namespace {

constexpr int64_t kMaxN = NBODY_NOALLOC_MAX_N;
constexpr size_t kAlign = 256;
constexpr size_t round_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

constexpr int64_t kMaxTiles = (kMaxN + kSortTileKeys - 1) / kSortTileKeys;

// Scratch layout: alternate keys | alternate ids | digit histogram | per-tile digit counts |
// box partials | root box | level tables.
constexpr size_t kOffKeys = 0;
constexpr size_t kOffIds = kOffKeys + round_up(sizeof(uint64_t) * kMaxN);
constexpr size_t kOffHist = kOffIds + round_up(sizeof(uint32_t) * kMaxN);
// the sort of one system clears and fills kSortKeyPasses rows of 256 digit totals
constexpr size_t kOffCounts = kOffHist + round_up(sizeof(uint32_t) * kSortKeyPasses * 256);
constexpr size_t kOffPartials = kOffCounts + round_up(sizeof(uint32_t) * 256 * kMaxTiles);
constexpr size_t kPartialBytes = 64 * 1024;
constexpr size_t kOffBox = kOffPartials + kPartialBytes;
constexpr size_t kOffTab = kOffBox + round_up(sizeof(Box));
constexpr size_t kScratchBytes = kOffTab + round_up(sizeof(LevelTables));
static_assert(kOffCounts - kOffHist >= sizeof(uint32_t) * kSortKeyPasses * 256 &&
                  kOffPartials - kOffCounts >= sizeof(uint32_t) * 256 * kMaxTiles,
              "scratch regions hold what the sort writes");

// The scratch.  In host code this name is only a host-side stand-in for the device array, not a
// device address: kernels receive the address cudaGetSymbolAddress returns for it.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_dev_scratch[kMaxDevices] = {};

// With the caller's device current: the scratch's device address, looked up on every call (the
// lookup enqueues nothing, and a context created after a device reset gets its own address).  The
// first call on a device, and any call that finds a different address there, also sets the sort's
// shared-memory attribute.
nbody_status setup(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NBODY_ECUDA;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return NBODY_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_dev_scratch[dev] != p) {
        if (sort_prepare() != cudaSuccess) return NBODY_ECUDA;
        g_dev_scratch[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_scratch[dev];
    return NBODY_OK;
}

}  // namespace

extern "C" nbody_status nbody_sort_keys_noalloc(const double *d_pos, const double *d_mass,
                                                int64_t n, uint64_t *d_keys_sorted,
                                                uint32_t *d_ids_sorted, void *cuda_stream)
{
    if (n < 0 || n > kMaxN) return NBODY_EINVAL;
    if (n == 0) return NBODY_OK;
    if (!d_pos || !d_mass || !d_keys_sorted || !d_ids_sorted) return NBODY_EINVAL;
    const int nblk = bbox_blocks(n);
    if ((size_t)nblk * bbox_partial_doubles() * sizeof(double) > kPartialBytes) return NBODY_EINVAL;
    if (sort_tiles((int)n) > kMaxTiles) return NBODY_EINVAL;
    unsigned char *base = nullptr;
    const nbody_status st = setup(&base);
    if (st != NBODY_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *partials = reinterpret_cast<double *>(base + kOffPartials);
    Box *box = reinterpret_cast<Box *>(base + kOffBox);
    LevelTables *tab = reinterpret_cast<LevelTables *>(base + kOffTab);
    launch_bbox_partials(d_pos, d_mass, (int)n, partials, nblk, nullptr, s);
    launch_bbox_finalize(partials, nblk, box, tab, 0.0, s);
    launch_keys(d_pos, (int)n, box, Systems{nullptr, nullptr, 1}, d_keys_sorted, d_ids_sorted, s);
    SortScratch sc{reinterpret_cast<uint64_t *>(base + kOffKeys),
                   reinterpret_cast<uint32_t *>(base + kOffIds),
                   reinterpret_cast<uint32_t *>(base + kOffHist),
                   reinterpret_cast<uint32_t *>(base + kOffCounts), (int)kMaxTiles};
    // the sort clears its digit histogram itself; every other scratch word is written before
    // it is read
    launch_radix_sort(d_keys_sorted, d_ids_sorted, (int)n, sc, s);
    // the status covers every launch above and any CUDA error still pending on this thread
    return cudaGetLastError() == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
}

// Re-sort of the bodies from the previous step's sorted order (temporal coherence, §4.4).
//
// Bodies move little in one step, so the previous step's sorted list is almost sorted under the
// new keys; the paper finishes it with an insertion sort.  Here the same result -- the stable
// sort by (system, key, caller's index); one system for a single-system context -- comes from
// data-parallel phases:
//   1. extract: the keys of the bodies taken in the previous order; every position that takes
//      part in a descent (two neighbours in the wrong order) is removed, and removal repeats on
//      what is left until the rest ascends.  Inside a tile of 2048 positions this runs in shared
//      memory; the seams between tiles are then checked in parallel, and the few that still
//      descend are repaired by one thread walking outwards from each seam.
//   2. the removed bodies (about 5% per step on the 16.8M two-cluster workload) are sorted by
//      (system, key, id) with the radix sort;
//   3. merge path of the two ascending sequences.
// The kept sequence ascends whatever the starting order, so the result is exact for any
// permutation; a start far from sorted only makes the removed set large.  Every loop is
// bounded: a tile still descending after 32 removal rounds is removed whole, and the seam repair
// gives up after a fixed number of steps.  The choice between this and the full sort (repair gave
// up, or too many removed) is made on the device and the kernels of the path not taken return at
// once, so a caller may launch both paths without reading the choice back (a forest step does).
#include "nbody_internal.cuh"

namespace nb {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kOrdThreads = 256;
constexpr int kOrdTile = 2048;                     // positions per extract tile
constexpr int kOrdItems = kOrdTile / kOrdThreads;  // 8 per thread
constexpr int kOrdWords = kOrdTile / 32;           // keep words per tile
constexpr int kOrdRounds = 32;                     // removal rounds before a tile is emptied
constexpr int kRepairBudget = 1 << 14;             // steps of the seam repair before it gives up
constexpr int kMergeTile = 2048;                   // outputs per merge block
constexpr int kMergeThreads = 256;

static_assert(kOrdWords == 64, "the count kernel reads two keep words per lane");

// (sa, ka, ia) comes after (sb, kb, ib) in the (system, key, id) order.
__device__ __forceinline__ bool after(unsigned sa, uint64_t ka, uint32_t ia, unsigned sb,
                                      uint64_t kb, uint32_t ib)
{
    if (sa != sb) return sa > sb;
    return ka > kb || (ka == kb && ia > ib);
}

__device__ __forceinline__ unsigned sys_of(const uint16_t *sys, uint32_t id)
{
    return sys ? (unsigned)sys[id] : 0u;
}

// The same for two positions of the previous order (their keys and ids in global memory).
__device__ __forceinline__ bool after_at(const uint64_t *keys, const uint32_t *prev,
                                         const uint16_t *sys, int a, int b)
{
    const uint32_t ia = prev[a], ib = prev[b];
    return after(sys_of(sys, ia), keys[a], ia, sys_of(sys, ib), keys[b], ib);
}

// ------------------------------------------------------------------------------------------
// 1. Extract.  Block t owns positions [2048 t, 2048 t + 2048) of the previous order.
// ------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(kOrdThreads) order_extract_kernel(
    const D4 *__restrict__ aos, const uint32_t *__restrict__ prev, int n,
    const Box *__restrict__ box, const uint16_t *__restrict__ sys, uint64_t *__restrict__ keys,
    uint32_t *__restrict__ keep, int2 *__restrict__ ends)
{
    // slot j + 1 holds position base + j; slots 0 and tn + 1 the neighbours across the tile ends
    __shared__ uint64_t sk[kOrdTile + 2];
    __shared__ uint32_t si[kOrdTile + 2];
    __shared__ uint16_t ss[kOrdTile + 2];  // system of each
    __shared__ uint32_t sw[kOrdWords];   // keep bits: bit j & 31 of word j >> 5
    __shared__ uint32_t sd[kOrdWords];   // bits removed in the current round
    __shared__ int snext[kOrdWords];     // first word after w with a kept position (-1: none)
    const int base = blockIdx.x * kOrdTile;
    const int tn = min(kOrdTile, n - base);
    const int lane = threadIdx.x & 31;

    for (int j = (int)threadIdx.x - 1; j <= tn; j += kOrdThreads) {
        const int g = base + j;
        if (g < 0 || g >= n) continue;
        const uint32_t id = prev[g];
        const unsigned sy = sys_of(sys, id);
        const D4 *r = aos + id;
        const uint64_t k = morton_key(r->x, r->y, r->z, box[sy]);
        sk[j + 1] = k;
        si[j + 1] = id;
        ss[j + 1] = (uint16_t)sy;
        if (j >= 0 && j < tn) keys[g] = k;
    }
    if (threadIdx.x < kOrdWords) sd[threadIdx.x] = 0u;
    __syncthreads();

    // first removal: both ends of every descent (the pairs across the tile ends included)
#pragma unroll
    for (int r = 0; r < kOrdItems; ++r) {
        const int j = r * kOrdThreads + threadIdx.x;  // j & 31 == lane
        const int g = base + j;
        bool kept = false;
        if (j < tn) {
            const bool dl = g > 0 && after(ss[j], sk[j], si[j], ss[j + 1], sk[j + 1], si[j + 1]);
            const bool dr =
                g + 1 < n && after(ss[j + 1], sk[j + 1], si[j + 1], ss[j + 2], sk[j + 2], si[j + 2]);
            kept = !(dl || dr);
        }
        const unsigned word = __ballot_sync(kFull, kept);
        if (lane == 0) sw[j >> 5] = word;
    }
    __syncthreads();

    // further rounds: every kept position against the next kept one of the tile
    for (int round = 0;; ++round) {
        if (threadIdx.x < kOrdWords) {
            int w = threadIdx.x + 1;
            while (w < kOrdWords && sw[w] == 0u) ++w;
            snext[threadIdx.x] = w < kOrdWords ? w : -1;
        }
        __syncthreads();
        bool found = false;
#pragma unroll
        for (int r = 0; r < kOrdItems; ++r) {
            const int j = r * kOrdThreads + threadIdx.x;
            const int w = j >> 5;
            const unsigned word = sw[w];
            if (j >= tn || !((word >> lane) & 1u)) continue;
            const unsigned above = lane == 31 ? 0u : word & (kFull << (lane + 1));
            int jn = -1;
            if (above) {
                jn = (w << 5) + __ffs(above) - 1;
            } else {
                const int wn = snext[w];
                if (wn >= 0) jn = (wn << 5) + __ffs(sw[wn]) - 1;
            }
            if (jn >= 0 &&
                after(ss[j + 1], sk[j + 1], si[j + 1], ss[jn + 1], sk[jn + 1], si[jn + 1])) {
                atomicOr(&sd[w], 1u << lane);
                atomicOr(&sd[jn >> 5], 1u << (jn & 31));
                found = true;
            }
        }
        if (!__syncthreads_or(found)) break;
        const bool last = round + 1 >= kOrdRounds;
        if (threadIdx.x < kOrdWords) {
            sw[threadIdx.x] = last ? 0u : (sw[threadIdx.x] & ~sd[threadIdx.x]);
            sd[threadIdx.x] = 0u;
        }
        __syncthreads();
        if (last) break;
    }

    if (threadIdx.x < kOrdWords) keep[(size_t)blockIdx.x * kOrdWords + threadIdx.x] = sw[threadIdx.x];
    if (threadIdx.x == 0) {
        int f = -1, l = -1;
        for (int w = 0; w < kOrdWords; ++w)
            if (sw[w]) {
                f = base + (w << 5) + __ffs(sw[w]) - 1;
                break;
            }
        for (int w = kOrdWords - 1; w >= 0; --w)
            if (sw[w]) {
                l = base + (w << 5) + 31 - __clz(sw[w]);
                break;
            }
        ends[blockIdx.x] = make_int2(f, l);
    }
}

// Marks tile t when its first kept position comes before the last kept position of the tiles
// in front of it (looked up over at most 64 empty tiles; beyond that the tile is marked anyway
// and the repair decides).
__global__ void order_seams_kernel(const uint64_t *__restrict__ keys,
                                   const uint32_t *__restrict__ prev,
                                   const uint16_t *__restrict__ sys,
                                   const int2 *__restrict__ ends, int tiles,
                                   uint32_t *__restrict__ seams, unsigned *__restrict__ stats)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 1 || t >= tiles) return;
    const int b = ends[t].x;
    if (b < 0) return;
    int a = -1, u = t - 1;
    for (int k = 0; k < 64 && u >= 0 && a < 0; ++k) a = ends[u--].y;
    const bool mark = a >= 0 ? after_at(keys, prev, sys, a, b) : u >= 0;
    if (mark) {
        atomicOr(&seams[t >> 5], 1u << (t & 31));
        atomicAdd(&stats[kOrderSeams], 1u);
    }
}

// Largest kept position <= i (-1: none, or the budget ran out).
__device__ __forceinline__ int kept_at_or_before(const uint32_t *keep, int i, int &budget)
{
    if (i < 0) return -1;
    int w = i >> 5;
    uint32_t m = keep[w] & (kFull >> (31 - (i & 31)));
    while (m == 0u) {
        if (--w < 0 || --budget < 0) return -1;
        m = keep[w];
    }
    return (w << 5) + 31 - __clz(m);
}

// Smallest kept position >= i (-1: none, or the budget ran out).
__device__ __forceinline__ int kept_at_or_after(const uint32_t *keep, int i, int nw, int &budget)
{
    int w = i >> 5;
    if (w >= nw) return -1;
    uint32_t m = keep[w] & (kFull << (i & 31));
    while (m == 0u) {
        if (++w >= nw || --budget < 0) return -1;
        m = keep[w];
    }
    return (w << 5) + __ffs(m) - 1;
}

// One thread, seams in ascending order: while the last kept position before the seam comes
// after the first kept one behind it, both are removed.  Everything in front of a repaired seam
// ascends (earlier seams are repaired first, and removal keeps an ascending run ascending), so
// after the last seam the whole kept sequence ascends.
__global__ void order_repair_kernel(const uint64_t *__restrict__ keys,
                                    const uint32_t *__restrict__ prev,
                                    const uint16_t *__restrict__ sys, int n, int tiles,
                                    uint32_t *__restrict__ keep,
                                    const uint32_t *__restrict__ seams, unsigned *stats)
{
    if (stats[kOrderSeams] == 0u) return;
    const int nw = (n + 31) >> 5;
    int budget = kRepairBudget;
    for (int v = 0; v < (tiles + 31) >> 5; ++v) {
        unsigned bits = seams[v];
        while (bits) {
            const int t = (v << 5) + __ffs(bits) - 1;
            bits &= bits - 1u;
            const int start = t * kOrdTile;
            int a = kept_at_or_before(keep, start - 1, budget);
            int b = kept_at_or_after(keep, start, nw, budget);
            while (a >= 0 && b >= 0 && after_at(keys, prev, sys, a, b)) {
                keep[a >> 5] &= ~(1u << (a & 31));
                keep[b >> 5] &= ~(1u << (b & 31));
                if (--budget < 0) break;
                a = kept_at_or_before(keep, a - 1, budget);
                b = kept_at_or_after(keep, b + 1, nw, budget);
            }
            if (budget < 0) {
                stats[kOrderGaveUp] = 1u;
                return;
            }
        }
    }
}

// Kept positions per tile (one warp per tile).
__global__ void order_count_kernel(const uint32_t *__restrict__ keep, int tiles,
                                   uint32_t *__restrict__ kept_cnt)
{
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= tiles) return;
    const uint32_t *w = keep + (size_t)t * kOrdWords;
    const unsigned c = __reduce_add_sync(kFull, (unsigned)(__popc(w[lane]) + __popc(w[lane + 32])));
    if (lane == 0) kept_cnt[t] = c;
}

// In-place exclusive scan of the per-tile counts (one block); then the choice of path: the
// re-sort unless the repair gave up or (auto_limit) more than a quarter of the n were removed.
__global__ void __launch_bounds__(1024) order_scan_kernel(uint32_t *kept_off, int tiles, int n,
                                                          int auto_limit, unsigned *stats)
{
    __shared__ uint32_t wsum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int t0 = 0; t0 < tiles; t0 += 1024) {
        const int t = t0 + threadIdx.x;
        const uint32_t v = t < tiles ? kept_off[t] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            uint32_t s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const uint32_t before = (wid > 0 ? wsum[wid - 1] : 0u) + x - v;
        if (t < tiles) kept_off[t] = carry + before;
        carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned removed = (unsigned)n - carry;
        const bool resort =
            stats[kOrderGaveUp] == 0u && !(auto_limit && 4ull * removed > (unsigned long long)n);
        stats[kOrderKept] = carry;
        stats[kOrderRemoved] = removed;
        stats[kOrderXn] = resort ? removed : 0u;
        stats[kOrderFullN] = resort ? 0u : (unsigned)n;
        stats[kOrderResorted] = resort ? 1u : 0u;
    }
}

// ------------------------------------------------------------------------------------------
// 2. Split the previous order into the kept (ascending) and removed bodies, both in order.
// ------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(kOrdThreads) order_split_kernel(
    const uint64_t *__restrict__ keys, const uint32_t *__restrict__ prev, int n,
    const uint32_t *__restrict__ keep, const uint32_t *__restrict__ kept_off,
    uint64_t *__restrict__ rk, uint32_t *__restrict__ ri, uint64_t *__restrict__ xk,
    uint32_t *__restrict__ xi, const unsigned *__restrict__ stats)
{
    if (stats[kOrderResorted] == 0u) return;
    __shared__ uint32_t sw[kOrdWords];
    __shared__ uint32_t spre[kOrdWords];  // kept positions of the tile before word w
    const int t = blockIdx.x, base = t * kOrdTile, tn = min(kOrdTile, n - base);
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < kOrdWords) {
        const uint32_t w = keep[(size_t)t * kOrdWords + threadIdx.x];
        sw[threadIdx.x] = w;
        const uint32_t c = __popc(w);
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        spre[threadIdx.x] = x - c;
    }
    __syncthreads();
    if (threadIdx.x >= 32 && threadIdx.x < kOrdWords) spre[threadIdx.x] += spre[31] + __popc(sw[31]);
    __syncthreads();
    const uint32_t kbase = kept_off[t];
    const uint32_t xbase = (uint32_t)base - kbase;
#pragma unroll
    for (int r = 0; r < kOrdItems; ++r) {
        const int j = r * kOrdThreads + threadIdx.x;
        if (j >= tn) break;
        const int g = base + j;
        const int w = j >> 5;
        const uint32_t word = sw[w];
        const uint32_t kb = spre[w] + __popc(word & ((1u << lane) - 1u));
        const uint64_t k = keys[g];
        const uint32_t id = prev[g];
        if ((word >> lane) & 1u) {
            rk[kbase + kb] = k;
            ri[kbase + kb] = id;
        } else {
            const uint32_t o = xbase + (uint32_t)j - kb;
            xk[o] = k;
            xi[o] = id;
        }
    }
}

// ------------------------------------------------------------------------------------------
// 3. Merge path: output tile t takes split[t] .. split[t+1] of the kept sequence and the rest of
// its outputs from the sorted removed sequence.
// ------------------------------------------------------------------------------------------

__global__ void order_partition_kernel(const uint64_t *__restrict__ rk,
                                       const uint32_t *__restrict__ ri,
                                       const uint64_t *__restrict__ xk,
                                       const uint32_t *__restrict__ xi,
                                       const uint16_t *__restrict__ sys, int tiles,
                                       const unsigned *__restrict__ stats, int *__restrict__ split)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > tiles || stats[kOrderResorted] == 0u) return;
    const int nr = (int)stats[kOrderKept], nx = (int)stats[kOrderXn];
    const int64_t total = (int64_t)nr + nx;
    const int diag = (int)min((int64_t)t * kMergeTile, total);
    int lo = max(0, diag - nx), hi = min(diag, nr);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int xo = diag - 1 - mid;
        if (after(sys_of(sys, xi[xo]), xk[xo], xi[xo], sys_of(sys, ri[mid]), rk[mid], ri[mid]))
            lo = mid + 1;
        else hi = mid;
    }
    split[t] = lo;
}

__global__ void __launch_bounds__(kMergeThreads) order_merge_kernel(
    const uint64_t *__restrict__ rk, const uint32_t *__restrict__ ri,
    const uint64_t *__restrict__ xk, const uint32_t *__restrict__ xi,
    const uint16_t *__restrict__ sys, const unsigned *__restrict__ stats,
    const int *__restrict__ split, uint64_t *__restrict__ keys, uint32_t *__restrict__ ids)
{
    if (stats[kOrderResorted] == 0u) return;
    const int nr = (int)stats[kOrderKept], nx = (int)stats[kOrderXn];
    __shared__ uint64_t sk[kMergeTile];  // this tile's kept bodies, then its removed ones
    __shared__ uint32_t si[kMergeTile];
    __shared__ uint16_t ss[kMergeTile];
    const int total = nr + nx;
    const int d0 = blockIdx.x * kMergeTile, d1 = min(d0 + kMergeTile, total);
    const int i0 = split[blockIdx.x], i1 = split[blockIdx.x + 1];
    const int j0 = d0 - i0, j1 = d1 - i1;
    const int cr = i1 - i0, cx = j1 - j0;
    for (int k = threadIdx.x; k < cr; k += kMergeThreads) {
        sk[k] = rk[i0 + k];
        si[k] = ri[i0 + k];
        ss[k] = (uint16_t)sys_of(sys, si[k]);
    }
    for (int k = threadIdx.x; k < cx; k += kMergeThreads) {
        sk[cr + k] = xk[j0 + k];
        si[cr + k] = xi[j0 + k];
        ss[cr + k] = (uint16_t)sys_of(sys, si[cr + k]);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < cr + cx; k += kMergeThreads) {
        const uint64_t key = sk[k];
        const uint32_t id = si[k];
        const unsigned sy = ss[k];
        // the other sequence's bodies of this tile that come before this one
        const bool kept = k < cr;
        const int o0 = kept ? cr : 0, len = kept ? cx : cr;
        int lo = 0, hi = len;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (after(sy, key, id, ss[o0 + mid], sk[o0 + mid], si[o0 + mid])) lo = mid + 1;
            else hi = mid;
        }
        const int p = d0 + (kept ? k : k - cr) + lo;
        keys[p] = key;
        ids[p] = id;
    }
}

}  // namespace

int order_tiles(int n) { return (n + kOrdTile - 1) / kOrdTile; }
int order_merge_tiles(int n) { return (n + kMergeTile - 1) / kMergeTile; }

void launch_order_extract(const D4 *aos, const uint32_t *prev, int n, const Box *box,
                          const Systems &ss, bool auto_limit, uint64_t *keys,
                          const OrderScratch &o, cudaStream_t s)
{
    const int tiles = order_tiles(n);
    cudaMemsetAsync(o.stats, 0, sizeof(unsigned) * kOrderStats, s);
    cudaMemsetAsync(o.seams, 0, sizeof(uint32_t) * ((tiles + 31) / 32), s);
    order_extract_kernel<<<tiles, kOrdThreads, 0, s>>>(aos, prev, n, box, ss.sys, keys, o.keep,
                                                       o.ends);
    order_seams_kernel<<<(tiles + 255) / 256, 256, 0, s>>>(keys, prev, ss.sys, o.ends, tiles,
                                                          o.seams, o.stats);
    order_repair_kernel<<<1, 1, 0, s>>>(keys, prev, ss.sys, n, tiles, o.keep, o.seams, o.stats);
    order_count_kernel<<<(tiles + 7) / 8, 256, 0, s>>>(o.keep, tiles, o.kept_off);
    order_scan_kernel<<<1, 1024, 0, s>>>(o.kept_off, tiles, n, auto_limit ? 1 : 0, o.stats);
    count_launches(5);
}

void launch_order_merge(uint64_t *keys, uint32_t *ids, int n, const Systems &ss,
                        const OrderScratch &o, const SortScratch &sc, cudaStream_t s)
{
    const int tiles = order_tiles(n);
    order_split_kernel<<<tiles, kOrdThreads, 0, s>>>(keys, ids, n, o.keep, o.kept_off, o.rk, o.ri,
                                                     o.xk, o.xi, o.stats);
    count_launches(1);
    int id_bits = 1;
    while (id_bits < 32 && ((uint64_t)(n - 1) >> id_bits) != 0) ++id_bits;
    // the removed bodies, sorted by (system, key, id): id passes, key passes, and for a forest
    // the system passes with digit totals counted over the removed bodies only
    SortScratch sx = sc;
    sx.sys = ss.sys;
    sx.sys_hist = nullptr;
    sx.d_n = reinterpret_cast<const int *>(o.stats + kOrderXn);
    uint64_t *xk = o.xk;
    uint32_t *xi = o.xi;
    launch_radix_sort_key_id(o.xk, o.xi, n, id_bits, sx, s, &xk, &xi);
    const int mt = order_merge_tiles(n);
    order_partition_kernel<<<(mt + 1 + 255) / 256, 256, 0, s>>>(o.rk, o.ri, xk, xi, ss.sys, mt,
                                                                 o.stats, o.split);
    order_merge_kernel<<<mt, kMergeThreads, 0, s>>>(o.rk, o.ri, xk, xi, ss.sys, o.stats, o.split,
                                                    keys, ids);
    count_launches(2);
}

}  // namespace nb

// Tree-build kernels: root box, Morton keys, LSD radix sort, body permutation, octree node
// split and bottom-up moments.
//
// Paper: Algorithm 2 ("Build Tree", moments from the leaves to the root), §4.4 (Morton keys:
// 21 bits per axis interleaved with x > y > z), §4.7 (hashed cell keys), §4.2 (pre-order node
// serialisation).  Every step here is integer or exact FP64 work, so keys, order and topology
// are bit-identical to a plain CPU evaluation of the same definitions.
#include <float.h>
#include <algorithm>
#include <atomic>
#include <math.h>

#include "nbody_internal.cuh"

namespace nb {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------------------------------
// Root box (§3: the root is the bounding box of all particles; §4.4 maps it onto [0, 2^21)).
// ------------------------------------------------------------------------------------------

constexpr int kBoxThreads = 256;
constexpr int kPart = 10;  // per-block partials: min x,y,z, max x,y,z, sum m, m x, m y, m z

// Block reduction of v[0..2] (min), v[3..5] (max), v[6..9] (sum) -> out[0..9] by thread 0.  The
// order of every operation is fixed by the launch shape, so the sums are deterministic.
__device__ __forceinline__ void block_reduce10(double v[kPart], double *out)
{
    __shared__ double sh[kPart][kBoxThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kPart; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(kFull, x, o);
            x = k < 3 ? fmin(x, y) : (k < 6 ? fmax(x, y) : __dadd_rn(x, y));
        }
        if (lane == 0) sh[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < kPart; ++k) {
            double x = sh[k][0];
            for (int w = 1; w < kBoxThreads / 32; ++w)
                x = k < 3 ? fmin(x, sh[k][w]) : (k < 6 ? fmax(x, sh[k][w]) : __dadd_rn(x, sh[k][w]));
            out[k] = x;
        }
    }
}

__device__ __forceinline__ void init10(double v[kPart])
{
    v[0] = v[1] = v[2] = DBL_MAX;
    v[3] = v[4] = v[5] = -DBL_MAX;
    v[6] = v[7] = v[8] = v[9] = 0.0;
}

// Order-preserving image of a finite double as a signed 64-bit integer (and back): a body's
// contribution to the box's min / max runs on the integer units instead of the FP64 pipe, which
// the kick, the drift and the mass-weighted sums already keep busy.  The extremes are the same
// values (-0 orders below +0, which changes neither the box's cube nor any key).
__device__ __forceinline__ long long dord(double x)
{
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}

__device__ __forceinline__ double dord_inv(long long o)
{
    return __longlong_as_double(o >= 0 ? o : (o ^ 0x7fffffffffffffffll));
}

// One thread's share of a box: integer images of the min and max corner, FP64 sums of m, m x,
// m y, m z (in the thread's body order).
struct BoxPart {
    long long lo[3], hi[3];
    double s[4];
};

__device__ __forceinline__ void box_init(BoxPart &p)
{
    for (int d = 0; d < 3; ++d) {
        p.lo[d] = dord(DBL_MAX);
        p.hi[d] = dord(-DBL_MAX);
    }
    p.s[0] = p.s[1] = p.s[2] = p.s[3] = 0.0;
}

__device__ __forceinline__ void add_body(BoxPart &p, double x, double y, double z, double m)
{
    const long long ox = dord(x), oy = dord(y), oz = dord(z);
    p.lo[0] = min(p.lo[0], ox); p.hi[0] = max(p.hi[0], ox);
    p.lo[1] = min(p.lo[1], oy); p.hi[1] = max(p.hi[1], oy);
    p.lo[2] = min(p.lo[2], oz); p.hi[2] = max(p.hi[2], oz);
    p.s[0] = __dadd_rn(p.s[0], m);
    p.s[1] = __fma_rn(m, x, p.s[1]);
    p.s[2] = __fma_rn(m, y, p.s[2]);
    p.s[3] = __fma_rn(m, z, p.s[3]);
}

// The thread's share as the 10 partials of block_reduce10.
__device__ __forceinline__ void box_values(const BoxPart &p, double v[kPart])
{
    for (int d = 0; d < 3; ++d) {
        v[d] = dord_inv(p.lo[d]);
        v[3 + d] = dord_inv(p.hi[d]);
    }
    for (int k = 0; k < 4; ++k) v[6 + k] = p.s[k];
}

// aos (may be null): the bodies as (x, y, z, m) records in the caller's order, which the
// permutation gathers with one 32-byte access per body.
__global__ void __launch_bounds__(kBoxThreads) bbox_partials_kernel(const double *__restrict__ pos,
                                                                    const double *__restrict__ mass,
                                                                    int n, double *partials,
                                                                    D4 *__restrict__ aos)
{
    BoxPart bp;
    box_init(bp);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        D4 b;
        b.x = pos[i];
        b.y = pos[(size_t)n + i];
        b.z = pos[2 * (size_t)n + i];
        b.w = mass[i];
        add_body(bp, b.x, b.y, b.z, b.w);
        if (aos) aos[i] = b;
    }
    double v[kPart];
    box_values(bp, v);
    block_reduce10(v, partials + kPart * blockIdx.x);
}

// One kick-and-drift coordinate (eqs. leapkick1, leapdrift of §2.4) in FP64: separately rounded
// products and sums as the oracle does them (FP64 contexts), or fused multiply-adds (FP32
// contexts, whose forces are FP32 anyway: half the FP64 operations, which bound these passes on
// GB300's narrow FP64 pipe).
template <bool kFused>
__device__ __forceinline__ void kick_drift1(double &v, double &x, double a, double h, double dt)
{
    if (kFused) {
        v = __fma_rn(a, h, v);
        x = __fma_rn(v, dt, x);
    } else {
        v = __dadd_rn(v, __dmul_rn(a, h));
        x = __dadd_rn(x, __dmul_rn(v, dt));
    }
}

// Kick and drift of the leapfrog (eqs. leapkick1, leapdrift of §2.4), fused with the box and
// centre-of-mass partials of the new positions.
template <bool kFused>
__global__ void __launch_bounds__(kBoxThreads) kick_drift_bbox_kernel(
    double *__restrict__ pos, double *__restrict__ vel, const double *__restrict__ acc,
    const double *__restrict__ mass, int n, double h, double dt, double *partials,
    D4 *__restrict__ aos)
{
    BoxPart bp;
    box_init(bp);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double x[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const size_t k = (size_t)d * n + i;
            double vh = vel[k];
            x[d] = pos[k];
            kick_drift1<kFused>(vh, x[d], acc[k], h, dt);
            vel[k] = vh;
            pos[k] = x[d];
        }
        const double m = mass[i];
        add_body(bp, x[0], x[1], x[2], m);
        D4 b;
        b.x = x[0];
        b.y = x[1];
        b.z = x[2];
        b.w = m;
        aos[i] = b;
    }
    double v[kPart];
    box_values(bp, v);
    block_reduce10(v, partials + kPart * blockIdx.x);
}

// Root cube (min corner, side = largest extent, 1 when all bodies coincide), the scale 2^21 / L,
// the per-level tables, and the origin of the FP32 coordinates: the centre of mass, so that FP32
// offsets stay small where the mass is (their absolute rounding error is 2^-24 of the offset).
// r: min x,y,z, max x,y,z, sum m, sum m x, m y, m z.
__device__ void finalize_box(const double r[kPart], double theta, Box *box, LevelTables *tab)
{
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        double e = __dsub_rn(r[3 + d], r[d]);
        if (e > ext) ext = e;
    }
    if (!(ext > 0.0)) ext = 1.0;
    for (int d = 0; d < 3; ++d) {
        box->o[d] = r[d];
        double c = r[6] > 0.0 ? r[7 + d] / r[6] : __dadd_rn(r[d], __dmul_rn(ext, 0.5));
        // keep the origin inside the box (guards against a non-finite or stray quotient)
        if (!(c >= r[d] && c <= r[3 + d])) c = __dadd_rn(r[d], __dmul_rn(ext, 0.5));
        box->c[d] = c;
    }
    box->L = ext;
    box->s = __ddiv_rn(2097152.0, ext);
    const double th2 = __dmul_rn(theta, theta);
    for (int lev = 0; lev < kLevels; ++lev) {
        double l = ldexp(ext, -lev);
        double l2 = __dmul_rn(l, l);
        tab->l2[lev] = l2;
        tab->crit32[lev] = th2 > 0.0 ? (float)__ddiv_rn(l2, th2) : __int_as_float(0x7f800000);
    }
}

__global__ void __launch_bounds__(kBoxThreads) bbox_finalize_kernel(const double *partials,
                                                                    int nblk, Box *box,
                                                                    LevelTables *tab, double theta)
{
    double v[kPart];
    init10(v);
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        const double *p = partials + kPart * b;
        for (int k = 0; k < 3; ++k) v[k] = fmin(v[k], p[k]);
        for (int k = 3; k < 6; ++k) v[k] = fmax(v[k], p[k]);
        for (int k = 6; k < kPart; ++k) v[k] = __dadd_rn(v[k], p[k]);
    }
    __shared__ double r[kPart];
    block_reduce10(v, r);
    __syncthreads();
    if (threadIdx.x == 0) finalize_box(r, theta, box, tab);
}

// Forest: leapfrog kick and drift of every body (eqs. leapkick1, leapdrift of §2.4).
// Forest: one block per system reduces its bodies and writes its root box and level tables.
// Forest: the partial box of one chunk of bodies per block (a chunk never crosses a system),
// with a step's kick and drift fused in when vel is non-null (the same operations as
// kick_drift_bbox_kernel), writing the (x, y, z, m) records.  chunks[b] = (first body, end,
// system).
template <bool kFused>
__global__ void __launch_bounds__(kBoxThreads) forest_box_partials_kernel(
    double *__restrict__ pos, double *__restrict__ vel, const double *__restrict__ acc,
    const double *__restrict__ mass, int n, const int4 *__restrict__ chunks, double h, double dt,
    double *__restrict__ partials, D4 *__restrict__ aos)
{
    const int4 ch = chunks[blockIdx.x];
    BoxPart bp;
    box_init(bp);
    for (int i = ch.x + threadIdx.x; i < ch.y; i += blockDim.x) {
        double r[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const size_t k = (size_t)d * n + i;
            if (vel) {
                double vh = vel[k];
                r[d] = pos[k];
                kick_drift1<kFused>(vh, r[d], acc[k], h, dt);
                vel[k] = vh;
                pos[k] = r[d];
            } else {
                r[d] = pos[k];
            }
        }
        D4 b;
        b.x = r[0];
        b.y = r[1];
        b.z = r[2];
        b.w = mass[i];
        add_body(bp, b.x, b.y, b.z, b.w);
        aos[i] = b;
    }
    double v[kPart];
    box_values(bp, v);
    block_reduce10(v, partials + kPart * blockIdx.x);
}

// Forest: one block per system, its root box from its chunks' partials (chunks chunk_start[k]
// .. chunk_start[k + 1] - 1; none for an empty system).
__global__ void __launch_bounds__(kBoxThreads) forest_box_finalize_kernel(
    const double *__restrict__ partials, const int *__restrict__ chunk_start, Box *box,
    LevelTables *tab, double theta)
{
    const int k = blockIdx.x;
    double v[kPart];
    init10(v);
    for (int b = chunk_start[k] + threadIdx.x; b < chunk_start[k + 1]; b += blockDim.x) {
        const double *p = partials + kPart * b;
        for (int e = 0; e < 3; ++e) v[e] = fmin(v[e], p[e]);
        for (int e = 3; e < 6; ++e) v[e] = fmax(v[e], p[e]);
        for (int e = 6; e < kPart; ++e) v[e] = __dadd_rn(v[e], p[e]);
    }
    __shared__ double r[kPart];
    block_reduce10(v, r);
    __syncthreads();
    if (threadIdx.x == 0) finalize_box(r, theta, box + k, tab + k);
}

// ------------------------------------------------------------------------------------------
// Morton keys (§4.4) of the bodies in the caller's order (morton_key), with ids = 0 .. n-1.
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ int system_of(const Systems &ss, int i)
{
    return ss.sys ? (int)ss.sys[i] : 0;
}

__global__ void keys_kernel(const double *__restrict__ pos, int n, const Box *__restrict__ box,
                            Systems ss, uint64_t *__restrict__ keys, uint32_t *__restrict__ ids,
                            const int *__restrict__ gate)
{
    if (gate && *gate == 0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Box *b = box + system_of(ss, i);
        keys[i] = morton_key(pos[i], pos[(size_t)n + i], pos[2 * (size_t)n + i], *b);
        ids[i] = (uint32_t)i;
    }
}

// ------------------------------------------------------------------------------------------
// Stable LSD radix sort of (key, id) pairs, 8 passes of 8 bits (keys have 63 significant bits).
// Per pass: tile digit counts (upsweep) -> per-digit scan over tiles (row scan, seeded by the
// global digit histogram) -> stable scatter through a shared-memory reorder (downsweep).
// No inter-block waiting anywhere: every kernel only reads what earlier launches wrote.
// ------------------------------------------------------------------------------------------

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                         // per thread
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096 keys per tile
constexpr int kPasses = kSortKeyPasses;  // key passes
constexpr int kSysPasses = 2;    // forest: system passes (systems < 2^16)
constexpr int kIdPasses = 4;     // at most: passes on the id bytes before the key passes
constexpr int kHistRows = kPasses + kIdPasses + kSysPasses;  // key, id, system digit totals
static_assert(kSortTile == kSortTileKeys && kHistRows == kSortHistRows,
              "sort geometry shared through nbody_internal.cuh");

// Pairs to sort: n, or (d_n non-null) the count on the device, at most n (the grids are sized
// for n and the blocks past the device count return at once).
__device__ __forceinline__ int sort_count(int n, const int *d_n) { return d_n ? min(*d_n, n) : n; }
__device__ __forceinline__ int sort_tiles_dev(int n) { return (n + kSortTile - 1) / kSortTile; }
constexpr size_t kDownSmem = (size_t)kSortTile * 8 + (size_t)kSortTile * 4 +
                             (size_t)kSortWarps * 256 * 4 + 256 * 4 + 256 * 4;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Digit totals of every pass: rows 0-7 the key bytes, rows 8.. the low id bytes (id_passes), rows
// 12-13 the bytes of the system of each id (sys non-null: a subset of a forest's bodies).
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t *__restrict__ keys,
                                                                 const uint32_t *__restrict__ ids,
                                                                 int n, const int *d_n,
                                                                 int id_passes,
                                                                 const uint16_t *__restrict__ sys,
                                                                 uint32_t *hist)
{
    __shared__ uint32_t sh[kHistRows][256];
    const int rows = sys ? kHistRows : kPasses + id_passes;
    for (int k = threadIdx.x; k < kHistRows * 256; k += blockDim.x) (&sh[0][0])[k] = 0;
    __syncthreads();
    n = sort_count(n, d_n);
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int i = base + threadIdx.x;
        const bool ok = i < n;
        const uint64_t k = ok ? keys[i] : 0;
#pragma unroll
        for (int p = 0; p < kPasses; ++p) {
            const unsigned d = ok ? (unsigned)((k >> (8 * p)) & 255u) : 256u;
            const unsigned peers = __match_any_sync(kFull, d);
            if (ok && (__ffs(peers) - 1) == lane) atomicAdd(&sh[p][d], __popc(peers));
        }
        if (id_passes > 0 || sys) {
            const uint32_t id = ok ? ids[i] : 0u;
            for (int p = 0; p < id_passes; ++p) {
                const unsigned d = ok ? (id >> (8 * p)) & 255u : 256u;
                const unsigned peers = __match_any_sync(kFull, d);
                if (ok && (__ffs(peers) - 1) == lane)
                    atomicAdd(&sh[kPasses + p][d], __popc(peers));
            }
            if (sys) {
                const unsigned sv = ok ? (unsigned)sys[id] : 0u;
                for (int p = 0; p < kSysPasses; ++p) {
                    const unsigned d = ok ? (sv >> (8 * p)) & 255u : 256u;
                    const unsigned peers = __match_any_sync(kFull, d);
                    if (ok && (__ffs(peers) - 1) == lane)
                        atomicAdd(&sh[kPasses + kIdPasses + p][d], __popc(peers));
                }
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < rows * 256; k += blockDim.x) {
        uint32_t v = (&sh[0][0])[k];
        if (v) atomicAdd(&hist[k], v);
    }
}

// Digit of an element: a byte of its key, a byte of the system of its id (forest passes) or a
// byte of its id (passes that order equal keys by id when the ids are not ascending).
enum : int { kDigitKey = 0, kDigitSys = 1, kDigitId = 2 };
template <int kMode>
__device__ __forceinline__ unsigned sort_digit(uint64_t key, uint32_t id, int shift,
                                               const uint16_t *sys)
{
    if (kMode == kDigitSys) return ((unsigned)sys[id] >> shift) & 255u;
    if (kMode == kDigitId) return (id >> shift) & 255u;
    return (unsigned)((key >> shift) & 255u);
}

template <int kMode>
__global__ void __launch_bounds__(kSortThreads) radix_upsweep_kernel(const uint64_t *__restrict__ keys,
                                                                    const uint32_t *__restrict__ ids,
                                                                    int n, const int *d_n,
                                                                    int shift, uint32_t *counts,
                                                                    int tiles,
                                                                    const uint16_t *__restrict__ sys)
{
    n = sort_count(n, d_n);
    if ((int)blockIdx.x >= sort_tiles_dev(n)) return;
    __shared__ uint32_t sh[256];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int tile0 = blockIdx.x * kSortTile + wid * (kSortItems * 32);
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        const int i = tile0 + r * 32 + lane;
        const bool ok = i < n;
        const unsigned d =
            ok ? sort_digit<kMode>(kMode == kDigitKey ? keys[i] : 0ull,
                                   kMode != kDigitKey ? ids[i] : 0u, shift, sys)
               : 256u;
        const unsigned peers = __match_any_sync(kFull, d);
        if (ok && (__ffs(peers) - 1) == lane) atomicAdd(&sh[d], __popc(peers));
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * tiles + blockIdx.x] = sh[threadIdx.x];
}

// Block-wide exclusive scan of one uint32 per thread; *total receives the block sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t sh[33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < nw ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const uint32_t before = wid > 0 ? sh[wid - 1] : 0u;
    *total = sh[nw - 1];
    __syncthreads();
    return before + x - v;
}

// One block per digit: offsets of that digit's run in every tile, seeded by the number of keys
// with a smaller digit (from the global histogram of this pass).  Rows are `tiles` apart; the
// tiles in use follow from the pair count.
__global__ void __launch_bounds__(kSortThreads) radix_rowscan_kernel(uint32_t *counts, int tiles,
                                                                    int n, const int *d_n,
                                                                    const uint32_t *hist_pass)
{
    const int used = sort_tiles_dev(sort_count(n, d_n));
    const int d = blockIdx.x;
    uint32_t part = 0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) part += hist_pass[k];
    uint32_t base;
    (void)block_exclusive_scan(part, &base);
    uint32_t *row = counts + (size_t)d * tiles;
    uint32_t carry = base;
    for (int t0 = 0; t0 < used; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const uint32_t v = t < used ? row[t] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, &tot);
        if (t < used) row[t] = carry + ex;
        carry += tot;
    }
}

template <int kMode>
__global__ void __launch_bounds__(kSortThreads) radix_downsweep_kernel(
    const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ ids_in,
    uint64_t *__restrict__ keys_out, uint32_t *__restrict__ ids_out, int n, const int *d_n,
    int shift, const uint32_t *__restrict__ offsets, int tiles, const uint16_t *__restrict__ sys)
{
    n = sort_count(n, d_n);
    if ((int)blockIdx.x >= sort_tiles_dev(n)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *s_keys = reinterpret_cast<uint64_t *>(smem);
    uint32_t *s_ids = reinterpret_cast<uint32_t *>(s_keys + kSortTile);
    uint32_t *s_warp = s_ids + kSortTile;                 // [warp][256]
    uint32_t *s_start = s_warp + kSortWarps * 256;        // digit start inside the tile
    int *s_gofs = reinterpret_cast<int *>(s_start + 256); // global offset minus s_start

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int tile_base = blockIdx.x * kSortTile;
    const int tile_n = min(kSortTile, n - tile_base);
    for (int k = threadIdx.x; k < kSortWarps * 256; k += blockDim.x) s_warp[k] = 0;
    __syncthreads();

    uint64_t k[kSortItems];
    uint32_t id[kSortItems];
    uint32_t rank[kSortItems];
    const int w0 = tile_base + wid * (kSortItems * 32);
    uint32_t *hist = s_warp + wid * 256;
    const unsigned below = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int i = w0 + r * 32 + lane;
        const bool ok = i < n;
        k[r] = ok ? keys_in[i] : 0ull;
        id[r] = ok ? ids_in[i] : 0u;
        const unsigned d = ok ? sort_digit<kMode>(k[r], id[r], shift, sys) : 256u;
        const unsigned peers = __match_any_sync(kFull, d);
        const uint32_t before = ok ? hist[d] : 0u;
        __syncwarp();
        rank[r] = before + __popc(peers & below);
        if (ok && (__ffs(peers) - 1) == lane) hist[d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps for every digit; digit totals of the tile
    {
        const int d = threadIdx.x;  // 256 threads <-> 256 digits
        uint32_t sum = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t t = s_warp[w * 256 + d];
            s_warp[w * 256 + d] = sum;
            sum += t;
        }
        uint32_t tot;
        const uint32_t start = block_exclusive_scan(sum, &tot);
        s_start[d] = start;
        s_gofs[d] = (int)offsets[(size_t)d * tiles + blockIdx.x] - (int)start;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int i = w0 + r * 32 + lane;
        if (i < n) {
            const unsigned d = sort_digit<kMode>(k[r], id[r], shift, sys);
            const uint32_t p = s_start[d] + s_warp[wid * 256 + d] + rank[r];
            s_keys[p] = k[r];
            s_ids[p] = id[r];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < tile_n; i += blockDim.x) {
        const uint64_t kk = s_keys[i];
        const unsigned d = sort_digit<kMode>(kk, s_ids[i], shift, sys);
        const int o = s_gofs[d] + i;
        keys_out[o] = kk;
        ids_out[o] = s_ids[i];
    }
}

// ------------------------------------------------------------------------------------------
// Permutation into Morton order: FP64 (x, y, z, m) and the FP32 copy relative to the box
// centre with w = G m.
// ------------------------------------------------------------------------------------------

__global__ void permute_kernel(const D4 *__restrict__ aos, const uint32_t *__restrict__ ids, int n,
                               const Box *__restrict__ box, Systems ss, double G,
                               D4 *__restrict__ sbody64, float4 *__restrict__ sbody32)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Box *bx = box + system_of(ss, i);
        const double cx = bx->c[0], cy = bx->c[1], cz = bx->c[2];
        const D4 b = aos[ids[i]];
        sbody64[i] = b;
        sbody32[i] = make_float4((float)(b.x - cx), (float)(b.y - cy), (float)(b.z - cz),
                                 (float)(G * b.w));
    }
}

// ------------------------------------------------------------------------------------------
// Node split.  With lcp(i) = number of leading 3-bit digits shared by sorted keys i and i+1
// (21 when the keys are equal; -1 past either end), the uncompressed octree has
//   - an internal cell at level l (0 <= l <= 20) for every maximal run of pairs with lcp >= l,
//   - a level-21 bucket for every maximal run of pairs with lcp == 21,
//   - a one-body leaf at level max(lcp(a-1), lcp(a)) + 1 for every body a outside a bucket.
// In pre-order a node's subtree is a contiguous index range, nodes are ordered by
// (first body, level), and body a starts the nodes at levels lcp(a-1)+1 .. onwards.  A count
// per body, one exclusive scan and one emit pass therefore lay the tree out in pre-order.
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ int lcp_digits(uint64_t a, uint64_t b)
{
    const uint64_t x = a ^ b;
    if (x == 0) return kMaxLevel;
    return (__clzll((long long)x) - 1) / 3;
}

// Body a's system spans sorted indices lo .. hi - 1 (0 .. n - 1 for a single system).
__device__ __forceinline__ void system_range(const Systems &ss, int n, int a, int &lo, int &hi)
{
    if (ss.sys) {
        const int k = ss.sys[a];
        lo = ss.start[k];
        hi = ss.start[k + 1];
    } else {
        lo = 0;
        hi = n;
    }
}

// lcp with the previous and the next body of the same system (-1 past either end).
__device__ __forceinline__ void body_lcps(const uint64_t *keys, int lo, int hi, int a, int &lp,
                                          int &la)
{
    const uint64_t ka = keys[a];
    lp = a > lo ? lcp_digits(keys[a - 1], ka) : -1;
    la = a + 1 < hi ? lcp_digits(ka, keys[a + 1]) : -1;
}

__device__ __forceinline__ uint32_t nodes_started(int lp, int la)
{
    if (la == kMaxLevel) return lp == kMaxLevel ? 0u : (uint32_t)(kMaxLevel - lp);
    if (lp == kMaxLevel) return 0u;
    return (uint32_t)(max(0, la - lp) + 1);
}

// Nodes started by every body, and (atomic max into *max_level) the deepest node level.
__global__ void count_nodes_kernel(const uint64_t *__restrict__ keys, int n, Systems ss,
                                   uint32_t *counts, unsigned *max_level)
{
    unsigned deepest = 0;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a <= n; a += gridDim.x * blockDim.x) {
        if (a == n) { counts[n] = 0; continue; }
        int lo, hi, lp, la;
        system_range(ss, n, a, lo, hi);
        body_lcps(keys, lo, hi, a, lp, la);
        counts[a] = nodes_started(lp, la);
        const int lv = (la == kMaxLevel || lp == kMaxLevel) ? kMaxLevel : max(lp, la) + 1;
        deepest = max(deepest, (unsigned)lv);
    }
    deepest = __reduce_max_sync(kFull, deepest);
    if ((threadIdx.x & 31) == 0 && deepest > 0) atomicMax(max_level, deepest);
}

// First index c > lo (c <= n) whose key differs from keys[lo] above `shift`, given that
// keys[lo] already shares the prefix.  Exponential then binary search.
__device__ int run_end(const uint64_t *keys, int n, int lo, uint64_t prefix, int shift)
{
    int step = 1;
    for (;;) {
        const int probe = lo + step;
        if (probe >= n || (keys[probe] >> shift) != prefix) break;
        lo = probe;
        step <<= 1;
    }
    int hi = min(lo + step, n);
    while (hi - lo > 1) {
        const int mid = lo + ((hi - lo) >> 1);
        if ((keys[mid] >> shift) == prefix) lo = mid; else hi = mid;
    }
    return hi;
}

__global__ void emit_nodes_kernel(const uint64_t *__restrict__ keys, int n, Systems ss,
                                  const uint32_t *__restrict__ node_off, NodeArrays na, int *err)
{
    if (*na.d_nn == 0u) return;  // the tree did not fit: no node is written (see clamp_count)
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        int lo, hi, lp, la;
        system_range(ss, n, a, lo, hi);
        body_lcps(keys, lo, hi, a, lp, la);
        const uint32_t k = nodes_started(lp, la);
        if (k == 0) continue;
        const int base = (int)node_off[a];
        if ((int64_t)base + k > na.cap) {   // more nodes than the arrays hold: write none
            atomicOr(err, kErrNodeCap);
            continue;
        }
        const uint64_t ka = keys[a];
        // levels of the cells (internal or bucket) that start at body a, deepest first so each
        // search starts from the end of the nested deeper run.
        const int top = lp + 1;
        const int deepest_run = (la == kMaxLevel) ? kMaxLevel : la;  // may be < top: no runs
        int end = a + 1;
        for (int l = deepest_run; l >= top; --l) {
            const int shift = 3 * (kMaxLevel - l);
            const uint64_t prefix = shift >= 64 ? 0ull : (ka >> shift);
            end = run_end(keys, hi, max(a + 1, end - 1), prefix, shift);
            const int idx = base + (l - top);
            WalkNode w;
            w.c = make_float4(0.f, 0.f, 0.f, 0.f);
            w.first = a;
            w.count = (l == kMaxLevel) ? (end - a) : 0;   // buckets are leaves
            w.skip = (int)node_off[end];
            w.crit = 0.f;
            na.wn[idx] = w;
            na.level[idx] = (uint8_t)l;
        }
        if (la != kMaxLevel) {
            const int l = max(lp, la) + 1;  // one-body leaf
            const int idx = base + (int)k - 1;
            WalkNode w;
            w.c = make_float4(0.f, 0.f, 0.f, 0.f);
            w.first = a;
            w.count = 1;
            w.skip = idx + 1;
            w.crit = 0.f;
            na.wn[idx] = w;
            na.level[idx] = (uint8_t)l;
        }
    }
}

__device__ __forceinline__ D4 ld_cg(const D4 *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const double2 a = __ldcg(q), b = __ldcg(q + 1);
    D4 r;
    r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
    return r;
}

// Adds a mass m at offset (x, y, z) from a centre of mass to a quadrupole (§2.2):
// Q_ab += m (3 x_a x_b - r^2 delta_ab), components xx, yy, zz, xy, xz, yz.
__device__ __forceinline__ void quad_add(double q[6], double m, double x, double y, double z)
{
    const double r2 = x * x + y * y + z * z;
    q[0] += m * (3.0 * x * x - r2);
    q[1] += m * (3.0 * y * y - r2);
    q[2] += m * (3.0 * z * z - r2);
    q[3] += m * (3.0 * x * y);
    q[4] += m * (3.0 * x * z);
    q[5] += m * (3.0 * y * z);
}

__device__ __forceinline__ void store_quad(NodeArrays &na, int j, int b, const double q[6],
                                           double G)
{
    for (int k = 0; k < 6; ++k) {
        na.q_lo[6 * (size_t)b + k] = q[k];
        na.q64[6 * (size_t)j + k] = q[k];
    }
    if (na.gq) {
        na.gq[2 * (size_t)b] = make_float4((float)(G * q[0]), (float)(G * q[1]), (float)(G * q[2]),
                                           (float)(G * q[3]));
        na.gq[2 * (size_t)b + 1] = make_float4((float)(G * q[4]), (float)(G * q[5]), 0.f, 0.f);
    }
}

__device__ __forceinline__ void store_node(NodeArrays &na, int j, const WalkNode &w0, const D4 &m,
                                           const Box *box, double G, float crit)
{
    na.com64[j] = m;
    WalkNode w = w0;
    w.c = make_float4((float)(m.x - box->c[0]), (float)(m.y - box->c[1]),
                      (float)(m.z - box->c[2]), (float)(G * m.w));
    w.crit = crit;
    na.wn[j] = w;
}

// Child masks and node kinds, plus the moments of every leaf (Algorithm 2, moments from the
// leaves up): a one-body leaf holds its body; a level-21 bucket the mass-weighted mean of its
// bodies in Morton order, every product and sum separately rounded.
__global__ void link_leaves_kernel(const uint64_t *__restrict__ keys, NodeArrays na,
                                   const D4 *__restrict__ sbody64, const Box *__restrict__ box,
                                   Systems ss, double G)
{
    const int n_nodes = (int)min((int64_t)*na.d_nn, na.cap);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_nodes; j += gridDim.x * blockDim.x) {
        const WalkNode w = na.wn[j];
        const int lev = na.level[j];
        if (w.count != 0) {
            na.mask[j] = 0;
            na.kind[j] = kLeafKind;
            D4 m;
            if (w.count == 1) {
                m = sbody64[w.first];
            } else {
                double s = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
                for (int b = w.first; b < w.first + w.count; ++b) {
                    const D4 q = sbody64[b];
                    s = __dadd_rn(s, q.w);
                    sx = __dadd_rn(sx, __dmul_rn(q.w, q.x));
                    sy = __dadd_rn(sy, __dmul_rn(q.w, q.y));
                    sz = __dadd_rn(sz, __dmul_rn(q.w, q.z));
                }
                m.w = s;
                m.x = __ddiv_rn(sx, s);
                m.y = __ddiv_rn(sy, s);
                m.z = __ddiv_rn(sz, s);
            }
            store_node(na, j, w, m, box + system_of(ss, w.first), G, 0.f);
            const int b = na.order[j];
            na.com_lo[b] = m;
            na.lo_child[b] = make_int4(0, 0, w.first, 0);
            if (na.q_lo) {
                // quadrupole of the leaf's bodies about their centre of mass (§2.2): 0 for one
                // body; a bucket sums over its members
                double q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                for (int p = w.first; w.count > 1 && p < w.first + w.count; ++p) {
                    const D4 r = sbody64[p];
                    quad_add(q, r.w, r.x - m.x, r.y - m.y, r.z - m.z);
                }
                store_quad(na, j, b, q, G);
            }
            continue;
        }
        const int shift = 3 * (kMaxLevel - 1 - lev);
        unsigned mask = 0;
        int nc = 0;
        // an internal cell has at most 8 children; the bound also ends the loop on a malformed
        // skip chain
        for (int c = j + 1; c < w.skip && nc < 8; c = max(na.wn[c].skip, c + 1), ++nc)
            mask |= 1u << (unsigned)((keys[na.wn[c].first] >> shift) & 7u);
        na.mask[j] = (uint8_t)mask;
        na.kind[j] = (uint8_t)lev;
        // children of a cell are consecutive in level order, starting with the next pre-order node
        na.lo_child[na.order[j]] = make_int4(na.order[j + 1], __popc(mask), w.first, 0);
    }
}

// Moments of the internal cells of one level, from their children (one level deeper, already
// done): m = sum m_c, r = (sum m_c r_c) / m over the children in octant order, every product and
// sum separately rounded.  Launched for the levels from the deepest up to the root.
__global__ void moments_level_kernel(int level, NodeArrays na, double G)
{
    // the nodes of this level are level-order indices [start(level), start(level + 1)); the
    // children of each cell are a contiguous level-order run (in octant order)
    const int lo = (int)na.tile_offsets[level * na.tiles];
    const int hi = (int)na.tile_offsets[(level + 1) * na.tiles];
    for (int t = lo + blockIdx.x * blockDim.x + threadIdx.x; t < hi; t += gridDim.x * blockDim.x) {
        const int4 ch = na.lo_child[t];
        if (ch.y == 0) continue;  // leaf: done by link_leaves
        double s = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int k = 0; k < min(ch.y, 8); ++k) {
            const D4 q = ld_cg(&na.com_lo[ch.x + k]);
            s = __dadd_rn(s, q.w);
            sx = __dadd_rn(sx, __dmul_rn(q.w, q.x));
            sy = __dadd_rn(sy, __dmul_rn(q.w, q.y));
            sz = __dadd_rn(sz, __dmul_rn(q.w, q.z));
        }
        D4 m;
        m.w = s;
        m.x = __ddiv_rn(sx, s);
        m.y = __ddiv_rn(sy, s);
        m.z = __ddiv_rn(sz, s);
        na.com_lo[t] = m;
        const int j = na.inv[t];
        na.com64[j] = m;  // its FP32 copy for the walk is made by group_nodes_kernel
        if (na.q_lo) {
            // parallel-axis sum: each child's quadrupole plus its mass at its offset
            double q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int c = 0; c < min(ch.y, 8); ++c) {
                const D4 r = ld_cg(&na.com_lo[ch.x + c]);
                const double *qc = na.q_lo + 6 * (size_t)(ch.x + c);
                for (int e = 0; e < 6; ++e) q[e] += __ldcg(qc + e);
                quad_add(q, r.w, r.x - m.x, r.y - m.y, r.z - m.z);
            }
            store_quad(na, j, t, q, G);
        }
    }
}

// ------------------------------------------------------------------------------------------
// Moments of FP32 contexts without quadrupoles.  The FP32 walks read each cell's centre of mass
// in FP32 only, so the leaves-to-root pass keeps FP64 sums instead of FP64 means: every node
// holds (sum m x, sum m y, sum m z, sum m) over its bodies, a cell adds its children's sums in
// octant order, and the centre of mass is formed once per node (one FP64 reciprocal, three
// products) when the level-order copy for the walk is written.  The FP64 contexts, and the
// quadrupole terms, keep the means of link_leaves / moments_level, bit for bit the oracle's.
// ------------------------------------------------------------------------------------------

// FP32 (x - c, y - c, z - c, G m) of a node from its sums: centre of mass = sums / m.
__device__ __forceinline__ float4 com32_from_sums(const D4 &sm, const Box *bx, double G)
{
    const double r = __drcp_rn(sm.w);
    return make_float4((float)(sm.x * r - bx->c[0]), (float)(sm.y * r - bx->c[1]),
                       (float)(sm.z * r - bx->c[2]), (float)(G * sm.w));
}

// One block per pre-order tile of kSubT nodes.  A node's subtree is the pre-order range
// [j, skip); when it ends inside the tile the block finishes the node here: a leaf's sums over its
// bodies in sorted order, a cell's as its children's sums in octant order, level by level from
// the deepest up, in shared memory.  Every node gets its child mask and its level-order GroupNode
// record.  The nodes whose subtree runs past the tile are ancestors of the first node after it,
// at most one per level: their records are written without the centre of mass, and their
// level-order index goes to spine[level * tiles + tile] (-1 where the tile has none) for
// spine_sums_kernel.  com_lo keeps the FP64 sums of the nodes the spine cells read (those whose
// parent is not finished in the same tile), or of every node with all_sums.  The FP64 pipe is narrow, so its work runs on compacted lists: the tile's
// cells are counting-sorted by level (deepest first), and each level's cells, then all of them
// for the centres of mass, take one thread each.
constexpr int kSubT = 1024;
constexpr int kSubThreads = 256;
constexpr int kSubPer = kSubT / kSubThreads;

__global__ void __launch_bounds__(kSubThreads, 4)
subtree_sums_kernel(const uint64_t *__restrict__ keys, NodeArrays na,
                    const D4 *__restrict__ sbody64, const float4 *__restrict__ sbody32,
                    const Box *__restrict__ box, const LevelTables *__restrict__ tab, Systems ss,
                    double G, GroupNode *__restrict__ gn, int4 *__restrict__ spine, int tiles,
                    int all_sums)
{
    __shared__ D4 s_sum[kSubT];
    __shared__ int s_skip[kSubT];          // skip - j0 (past kSubT for the spine)
    __shared__ uint16_t s_list[kSubT];     // the tile's cells, deepest level first
    __shared__ uint16_t s_sys[kSubT];      // system of the node
    __shared__ uint8_t s_oct[kSubT];       // octant of the node in its parent
    __shared__ uint8_t s_mask[kSubT];      // child mask of a cell finished here
    __shared__ uint8_t s_in[kSubT];        // its parent is finished here too
    __shared__ int s_cnt[kMaxLevel];       // cells per level
    __shared__ int s_start[kMaxLevel + 1]; // start of each level's run in s_list; [kMaxLevel] all
    __shared__ int4 s_spine[kMaxLevel];    // (level-order index, first child, child count, system)
    const int tile = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int n_nodes = (int)min((int64_t)*na.d_nn, na.cap);
    const int j0 = tile * kSubT;
    if (threadIdx.x < kMaxLevel) {
        s_spine[threadIdx.x] = make_int4(-1, 0, 0, 0);
        s_cnt[threadIdx.x] = 0;
    }
    __syncthreads();
    // the loads of all four nodes first (independent of one another), then their use
    int4 w[kSubPer];  // skip, first, count, crit bits
    int lev[kSubPer];
#pragma unroll
    for (int q = 0; q < kSubPer; ++q) {
        const int j = j0 + threadIdx.x + q * kSubThreads;
        w[q] = make_int4(0, 0, -1, 0);
        lev[q] = -1;
        if (j < n_nodes) {
            w[q] = reinterpret_cast<const int4 *>(na.wn + j)[1];
            lev[q] = na.level[j];
        }
    }
    uint64_t key[kSubPer];
#pragma unroll
    for (int q = 0; q < kSubPer; ++q) key[q] = lev[q] > 0 ? keys[w[q].y] : 0ull;
    // single-body leaves: their body's record straight into the sums slot (async copy, no
    // registers); products formed below
#pragma unroll
    for (int q = 0; q < kSubPer; ++q) {
        const int i = threadIdx.x + q * kSubThreads;
        if (w[q].z == 1) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(&s_sum[i]);
            const D4 *src = sbody64 + w[q].y;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16u),
                         "l"(reinterpret_cast<const char *>(src) + 16));
        }
    }
    asm volatile("cp.async.commit_group;\n" ::);
    // cells: their rank within their level (warp-aggregated counts)
    int rank[kSubPer];
#pragma unroll
    for (int q = 0; q < kSubPer; ++q) {
        const int i = threadIdx.x + q * kSubThreads;
        const bool cell = lev[q] >= 0 && w[q].z == 0;
        const unsigned peers = __match_any_sync(kFull, cell ? lev[q] : -1);
        rank[q] = 0;
        if (cell) {
            const int leader = __ffs(peers) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&s_cnt[lev[q]], __popc(peers));
            base = __shfl_sync(peers, base, leader);
            rank[q] = base + __popc(peers & lanemask_lt());
        }
        if (lev[q] < 0) continue;
        s_skip[i] = w[q].x - j0;
        s_in[i] = 0;
        s_oct[i] = lev[q] == 0 ? 0 : (uint8_t)((key[q] >> (3 * (kMaxLevel - lev[q]))) & 7u);
        s_sys[i] = (uint16_t)system_of(ss, w[q].y);
        if (w[q].z > 1) {  // a level-21 bucket
            D4 sm = {0.0, 0.0, 0.0, 0.0};
            for (int p = w[q].y; p < w[q].y + w[q].z; ++p) {
                const D4 b = sbody64[p];
                sm.x += b.w * b.x;
                sm.y += b.w * b.y;
                sm.z += b.w * b.z;
                sm.w += b.w;
            }
            s_sum[i] = sm;
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
#pragma unroll
    for (int q = 0; q < kSubPer; ++q) {
        const int i = threadIdx.x + q * kSubThreads;
        if (w[q].z == 1) {
            D4 &r = s_sum[i];
            const D4 b = r;
            D4 sm = {0.0, 0.0, 0.0, 0.0};
            sm.x += b.w * b.x;
            sm.y += b.w * b.y;
            sm.z += b.w * b.z;
            sm.w += b.w;
            r = sm;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int l = kMaxLevel - 1; l >= 0; --l) {
            s_start[l] = acc;
            acc += s_cnt[l];
        }
        s_start[kMaxLevel] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSubPer; ++q)
        if (lev[q] >= 0 && w[q].z == 0)
            s_list[s_start[lev[q]] + rank[q]] = (uint16_t)(threadIdx.x + q * kSubThreads);
    __syncthreads();
    // cells whose subtree ends in the tile, deepest level first: children one level deeper are
    // done; a cell has at most 8 children (the bound also ends a malformed skip chain)
    for (int l = kMaxLevel - 1; l >= 0; --l) {
        const int e = s_start[l] + s_cnt[l];
        if (s_cnt[l] == 0) continue;  // the same for the whole block
        for (int t = s_start[l] + threadIdx.x; t < e; t += kSubThreads) {
            const int i = s_list[t];
            const int sk = s_skip[i];
            if (sk > kSubT) continue;  // spine cell: later
            D4 sm = {0.0, 0.0, 0.0, 0.0};
            unsigned m = 0;
            int k = 0;
            for (int c = i + 1; c < sk && k < 8; c = max(s_skip[c], c + 1), ++k) {
                const D4 r = s_sum[c];
                sm.x += r.x;
                sm.y += r.y;
                sm.z += r.z;
                sm.w += r.w;
                m |= 1u << s_oct[c];
                s_in[c] = 1;
            }
            s_sum[i] = sm;
            s_mask[i] = (uint8_t)m;
        }
        __syncthreads();
    }
    // centres of mass of the cells finished here (all lanes busy), with their FP64 sums
    for (int t = threadIdx.x; t < s_start[kMaxLevel]; t += kSubThreads) {
        const int i = s_list[t];
        if (s_skip[i] > kSubT) continue;
        const int b = na.order[j0 + i];
        const D4 sm = s_sum[i];
        if (all_sums || !s_in[i]) na.com_lo[b] = sm;
        reinterpret_cast<float4 *>(gn + b)[0] = com32_from_sums(sm, box + s_sys[i], G);
    }
    // the rest of every record: the loads of all four nodes first
    int b[kSubPer], nxt[kSubPer];
    float4 c1[kSubPer];
#pragma unroll
    for (int q = 0; q < kSubPer; ++q) {
        const int j = j0 + threadIdx.x + q * kSubThreads;
        b[q] = 0;
        nxt[q] = 0;
        c1[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lev[q] >= 0) {
            b[q] = na.order[j];
            if (w[q].z == 0) nxt[q] = na.order[j + 1];
            if (w[q].z == 1) c1[q] = sbody32[w[q].y];
        }
    }
#pragma unroll
    for (int q = 0; q < kSubPer; ++q) {
        const int i = threadIdx.x + q * kSubThreads;
        const int j = j0 + i;
        if (lev[q] < 0) continue;
        const int k = s_sys[i];
        if (w[q].z != 0) {
            const D4 sm = s_sum[i];
            GroupNode g;
            g.c = w[q].z == 1 ? c1[q] : com32_from_sums(sm, box + k, G);
            g.child = w[q].y;
            g.n = -w[q].z;
            g.crit = 0.f;
            g.pre = j;
            gn[b[q]] = g;
            if (all_sums || !s_in[i]) na.com_lo[b[q]] = sm;
            na.mask[j] = 0;
        } else {
            unsigned m;
            if (w[q].x <= j0 + kSubT) {
                m = s_mask[i];
            } else {
                // a spine cell: its children's octants, past the tile from the keys
                const int shift = 3 * (kMaxLevel - 1 - lev[q]);
                m = 0;
                int k8 = 0;
                for (int c = j + 1; c < w[q].x && k8 < 8; ++k8) {
                    int nc;
                    if (c < j0 + kSubT) {
                        nc = s_skip[c - j0] + j0;
                        m |= 1u << s_oct[c - j0];
                    } else {
                        const int2 v = reinterpret_cast<const int2 *>(na.wn + c)[2];  // skip, first
                        nc = v.x;
                        m |= 1u << (unsigned)((keys[v.y] >> shift) & 7u);
                    }
                    c = max(nc, c + 1);
                }
                s_spine[lev[q]] = make_int4(b[q], nxt[q], __popc(m), k);
            }
            reinterpret_cast<int4 *>(gn + b[q])[1] =
                make_int4(nxt[q], __popc(m), __float_as_int(tab[k].crit32[lev[q]]), j);
            na.mask[j] = (uint8_t)m;
        }
    }
    __syncthreads();
    if (threadIdx.x < kMaxLevel && tile < tiles) spine[threadIdx.x * tiles + tile] = s_spine[threadIdx.x];
}

// The spine cells of one level (one per tile at most): sums of their children (finished by
// subtree_sums_kernel or by this kernel at a deeper level) in octant order, and the centre of
// mass of their record.  Launched for the levels from the deepest up to the roots.
__global__ void spine_sums_kernel(int level, NodeArrays na, const Box *__restrict__ box, double G,
                                  GroupNode *__restrict__ gn, const int4 *__restrict__ spine,
                                  int tiles)
{
    const int n_nodes = (int)min((int64_t)*na.d_nn, na.cap);
    const int used = min(tiles, (n_nodes + kSubT - 1) / kSubT);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < used; t += gridDim.x * blockDim.x) {
        const int4 e = spine[level * tiles + t];  // (level-order index, first child, count, system)
        if (e.x < 0) continue;
        const int nc = min(e.z, 8);
        D4 q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < nc) q[k] = ld_cg(&na.com_lo[e.y + k]);
        D4 sm = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k < nc) {
                sm.x += q[k].x;
                sm.y += q[k].y;
                sm.z += q[k].z;
                sm.w += q[k].w;
            }
        }
        na.com_lo[e.x] = sm;
        reinterpret_cast<float4 *>(gn + e.x)[0] = com32_from_sums(sm, box + e.w, G);
    }
}

// ------------------------------------------------------------------------------------------
// Level-order copy of the tree for the group walk.  A stable partition of the pre-order nodes by
// level: within a level the nodes keep their pre-order (Morton) order, so the children of a
// cell, which are consecutive among the nodes of the next level, get consecutive indices.
// ------------------------------------------------------------------------------------------

constexpr int kLayThreads = 256;
constexpr int kLayWarps = kLayThreads / 32;
constexpr int kLayRounds = 16;
constexpr int kLayTile = kLayThreads * kLayRounds;  // nodes per tile
constexpr unsigned kNoLevel = 0xffu;

// Per tile: the number of nodes of every level, stored level-major (counts[l * tiles + t]) so
// that one exclusive scan gives every (level, tile) its first output index.
__global__ void __launch_bounds__(kLayThreads) level_tile_count_kernel(
    const uint8_t *__restrict__ level, const uint32_t *__restrict__ d_nn, int64_t cap, int tiles,
    uint32_t *counts)
{
    const int n_nodes = (int)min((int64_t)*d_nn, cap);
    __shared__ unsigned h[kLevels];
    if (threadIdx.x < kLevels) h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kLayTile;
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < kLayRounds; ++r) {
        const int j = base + r * kLayThreads + threadIdx.x;
        const unsigned l = j < n_nodes ? (unsigned)level[j] : kNoLevel;
        const unsigned peers = __match_any_sync(kFull, l);
        if (l < (unsigned)kLevels && lane == __ffs(peers) - 1) atomicAdd(&h[l], (unsigned)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < kLevels) counts[threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[kLevels * tiles] = 0;  // scans to the total
}

// Level-order index of every node: its (level, tile) offset plus its rank among the nodes of
// the same level earlier in the tile.
__global__ void __launch_bounds__(kLayThreads) level_tile_rank_kernel(
    const uint8_t *__restrict__ level, const uint32_t *__restrict__ d_nn, int64_t cap, int tiles,
    const uint32_t *__restrict__ offs, int *order, int *inv)
{
    const int n_nodes = (int)min((int64_t)*d_nn, cap);
    __shared__ unsigned run[kLevels];
    __shared__ unsigned wc[kLayWarps][kLevels];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x < kLevels) run[threadIdx.x] = offs[threadIdx.x * tiles + blockIdx.x];
    const int base = blockIdx.x * kLayTile;
    for (int r = 0; r < kLayRounds; ++r) {
        if (threadIdx.x < kLayWarps * kLevels) (&wc[0][0])[threadIdx.x] = 0;
        __syncthreads();
        const int j = base + r * kLayThreads + threadIdx.x;
        const unsigned l = j < n_nodes ? (unsigned)level[j] : kNoLevel;
        const unsigned peers = __match_any_sync(kFull, l);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (l < (unsigned)kLevels && lane == __ffs(peers) - 1) wc[wid][l] = (unsigned)__popc(peers);
        __syncthreads();
        if (l < (unsigned)kLevels) {
            unsigned o = run[l] + rank;
            for (int w = 0; w < wid; ++w) o += wc[w][l];
            order[j] = (int)o;
            inv[o] = j;
        }
        __syncthreads();
        if (threadIdx.x < kLevels) {
            unsigned t = 0;
            for (int w = 0; w < kLayWarps; ++w) t += wc[w][threadIdx.x];
            run[threadIdx.x] += t;
        }
        __syncthreads();
    }
}

// GroupNode records at their level-order positions.  The first child of an internal cell is
// the next node in pre-order; its children count is the population of the child mask.
// The level-order copy the FP32 walk reads.  Leaves keep the FP32 (x - c, y - c, z - c, G m)
// link_leaves wrote; a cell's is made here from its FP64 moments (off the FP64-bound moment
// pass), with its level's FP32 acceptance threshold.
__global__ void group_nodes_kernel(const uint32_t *__restrict__ d_nn, int64_t cap,
                                   const WalkNode *__restrict__ wn, const D4 *__restrict__ com64,
                                   const uint8_t *__restrict__ level,
                                   const uint8_t *__restrict__ mask, const int *__restrict__ order,
                                   const Box *__restrict__ box,
                                   const LevelTables *__restrict__ tab, Systems ss, double G,
                                   GroupNode *gn)
{
    const int n_nodes = (int)min((int64_t)*d_nn, cap);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_nodes; j += gridDim.x * blockDim.x) {
        const WalkNode w = wn[j];
        GroupNode g;
        g.pre = j;
        if (w.count != 0) {
            g.c = w.c;
            g.child = w.first;
            g.n = -w.count;
            g.crit = 0.f;
        } else {
            const D4 m = com64[j];
            const int k = system_of(ss, w.first);
            const Box *bx = box + k;
            g.c = make_float4((float)(m.x - bx->c[0]), (float)(m.y - bx->c[1]),
                              (float)(m.z - bx->c[2]), (float)(G * m.w));
            g.child = j + 1 < n_nodes ? order[j + 1] : n_nodes;  // out of range: the walk refuses it
            g.n = max(1, __popc((unsigned)mask[j]));
            g.crit = tab[k].crit32[level[j]];
        }
        gn[order[j]] = g;
    }
}

// Walk groups that follow the tree (see launch_cell_groups).  A cell of more than gmax bodies
// hands out its children: runs of consecutive small children merged up to gmax bodies, large
// buckets in chunks; a root of at most gmax bodies is one group.  Every body lands in exactly one
// group: the largest cell around it with at most gmax bodies is a child of a larger cell (or the
// root), and a body in no such cell sits in a bucket larger than gmax.
__device__ __forceinline__ void put_group(int4 *groups, unsigned *ngroups, int64_t cap, int *err,
                                          int first, int count, int sys)
{
    const unsigned k = atomicAdd(ngroups, 1u);
    if ((int64_t)k < cap) groups[k] = make_int4(first, count, sys, 0);
    else atomicOr(err, kErrNodeCap);
}

__global__ void cell_groups_kernel(NodeArrays na, const uint32_t *__restrict__ node_off,
                                   Systems ss, int n, int gmax, int4 *groups, unsigned *ngroups,
                                   int64_t cap, int *err)
{
    const int nn = (int)min((int64_t)*na.d_nn, na.cap);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nn; j += gridDim.x * blockDim.x) {
        const WalkNode w = na.wn[j];
        const int sy = system_of(ss, w.first);
        const int bend = ss.sys ? ss.start[sy + 1] : n;            // system's body end
        const int nend = ss.sys ? min((int)node_off[ss.start[sy + 1]], nn) : nn;  // node end
        const int cnt = w.count != 0 ? w.count
                                     : (w.skip < nend ? na.wn[w.skip].first : bend) - w.first;
        if (na.level[j] == 0 && cnt <= gmax) {
            put_group(groups, ngroups, cap, err, w.first, cnt, sy);
            continue;
        }
        if (w.count != 0 || cnt <= gmax) continue;  // handled by the parent
        int cf = 0, cc = 0;
        int k = 0;
        for (int c = j + 1; c < w.skip && k < 8; c = max(na.wn[c].skip, c + 1), ++k) {
            const WalkNode wc = na.wn[c];
            const int ccnt = wc.count != 0
                                 ? wc.count
                                 : (wc.skip < nend ? na.wn[wc.skip].first : bend) - wc.first;
            if (ccnt > gmax) {
                if (cc) put_group(groups, ngroups, cap, err, cf, cc, sy);
                cc = 0;
                if (wc.count != 0)  // a bucket of more than gmax bodies: chunks of gmax
                    for (int b = 0; b < ccnt; b += gmax)
                        put_group(groups, ngroups, cap, err, wc.first + b, min(gmax, ccnt - b), sy);
                continue;
            }
            if (cc && cc + ccnt > gmax) {
                put_group(groups, ngroups, cap, err, cf, cc, sy);
                cc = 0;
            }
            if (cc == 0) cf = wc.first;
            cc += ccnt;
        }
        if (cc) put_group(groups, ngroups, cap, err, cf, cc, sy);
    }
}

// Forest: level-order index of the root of every non-empty system (its first pre-order node).
__global__ void roots_kernel(const uint32_t *__restrict__ node_off, Systems ss,
                             const uint32_t *__restrict__ d_nn, const int *__restrict__ order,
                             int *roots)
{
    const uint32_t nn = *d_nn;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ss.count; k += gridDim.x * blockDim.x) {
        const uint32_t r = node_off[ss.start[k]];
        roots[k] = (ss.start[k + 1] > ss.start[k] && r < nn) ? order[r] : -1;
    }
}

// Forest: the node count the other kernels use.  A tree larger than the node arrays is not
// built at all (count 0, kErrNodeCap), so no kernel ever reads or writes past them.
__global__ void clamp_count_kernel(const uint32_t *__restrict__ total, int64_t cap, uint32_t *nn,
                                   int *err)
{
    const uint32_t t = *total;
    if ((int64_t)t > cap) {
        *nn = 0u;
        atomicOr(err, kErrNodeCap);
    } else {
        *nn = t;
    }
}

// ------------------------------------------------------------------------------------------
// Generic exclusive scan of uint32 (reduce -> spine -> downsweep).
// ------------------------------------------------------------------------------------------

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *__restrict__ in,
                                                                  int len, uint32_t *block_sums)
{
    const int base = blockIdx.x * kScanTile;
    uint32_t s = 0;
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
        const int i = base + k;
        if (i < len) s += in[i];
    }
    uint32_t tot;
    (void)block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) scan_spine_kernel(uint32_t *block_sums, int nb)
{
    uint32_t carry = 0;
    for (int t0 = 0; t0 < nb; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const uint32_t v = t < nb ? block_sums[t] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, &tot);
        if (t < nb) block_sums[t] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) block_sums[nb] = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const uint32_t *__restrict__ in,
                                                                uint32_t *__restrict__ out, int len,
                                                                const uint32_t *__restrict__ block_sums)
{
    __shared__ uint32_t tile[kScanTile];
    const int base = blockIdx.x * kScanTile;
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
        const int i = base + k;
        tile[k] = i < len ? in[i] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        v[r] = tile[threadIdx.x * kScanItems + r];
        s += v[r];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(s, &tot) + block_sums[blockIdx.x];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        tile[threadIdx.x * kScanItems + r] = run;
        run += v[r];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
        const int i = base + k;
        if (i < len) out[i] = tile[k];
    }
}

inline int grid_for(int64_t n, int threads, int max_blocks)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

constexpr int kMaxGrid = 152 * 16;

}  // namespace

// ---------------------------------------------------------------- launchers

namespace {
std::atomic<int64_t> g_launches{0};
}

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

int bbox_blocks(int64_t n) { return grid_for(n, kBoxThreads * 4, 152 * 8); }
int bbox_partial_doubles() { return kPart; }

void launch_bbox_partials(const double *pos, const double *mass, int n, double *partials, int nblk,
                          D4 *aos, cudaStream_t s)
{
    bbox_partials_kernel<<<nblk, kBoxThreads, 0, s>>>(pos, mass, n, partials, aos);
    count_launches(1);
}

void launch_kick_drift_bbox(double *pos, double *vel, const double *acc, const double *mass, int n,
                            double h, double dt, double *partials, int nblk, D4 *aos, bool fused,
                            cudaStream_t s)
{
    if (fused)
        kick_drift_bbox_kernel<true><<<nblk, kBoxThreads, 0, s>>>(pos, vel, acc, mass, n, h, dt,
                                                                  partials, aos);
    else
        kick_drift_bbox_kernel<false><<<nblk, kBoxThreads, 0, s>>>(pos, vel, acc, mass, n, h, dt,
                                                                   partials, aos);
    count_launches(1);
}

void launch_bbox_finalize(const double *partials, int nblk, Box *box, LevelTables *tab,
                          double theta, cudaStream_t s)
{
    bbox_finalize_kernel<<<1, kBoxThreads, 0, s>>>(partials, nblk, box, tab, theta);
    count_launches(1);
}

void launch_forest_boxes(double *pos, double *vel, const double *acc, const double *mass, int n,
                         const int4 *chunks, int nchunks, const int *chunk_start, int n_sys,
                         double h, double dt, double *partials, Box *box, LevelTables *tab,
                         double theta, D4 *aos, bool fused, cudaStream_t s)
{
    if (nchunks > 0 && fused)
        forest_box_partials_kernel<true><<<nchunks, kBoxThreads, 0, s>>>(
            pos, vel, acc, mass, n, chunks, h, dt, partials, aos);
    else if (nchunks > 0)
        forest_box_partials_kernel<false><<<nchunks, kBoxThreads, 0, s>>>(
            pos, vel, acc, mass, n, chunks, h, dt, partials, aos);
    forest_box_finalize_kernel<<<n_sys, kBoxThreads, 0, s>>>(partials, chunk_start, box, tab,
                                                             theta);
    count_launches(nchunks > 0 ? 2 : 1);
}

void launch_keys(const double *pos, int n, const Box *box, const Systems &ss, uint64_t *keys,
                 uint32_t *ids, cudaStream_t s, const int *gate)
{
    keys_kernel<<<grid_for(n, 256, kMaxGrid), 256, 0, s>>>(pos, n, box, ss, keys, ids, gate);
    count_launches(1);
}

int sort_tiles(int n) { return (n + kSortTile - 1) / kSortTile; }

cudaError_t sort_prepare()
{
    const void *fns[3] = {(const void *)radix_downsweep_kernel<kDigitKey>,
                          (const void *)radix_downsweep_kernel<kDigitSys>,
                          (const void *)radix_downsweep_kernel<kDigitId>};
    for (const void *f : fns) {
        const cudaError_t e =
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDownSmem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {

// The digit passes of one sort: `id_passes` passes on id bytes, the 8 key passes, then (forest)
// the system passes; the result ends in (keys, ids) or (keys_alt, ids_alt) by the parity of the
// pass count.  With sc.sys and no sc.sys_hist the system digit totals come from the data (a
// subset of a forest's bodies).
void radix_passes(uint64_t *keys, uint32_t *ids, int n, int id_passes, const SortScratch &sc,
                  cudaStream_t s, uint64_t **out_keys, uint32_t **out_ids)
{
    const int tiles = sort_tiles(n);
    const bool sys_data = sc.sys && !sc.sys_hist;
    const int rows = sys_data ? kHistRows : kPasses + id_passes;
    cudaMemsetAsync(sc.hist, 0, sizeof(uint32_t) * rows * 256, s);
    radix_hist_kernel<<<grid_for(n, kSortThreads * 8, 152 * 4), kSortThreads, 0, s>>>(
        keys, ids, n, sc.d_n, id_passes, sys_data ? sc.sys : nullptr, sc.hist);
    uint64_t *kin = keys, *kout = sc.keys_alt;
    uint32_t *iin = ids, *iout = sc.ids_alt;
    const int sys_passes = sc.sys ? kSysPasses : 0;
    const int passes = id_passes + kPasses + sys_passes;
    for (int p = 0; p < passes; ++p) {
        const int mode = p < id_passes ? kDigitId : (p < id_passes + kPasses ? kDigitKey : kDigitSys);
        int shift;
        const uint32_t *hist;
        if (mode == kDigitId) {
            shift = 8 * p;
            hist = sc.hist + 256 * (kPasses + p);
        } else if (mode == kDigitKey) {
            shift = 8 * (p - id_passes);
            hist = sc.hist + 256 * (p - id_passes);
        } else {
            const int q = p - id_passes - kPasses;
            shift = 8 * q;
            hist = sys_data ? sc.hist + 256 * (kPasses + kIdPasses + q) : sc.sys_hist + 256 * q;
        }
        if (mode == kDigitId)
            radix_upsweep_kernel<kDigitId><<<tiles, kSortThreads, 0, s>>>(
                kin, iin, n, sc.d_n, shift, sc.counts, tiles, nullptr);
        else if (mode == kDigitKey)
            radix_upsweep_kernel<kDigitKey><<<tiles, kSortThreads, 0, s>>>(
                kin, iin, n, sc.d_n, shift, sc.counts, tiles, nullptr);
        else
            radix_upsweep_kernel<kDigitSys><<<tiles, kSortThreads, 0, s>>>(
                kin, iin, n, sc.d_n, shift, sc.counts, tiles, sc.sys);
        radix_rowscan_kernel<<<256, kSortThreads, 0, s>>>(sc.counts, tiles, n, sc.d_n, hist);
        if (mode == kDigitId)
            radix_downsweep_kernel<kDigitId><<<tiles, kSortThreads, kDownSmem, s>>>(
                kin, iin, kout, iout, n, sc.d_n, shift, sc.counts, tiles, nullptr);
        else if (mode == kDigitKey)
            radix_downsweep_kernel<kDigitKey><<<tiles, kSortThreads, kDownSmem, s>>>(
                kin, iin, kout, iout, n, sc.d_n, shift, sc.counts, tiles, nullptr);
        else
            radix_downsweep_kernel<kDigitSys><<<tiles, kSortThreads, kDownSmem, s>>>(
                kin, iin, kout, iout, n, sc.d_n, shift, sc.counts, tiles, sc.sys);
        uint64_t *tk = kin; kin = kout; kout = tk;
        uint32_t *ti = iin; iin = iout; iout = ti;
    }
    count_launches(1 + 3 * passes);
    *out_keys = kin;
    *out_ids = iin;
}

}  // namespace

void launch_radix_sort(uint64_t *keys, uint32_t *ids, int n, const SortScratch &sc, cudaStream_t s)
{
    if (n <= 1) return;
    uint64_t *k;
    uint32_t *i;
    // an even number of passes (8, or 8 + 2) leaves the result in the caller's buffers
    radix_passes(keys, ids, n, 0, sc, s, &k, &i);
}

void launch_radix_sort_key_id(uint64_t *keys, uint32_t *ids, int n, int id_bits,
                              const SortScratch &sc, cudaStream_t s, uint64_t **out_keys,
                              uint32_t **out_ids)
{
    *out_keys = keys;
    *out_ids = ids;
    if (n <= 1) return;
    const int id_passes = std::min(kIdPasses, std::max(1, (id_bits + 7) / 8));
    radix_passes(keys, ids, n, id_passes, sc, s, out_keys, out_ids);
}

__global__ void check_finite_kernel(const double *__restrict__ pos,
                                    const double *__restrict__ mass, int n, int *flag)
{
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        bad = bad || !isfinite(pos[i]) || !isfinite(pos[(size_t)n + i]) ||
              !isfinite(pos[2 * (size_t)n + i]) || !isfinite(mass[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, kErrInput);
}

void launch_check_finite(const double *pos, const double *mass, int n, int *flag, cudaStream_t s)
{
    if (n <= 0) return;
    check_finite_kernel<<<std::min((n + 255) / 256, 152 * 8), 256, 0, s>>>(pos, mass, n, flag);
    count_launches(1);
}

void launch_permute(const D4 *aos, const uint32_t *ids, int n, const Box *box, const Systems &ss,
                    double G, D4 *sbody64, float4 *sbody32, cudaStream_t s)
{
    permute_kernel<<<grid_for(n, 256, kMaxGrid), 256, 0, s>>>(aos, ids, n, box, ss, G, sbody64,
                                                              sbody32);
    count_launches(1);
}

int scan_tiles(int len) { return (len + kScanTile - 1) / kScanTile; }

void launch_count_nodes(const uint64_t *keys, int n, const Systems &ss, uint32_t *counts,
                        unsigned *max_level, cudaStream_t s)
{
    count_nodes_kernel<<<grid_for((int64_t)n + 1, 256, kMaxGrid), 256, 0, s>>>(keys, n, ss, counts,
                                                                              max_level);
    count_launches(1);
}

void launch_exclusive_scan(const uint32_t *in, uint32_t *out, int len, const ScanScratch &sc,
                           cudaStream_t s)
{
    const int nb = scan_tiles(len);
    scan_reduce_kernel<<<nb, kScanThreads, 0, s>>>(in, len, sc.block_sums);
    scan_spine_kernel<<<1, 1024, 0, s>>>(sc.block_sums, nb);
    scan_down_kernel<<<nb, kScanThreads, 0, s>>>(in, out, len, sc.block_sums);
    count_launches(3);
}

void launch_emit_nodes(const uint64_t *keys, int n, const Systems &ss, const uint32_t *node_off,
                       NodeArrays na, int *err, cudaStream_t s)
{
    emit_nodes_kernel<<<grid_for(n, 128, kMaxGrid * 4), 128, 0, s>>>(keys, n, ss, node_off, na,
                                                                     err);
    count_launches(1);
}

int layout_tiles(int64_t n_nodes) { return (int)((n_nodes + kLayTile - 1) / kLayTile); }
int layout_scan_len(int64_t n_nodes) { return kLevels * layout_tiles(n_nodes) + 1; }

void launch_level_order(const NodeArrays &na, cudaStream_t s)
{
    const int tiles = na.tiles;
    const int len = kLevels * tiles + 1;
    level_tile_count_kernel<<<tiles, kLayThreads, 0, s>>>(na.level, na.d_nn, na.cap, tiles,
                                                          na.tile_offsets);
    ScanScratch ss{na.block_sums, scan_tiles(len)};
    launch_exclusive_scan(na.tile_offsets, na.tile_offsets, len, ss, s);
    level_tile_rank_kernel<<<tiles, kLayThreads, 0, s>>>(na.level, na.d_nn, na.cap, tiles,
                                                         na.tile_offsets, na.order, na.inv);
    count_launches(2);
}

void launch_moments(const uint64_t *keys, int max_level, const D4 *sbody64, const Box *box,
                    const LevelTables *tab, const Systems &ss, double G, NodeArrays na,
                    cudaStream_t s)
{
    const int64_t cap = na.cap;
    link_leaves_kernel<<<grid_for(cap, 256, kMaxGrid * 4), 256, 0, s>>>(keys, na, sbody64, box, ss,
                                                                       G);
    const int depth = min(max_level, kMaxLevel);
    for (int lev = depth - 1; lev >= 0; --lev) {
        // a level's node count is only known on the device: a grid for the widest level it can
        // have (8^lev cells per system) and a grid-stride loop over the level's range
        const int64_t widest = lev < 10 ? ((int64_t)ss.count << (3 * lev)) : cap;
        const int g = grid_for(std::min<int64_t>(widest, cap), 256, kMaxGrid * 2);
        moments_level_kernel<<<g, 256, 0, s>>>(lev, na, G);
    }
    count_launches(1 + max(0, depth));
}

int subtree_tiles(int64_t cap)
{
    return (int)((std::max<int64_t>(cap, 1) + kSubT - 1) / kSubT);
}

void launch_subtree_sums(const uint64_t *keys, int max_level, const D4 *sbody64,
                         const float4 *sbody32, const Box *box, const LevelTables *tab,
                         const Systems &ss, double G, NodeArrays na, GroupNode *gn,
                         bool all_sums, cudaStream_t s)
{
    const int tiles = subtree_tiles(na.cap);
    subtree_sums_kernel<<<tiles, kSubThreads, 0, s>>>(keys, na, sbody64, sbody32, box, tab, ss, G,
                                                      gn, na.spine, tiles, all_sums ? 1 : 0);
    const int depth = min(max_level, kMaxLevel);
    const int g = grid_for(tiles, 256, kMaxGrid);
    for (int lev = depth - 1; lev >= 0; --lev)
        spine_sums_kernel<<<g, 256, 0, s>>>(lev, na, box, G, gn, na.spine, tiles);
    count_launches(1 + max(0, depth));
}

void launch_group_nodes(const NodeArrays &na, const Box *box, const LevelTables *tab,
                        const Systems &ss, double G, GroupNode *gn, cudaStream_t s)
{
    group_nodes_kernel<<<grid_for(na.cap, 256, kMaxGrid * 4), 256, 0, s>>>(
        na.d_nn, na.cap, na.wn, na.com64, na.level, na.mask, na.order, box, tab, ss, G, gn);
    count_launches(1);
}

void launch_roots(const NodeArrays &na, const uint32_t *node_off, const Systems &ss, int *roots,
                  cudaStream_t s)
{
    roots_kernel<<<grid_for(ss.count, 256, kMaxGrid), 256, 0, s>>>(node_off, ss, na.d_nn, na.order,
                                                                   roots);
    count_launches(1);
}

void launch_cell_groups(const NodeArrays &na, const uint32_t *node_off, const Systems &ss, int n,
                        int gmax, int4 *groups, unsigned *ngroups, int64_t cap, int *err,
                        cudaStream_t s)
{
    cell_groups_kernel<<<grid_for(na.cap, 256, kMaxGrid * 4), 256, 0, s>>>(na, node_off, ss, n, gmax,
                                                                          groups, ngroups, cap,
                                                                          err);
    count_launches(1);
}

void launch_clamp_count(const uint32_t *total, int64_t cap, uint32_t *nn, int *err, cudaStream_t s)
{
    clamp_count_kernel<<<1, 1, 0, s>>>(total, cap, nn, err);
    count_launches(1);
}

}  // namespace nb

// C ABI of the Barnes-Hut timestep library: context, build / force / step entry points and
// introspection.  Every step of the method runs in the kernels of build_kernels.cu and
// walk_kernels.cu; this file only allocates, orders launches on the context stream and copies.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "nbody_internal.cuh"

using namespace nb;

struct nbody_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    nbody_params p{};
    int64_t cap = 0;

    // per-body working set (capacity `cap`)
    uint64_t *keys = nullptr, *keys_alt = nullptr;
    uint32_t *ids = nullptr, *ids_alt = nullptr;
    D4 *sbody64 = nullptr;
    D4 *aos = nullptr;              // (x, y, z, m) records in the caller's order
    float4 *sbody32 = nullptr;
    uint32_t *node_off = nullptr;   // cap + 1
    uint32_t *hist = nullptr;       // 14 x 256
    uint32_t *counts = nullptr;     // 256 x sort tiles
    uint32_t *block_sums = nullptr; // scan tiles + 1
    double *partials = nullptr;     // bbox_partial_doubles() x bbox blocks
    int nblk = 0;
    Box *box = nullptr;             // [0] last build, [1] direct sum
    LevelTables *tab = nullptr;     // [0] last build, [1] direct sum
    double *acc = nullptr;          // 3 x cap: a^(k) kept between steps
    uint32_t *pp = nullptr, *pc = nullptr;
    int *err = nullptr;             // device error word
    uint32_t *h_word = nullptr;     // pinned host words: node count, deepest level, then the
                                    // re-sort's stats (kOrderStats words from h_word + 2)
    unsigned *info = nullptr;       // device word: deepest node level of the last build

    // octree
    NodeArrays na{};
    int64_t n_nodes = 0;
    GroupNode *gn = nullptr;        // level-order copy for the FP32 group walk (capacity na.cap)
    // quadrupoles (NBODY_FLAG_QUADRUPOLE), capacity quad_cap nodes
    double *q_lo = nullptr, *q64 = nullptr;
    float4 *gq = nullptr;
    int64_t quad_cap = 0;

    // forest (n_sys > 0): systems packed in one set of arrays
    int n_sys = 0;
    uint16_t *sys = nullptr;        // system of every body
    int *sys_start = nullptr;       // n_sys + 1 body offsets
    uint32_t *sys_hist = nullptr;   // digit totals of the two system sort passes
    int4 *groups = nullptr;         // walk groups: (first body, count, system, 0)
    int n_groups = 0;
    int *roots = nullptr;           // level-order root of every system
    int4 *box_chunks = nullptr;     // (first body, end, system) chunks for the per-system boxes
    int *box_chunk_start = nullptr; // n_sys + 1: first chunk of every system
    int n_box_chunks = 0;
    double *box_partials = nullptr; // partial boxes, one per chunk
    uint32_t *nn = nullptr;         // node count the forest's kernels use (device)
    // walk groups that follow the tree's cells (FP32 walks with NBODY_FLAG_CELL_GROUPS or
    // NBODY_FLAG_GROUP_MAC), rebuilt on the device with every tree
    int4 *cgroups = nullptr;
    unsigned *cgroups_n = nullptr;
    unsigned *work = nullptr;       // group counter of the persistent FP32 walk
    // the shared far walk of 256-body spans (single systems, FP32 per-body walk), allocated on
    // first use: per-span lists (span_meta, span_off, span_pool) and per-warp scratch
    int4 *span_meta = nullptr;
    uint32_t *span_off = nullptr, *span_pool = nullptr, *span_tmp = nullptr;
    unsigned *span_next = nullptr;
    int64_t span_n = 0, span_pool_cap = 0, span_tmp_warps = 0;
    // walk limits (nbody_set_walk_limits; the defaults never bind) and the finite-input check
    int stack_limit = 1 << 30;
    int64_t step_limit = INT64_MAX;
    int fast_stack_limit = 1 << 30;
    int4 *overflow = nullptr;       // FP32 per-body walk: groups handed to the full-stack walk
    unsigned *n_overflow = nullptr;
    int64_t overflow_cap = 0;
    int *chk = nullptr;             // device word: kErrInput when NBODY_FLAG_CHECK_FINITE fails
    float *dscratch = nullptr;      // FP32 direct sum: sources + partial sums (grown on demand)
    int64_t dscratch_cap = 0;       // floats
    // one forest step captured as a CUDA graph, replayed on its own stream
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void *gkey[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t glaunches = 0;          // kernels per replayed step
    cudaEvent_t gev[2] = {};

    // re-sort from the previous order (allocated on first use, capacity ord_cap bodies)
    OrderScratch ord{};
    int64_t ord_cap = 0;
    int sort_mode = NBODY_SORT_AUTO;
    int64_t order_n = -1;       // c->ids holds the sorted order of the last build of this n
    int last_sort_path = -1;    // 0 full sort, 2 re-sort tried (the device's choice in ord.stats),
                                // -1 no build yet

    // launch shape of the walk per precision class (FP32 forms, FP64): set by nbody_set_walk_shape
    // or by nbody_autotune, which also keeps its choice per (N bucket, theta) in shape_cache
    int shape32 = kDefaultWalkShape, shape64 = kDefaultWalkShape;
    struct ShapeChoice {
        int bucket;    // floor(log2(n))
        double theta;
        int shape;
    };
    std::vector<ShapeChoice> shape_cache;
    int forced_shape = -1;          // the autotuner's candidate while it times it

    // host-buffer stepping: device copies, and a side stream that reads the positions back while
    // the last step's tree and walk run
    double *hpos = nullptr, *hvel = nullptr, *hmass = nullptr;
    cudaStream_t xstream = nullptr;
    cudaEvent_t xdrift = nullptr;

    // state
    int64_t n_built = -1;       // n of the last build (-1: none)
    int64_t n_forces = -1;      // n of the last force evaluation (counters valid)
    int64_t acc_n = -1;         // n for which ctx->acc holds a^(k)
    bool timing = false;
    bool timing_pending = false;  // events of the last call not yet read
    cudaEvent_t ev[6] = {};
    float ms[5] = {0, 0, 0, 0, 0};
    char msg[256] = {0};
};

namespace {

nbody_status fail(nbody_ctx *c, nbody_status st, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(c, e_ == cudaErrorMemoryAllocation ? NBODY_ENOMEM : NBODY_ECUDA,      \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define CKS(expr)                        \
    do {                                 \
        nbody_status s_ = (expr);        \
        if (s_ != NBODY_OK) return s_;   \
    } while (0)

// FP32 walks over groups that follow the tree's cells (the grouped acceptance test needs them).
constexpr int kResortMinN = 1 << 16;  // NBODY_SORT_AUTO re-sorts from this many bodies

bool cell_groups(const nbody_ctx *c)
{
    return (c->p.flags & (NBODY_FLAG_GROUP_MAC | NBODY_FLAG_CELL_GROUPS)) != 0;
}

bool params_ok(const nbody_params *p)
{
    if (!p) return false;
    if (!isfinite(p->G) || !isfinite(p->dt)) return false;
    if (!(p->eps >= 0.0) || !isfinite(p->eps)) return false;
    if (!(p->theta >= 0.0) || !isfinite(p->theta)) return false;
    if (p->precision < NBODY_FP64 || p->precision > NBODY_FP64_FAST) return false;
    const uint32_t fp32_only = NBODY_FLAG_GROUP_MAC | NBODY_FLAG_CELL_GROUPS;
    if ((p->flags & ~(fp32_only | NBODY_FLAG_QUADRUPOLE | NBODY_FLAG_CHECK_FINITE)) != 0)
        return false;
    if ((p->flags & fp32_only) && is_fp64(p->precision)) return false;
    return true;
}

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * count);
}

template <class T>
void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void free_nodes(nbody_ctx *c)
{
    dfree(c->na.wn);
    dfree(c->na.com64);
    dfree(c->na.level);
    dfree(c->na.mask);
    dfree(c->na.kind);
    dfree(c->na.order);
    dfree(c->na.inv);
    dfree(c->na.com_lo);
    dfree(c->na.lo_child);
    dfree(c->na.spine);
    dfree(c->na.tile_offsets);
    dfree(c->na.block_sums);
    dfree(c->gn);
    dfree(c->q_lo);
    dfree(c->q64);
    dfree(c->gq);
    c->quad_cap = 0;
    c->na.q_lo = c->na.q64 = nullptr;
    c->na.gq = nullptr;
    c->na.cap = 0;
}

// Quadrupole arrays for the current node capacity when the flag asks for them (allocates only
// when the capacity grew: at creation, set_params or a larger tree, never inside a forest step).
nbody_status ensure_quad(nbody_ctx *c)
{
    const bool quad = (c->p.flags & NBODY_FLAG_QUADRUPOLE) != 0;
    if (quad && c->quad_cap < c->na.cap) {
        dfree(c->q_lo);
        dfree(c->q64);
        dfree(c->gq);
        c->quad_cap = 0;
        CK(dalloc(&c->q_lo, 6 * (size_t)c->na.cap));
        CK(dalloc(&c->q64, 6 * (size_t)c->na.cap));
        CK(dalloc(&c->gq, 2 * (size_t)c->na.cap));
        c->quad_cap = c->na.cap;
    }
    c->na.q_lo = quad ? c->q_lo : nullptr;
    c->na.q64 = quad ? c->q64 : nullptr;
    c->na.gq = quad ? c->gq : nullptr;
    return NBODY_OK;
}

nbody_status ensure_nodes(nbody_ctx *c, int64_t need)
{
    if (need <= c->na.cap) return NBODY_OK;
    free_nodes(c);
    const int64_t cap = std::max<int64_t>(need + need / 8, 1024);
    CK(dalloc(&c->na.wn, cap));
    CK(dalloc(&c->na.com64, cap));
    CK(dalloc(&c->na.level, cap));
    CK(dalloc(&c->na.mask, cap));
    CK(dalloc(&c->na.kind, cap));
    CK(dalloc(&c->na.order, cap));
    CK(dalloc(&c->na.inv, cap));
    CK(dalloc(&c->na.com_lo, cap));
    CK(dalloc(&c->na.lo_child, cap));
    CK(dalloc(&c->na.spine, (size_t)kMaxLevel * subtree_tiles(cap)));
    const int len = layout_scan_len(cap);
    CK(dalloc(&c->na.tile_offsets, (size_t)len));
    CK(dalloc(&c->na.block_sums, (size_t)scan_tiles(len) + 1));
    c->na.tiles = layout_tiles(cap);
    CK(dalloc(&c->gn, cap));
    c->na.cap = cap;
    return NBODY_OK;
}

void free_order(nbody_ctx *c)
{
    dfree(c->ord.keep);
    dfree(c->ord.ends);
    dfree(c->ord.seams);
    dfree(c->ord.kept_off);
    dfree(c->ord.stats);
    dfree(c->ord.split);
    dfree(c->ord.rk);
    dfree(c->ord.xk);
    dfree(c->ord.ri);
    dfree(c->ord.xi);
    c->ord_cap = 0;
}

// Scratch of the re-sort for the context's capacity (first use only).
nbody_status ensure_order(nbody_ctx *c)
{
    if (c->ord_cap >= c->cap && c->ord.keep) return NBODY_OK;
    free_order(c);
    const size_t cap = (size_t)std::max<int64_t>(c->cap, 1);
    const int tiles = order_tiles((int)cap);
    CK(dalloc(&c->ord.keep, (size_t)tiles * 64));
    CK(dalloc(&c->ord.ends, (size_t)tiles));
    CK(dalloc(&c->ord.seams, (size_t)(tiles + 31) / 32));
    CK(dalloc(&c->ord.kept_off, (size_t)tiles));
    CK(dalloc(&c->ord.stats, (size_t)kOrderStats));
    CK(dalloc(&c->ord.split, (size_t)order_merge_tiles((int)cap) + 1));
    CK(dalloc(&c->ord.rk, cap));
    CK(dalloc(&c->ord.xk, cap));
    CK(dalloc(&c->ord.ri, cap));
    CK(dalloc(&c->ord.xi, cap));
    c->ord_cap = (int64_t)cap;
    return NBODY_OK;
}

void free_spans(nbody_ctx *c)
{
    dfree(c->span_meta);
    dfree(c->span_off);
    dfree(c->span_pool);
    dfree(c->span_tmp);
    dfree(c->span_next);
    c->span_n = c->span_pool_cap = c->span_tmp_warps = 0;
}

// FP32 contexts without quadrupoles keep FP64 sums in the tree instead of FP64 means (the FP32
// walk reads FP32 centres of mass only); FP64 contexts and quadrupole terms keep the means.
bool sums_moments(const nbody_ctx *c)
{
    return !is_fp64(c->p.precision) && (c->p.flags & NBODY_FLAG_QUADRUPOLE) == 0;
}

// Whether the FP32 walk of this context runs the shared far walk of the spans: single systems
// with the per-body acceptance test and monopole cells.
bool use_spans(const nbody_ctx *c)
{
    return c->n_sys == 0 && !is_fp64(c->p.precision) &&
           (c->p.flags & (NBODY_FLAG_GROUP_MAC | NBODY_FLAG_CELL_GROUPS | NBODY_FLAG_QUADRUPOLE)) == 0;
}

// Whether launch shape k changes this context's walk (the autotuner times only those): FP64
// walks and the flagged FP32 forms take the warps (threads) per block of shapes 0..2; the
// per-body FP32 walk all shapes, less the spans in a forest or with cell-following groups.
bool shape_applies(const nbody_ctx *c, int k)
{
    if (k < 0 || k >= kWalkShapes) return false;
    if (k < 3) return true;
    if (is_fp64(c->p.precision)) return false;
    if (c->p.flags & (NBODY_FLAG_GROUP_MAC | NBODY_FLAG_QUADRUPOLE)) return false;
    if (c->n_sys || (c->p.flags & NBODY_FLAG_CELL_GROUPS)) return k == 6 || k == 7;
    return true;
}

int size_bucket(int64_t n)
{
    int b = 0;
    while (n > 1) {
        n >>= 1;
        ++b;
    }
    return b;
}

// The walk's launch shape for n bodies: the autotuner's candidate while it times one, else its
// choice for this (N bucket, theta), else the context's shape.
int walk_shape_for(const nbody_ctx *c, int64_t n)
{
    if (c->forced_shape >= 0) return c->forced_shape;
    const int b = size_bucket(n);
    for (const auto &e : c->shape_cache)
        if (e.bucket == b && e.theta == c->p.theta) return e.shape;
    return is_fp64(c->p.precision) ? c->shape64 : c->shape32;
}

// Groups that follow the tree's cells: the flags, or (per-body FP32 walks) the launch shape.
bool cell_groups_for(const nbody_ctx *c, int64_t n)
{
    if (is_fp64(c->p.precision)) return false;
    return cell_groups(c) || walk_shape32(walk_shape_for(c, n)).cell_groups;
}

// Span scratch for n bodies (grown on demand; never inside a captured forest step).  The pool
// holds the spans' far lists and frontiers: about 4 / theta^2 node indices per body (clamped to
// 8 .. 48), plenty at the benchmark's theta; a span that finds no room walks from the root.
nbody_status ensure_spans(nbody_ctx *c, int n)
{
    const int64_t spans = ((int64_t)n + kSpanMinBodies - 1) / kSpanMinBodies;
    const double th = std::max(c->p.theta, 0.05);
    const int64_t per_body = std::min<int64_t>(48, std::max<int64_t>(8, (int64_t)(4.0 / (th * th))));
    const int64_t pool = std::max<int64_t>(1024, per_body * n);
    const int64_t warps = span_far_warps(n, kSpanMinBodies);
    if (spans <= c->span_n && pool <= c->span_pool_cap && warps <= c->span_tmp_warps)
        return NBODY_OK;
    free_spans(c);
    CK(dalloc(&c->span_meta, (size_t)spans));
    CK(dalloc(&c->span_off, (size_t)spans));
    CK(dalloc(&c->span_pool, (size_t)pool));
    CK(dalloc(&c->span_tmp, (size_t)warps * (kSpanFarTmp + 2 * kSpanFrTmp)));
    CK(dalloc(&c->span_next, 2));
    c->span_n = spans;
    c->span_pool_cap = pool;
    c->span_tmp_warps = warps;
    return NBODY_OK;
}

// The FP32 per-body walk's overflow list: one entry per group of the capacity (first FP32 walk
// of a single system; forests at creation, since their steps may be captured).
nbody_status ensure_overflow(nbody_ctx *c)
{
    const int64_t need = c->n_sys ? (int64_t)c->n_groups : (c->cap + 31) / 32;
    if (is_fp64(c->p.precision) || (c->overflow && c->overflow_cap >= need)) return NBODY_OK;
    dfree(c->overflow);
    dfree(c->n_overflow);
    c->overflow_cap = 0;
    CK(dalloc(&c->overflow, (size_t)std::max<int64_t>(need, c->cap + 1)));
    CK(dalloc(&c->n_overflow, 1));
    c->overflow_cap = std::max<int64_t>(need, c->cap + 1);
    return NBODY_OK;
}

nbody_status check_launch(nbody_ctx *c, const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, NBODY_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return NBODY_OK;
}

nbody_status check_n(nbody_ctx *c, int64_t n)
{
    if (n < 0 || n > c->cap)
        return fail(c, NBODY_EINVAL, "n = %lld outside [0, capacity %lld]", (long long)n,
                    (long long)c->cap);
    return NBODY_OK;
}

void record(nbody_ctx *c, int k)
{
    if (c->timing) cudaEventRecord(c->ev[k], c->stream);
}

// Keys and sort of the bodies into c->keys / c->ids (keys computed from c->aos and c->box).
// When the context's last build was of the same n, the re-sort from its order (§4.4) runs.  A
// forest launches the full sort behind it for the case the device chooses that (its kernels
// return at once otherwise) and reads nothing back, so its step stays capturable; a single
// system reads the choice and launches only the chosen path.
nbody_status sort_bodies(nbody_ctx *c, const double *pos, int n, const Systems &ss,
                         const SortScratch &sc)
{
    cudaStream_t s = c->stream;
    const bool resort = c->order_n == n && c->sort_mode != NBODY_SORT_FULL &&
                        (c->sort_mode == NBODY_SORT_RESORT || n >= kResortMinN);
    c->order_n = -1;
    if (resort) {
        CKS(ensure_order(c));
        launch_order_extract(c->aos, c->ids, n, c->box, ss, c->sort_mode == NBODY_SORT_AUTO,
                             c->keys, c->ord, s);
        record(c, 1);
        if (c->n_sys == 0) {
            // a single system synchronises later in its build anyway: read the device's choice
            // now and launch only that path
            CK(cudaMemcpyAsync(c->h_word + 2, c->ord.stats, sizeof(uint32_t) * kOrderStats,
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (c->h_word[2 + kOrderResorted] != 0u) {
                launch_order_merge(c->keys, c->ids, n, ss, c->ord, sc, s);
            } else {
                launch_keys(pos, n, c->box, ss, c->keys, c->ids, s);
                launch_radix_sort(c->keys, c->ids, n, sc, s);
            }
        } else {
            launch_order_merge(c->keys, c->ids, n, ss, c->ord, sc, s);
            const int *full_n = order_full_count(c->ord);
            launch_keys(pos, n, c->box, ss, c->keys, c->ids, s, full_n);
            SortScratch sf = sc;
            sf.d_n = full_n;
            launch_radix_sort(c->keys, c->ids, n, sf, s);
        }
    } else {
        launch_keys(pos, n, c->box, ss, c->keys, c->ids, s);
        record(c, 1);
        launch_radix_sort(c->keys, c->ids, n, sc, s);
    }
    CKS(check_launch(c, "sort"));
    c->last_sort_path = resort ? 2 : 0;
    c->order_n = n;
    return NBODY_OK;
}

// Root box, keys, sort, permutation, node split and moments of (pos, mass).  When
// `have_partials` the bbox partial reductions of pos are already in c->partials.
nbody_status build(nbody_ctx *c, const double *pos, const double *mass, int n,
                   bool have_partials)
{
    cudaStream_t s = c->stream;
    if (n == 0) {
        c->n_nodes = 0;
        c->n_built = 0;
        return NBODY_OK;
    }
    const Systems one{nullptr, nullptr, 1};
    const bool check = (c->p.flags & NBODY_FLAG_CHECK_FINITE) != 0;
    if (check) {
        CK(cudaMemsetAsync(c->chk, 0, sizeof(int), s));
        launch_check_finite(pos, mass, n, c->chk, s);
    }
    if (!have_partials) launch_bbox_partials(pos, mass, n, c->partials, c->nblk, c->aos, s);
    launch_bbox_finalize(c->partials, c->nblk, c->box, c->tab, c->p.theta, s);
    SortScratch sc{c->keys_alt, c->ids_alt, c->hist, c->counts, sort_tiles((int)c->cap), nullptr,
                   nullptr};
    CKS(sort_bodies(c, pos, n, one, sc));
    record(c, 2);
    launch_permute(c->aos, c->ids, n, c->box, one, c->p.G, c->sbody64, c->sbody32, s);
    CK(cudaMemsetAsync(c->info, 0, sizeof(unsigned), s));
    launch_count_nodes(c->keys, n, one, c->node_off, c->info, s);
    ScanScratch ss{c->block_sums, scan_tiles((int)c->cap + 1)};
    launch_exclusive_scan(c->node_off, c->node_off, n + 1, ss, s);
    CKS(check_launch(c, "tree build"));
    CK(cudaMemcpyAsync(c->h_word, c->node_off + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->h_word + 1, c->info, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    if (check) CK(cudaMemcpyAsync(c->h_word + 2, c->chk, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (check && c->h_word[2] != 0u) {
        c->n_built = -1;
        c->order_n = -1;
        return fail(c, NBODY_EINVAL, "a position or mass is NaN or infinite");
    }
    const int64_t nn = (int64_t)c->h_word[0];
    const int max_level = (int)c->h_word[1];
    if (nn < 1 || nn > 22 * (int64_t)n)
        return fail(c, NBODY_ECUDA, "node count %lld out of range for n = %d", (long long)nn, n);
    const bool group = !is_fp64(c->p.precision);
    if (group && nn > (int64_t)kMaxGroupNodes)
        return fail(c, NBODY_EINVAL, "%lld tree nodes: the FP32 walk indexes at most %lld",
                    (long long)nn, (long long)kMaxGroupNodes);
    CKS(ensure_nodes(c, nn));
    CKS(ensure_quad(c));
    c->n_nodes = nn;
    c->na.d_nn = c->node_off + n;
    launch_emit_nodes(c->keys, n, one, c->node_off, c->na, c->err, s);
    launch_level_order(c->na, s);
    if (sums_moments(c)) {
        launch_subtree_sums(c->keys, max_level, c->sbody64, c->sbody32, c->box, c->tab, one,
                            c->p.G, c->na, c->gn, false, s);
    } else {
        launch_moments(c->keys, max_level, c->sbody64, c->box, c->tab, one, c->p.G, c->na, s);
        if (group) launch_group_nodes(c->na, c->box, c->tab, one, c->p.G, c->gn, s);
    }
    if (group && cell_groups_for(c, n)) {
        CK(cudaMemsetAsync(c->cgroups_n, 0, sizeof(unsigned), s));
        launch_cell_groups(c->na, c->node_off, one, n, 32, c->cgroups, c->cgroups_n, c->cap + 1,
                           c->err, s);
    }
    record(c, 3);
    CKS(check_launch(c, "node split / moments"));
    c->n_built = n;
    return NBODY_OK;
}

nbody_status walk(nbody_ctx *c, int n, double *acc, double *vel, double h)
{
    if (n == 0) return NBODY_OK;
    WalkArgs a;
    a.wn = c->na.wn;
    a.com64 = c->na.com64;
    a.level = c->na.level;
    a.tab = c->tab;
    a.sbody64 = c->sbody64;
    a.sbody32 = c->sbody32;
    a.ids = c->ids;
    a.n = n;
    a.G = c->p.G;
    a.eps = c->p.eps;
    a.theta = c->p.theta;
    a.acc = acc;
    a.vel = vel;
    a.h = h;
    a.pp = c->pp;
    a.pc = c->pc;
    a.gn = c->gn;
    a.err = c->err;
    a.d_nn = c->na.d_nn;
    a.groups = c->groups;
    a.n_groups = c->n_groups;
    a.d_ngroups = nullptr;
    a.roots = c->roots;
    a.work = c->work;
    const int shape = walk_shape_for(c, n);
    const bool cells = cell_groups_for(c, n);
    if (cells) {
        a.groups = c->cgroups;
        a.n_groups = (int)std::min<int64_t>(c->cap + 1, INT32_MAX);
        a.d_ngroups = c->cgroups_n;
    }
    a.node_off = c->node_off;
    a.start = c->sys_start;
    a.group_mac = (c->p.flags & NBODY_FLAG_GROUP_MAC) != 0;
    a.q64 = c->na.q64;
    a.gq = !is_fp64(c->p.precision) ? c->na.gq : nullptr;
    a.stack_limit = c->stack_limit;
    a.step_limit = c->step_limit;
    a.fast_stack_limit = c->fast_stack_limit;
    CKS(ensure_overflow(c));
    a.overflow = c->overflow;
    a.n_overflow = c->n_overflow;
    a.span_meta = nullptr;
    a.span_off = a.span_pool = a.span_tmp = nullptr;
    a.span_next = nullptr;
    a.span_pool_cap = 0;
    a.span_bodies = 0;
    const int span = walk_shape32(shape).span_bodies;
    if (use_spans(c) && !cells && span > 0) {
        CKS(ensure_spans(c, n));
        a.span_bodies = span;
        a.span_meta = c->span_meta;
        a.span_off = c->span_off;
        a.span_pool = c->span_pool;
        a.span_pool_cap = c->span_pool_cap;
        a.span_tmp = c->span_tmp;
        a.span_next = c->span_next;
    }
    launch_walk(c->p.precision, a, shape, c->stream);
    record(c, 4);
    CKS(check_launch(c, "walk"));
    c->n_forces = n;
    return NBODY_OK;
}

// ---------------------------------------------------------------- forest
// Every step of a forest runs over all systems at once, with no host synchronisation: the node
// count stays on the device (the node arrays are sized at creation), so a step can be captured
// as a CUDA graph.

Systems systems(const nbody_ctx *c) { return Systems{c->sys, c->sys_start, c->n_sys}; }

// vel non-null: a step's kick and drift (half kick h) come first, fused with the boxes.
nbody_status forest_build(nbody_ctx *c, double *pos, const double *mass, double *vel = nullptr,
                          double h = 0.0)
{
    cudaStream_t s = c->stream;
    const int n = (int)c->cap;
    const Systems ss = systems(c);
    if (c->p.flags & NBODY_FLAG_CHECK_FINITE) launch_check_finite(pos, mass, n, c->err, s);
    launch_forest_boxes(pos, vel, c->acc, mass, n, c->box_chunks, c->n_box_chunks,
                        c->box_chunk_start, c->n_sys, h, c->p.dt, c->box_partials, c->box, c->tab,
                        c->p.theta, c->aos, !is_fp64(c->p.precision), s);
    SortScratch sc{c->keys_alt, c->ids_alt, c->hist, c->counts, sort_tiles(n), c->sys,
                   c->sys_hist};
    CKS(sort_bodies(c, pos, n, ss, sc));
    record(c, 2);
    launch_permute(c->aos, c->ids, n, c->box, ss, c->p.G, c->sbody64, c->sbody32, s);
    CK(cudaMemsetAsync(c->info, 0, sizeof(unsigned), s));
    launch_count_nodes(c->keys, n, ss, c->node_off, c->info, s);
    ScanScratch sn{c->block_sums, scan_tiles(n + 1)};
    launch_exclusive_scan(c->node_off, c->node_off, n + 1, sn, s);
    launch_clamp_count(c->node_off + n, c->na.cap, c->nn, c->err, s);
    CKS(ensure_quad(c));  // pointers only: the arrays exist since creation / set_params
    c->na.d_nn = c->nn;
    launch_emit_nodes(c->keys, n, ss, c->node_off, c->na, c->err, s);
    launch_level_order(c->na, s);
    if (sums_moments(c)) {
        launch_subtree_sums(c->keys, kMaxLevel, c->sbody64, c->sbody32, c->box, c->tab, ss,
                            c->p.G, c->na, c->gn, false, s);
    } else {
        launch_moments(c->keys, kMaxLevel, c->sbody64, c->box, c->tab, ss, c->p.G, c->na, s);
        if (!is_fp64(c->p.precision))
            launch_group_nodes(c->na, c->box, c->tab, ss, c->p.G, c->gn, s);
    }
    launch_roots(c->na, c->node_off, ss, c->roots, s);
    if (cell_groups_for(c, n)) {
        CK(cudaMemsetAsync(c->cgroups_n, 0, sizeof(unsigned), s));
        launch_cell_groups(c->na, c->node_off, ss, n, 32, c->cgroups, c->cgroups_n, c->cap + 1,
                           c->err, s);
    }
    record(c, 3);
    CKS(check_launch(c, "forest build"));
    c->n_built = n;
    c->n_nodes = -1;  // on the device only
    return NBODY_OK;
}

nbody_status forest_step_once(nbody_ctx *c, double *pos, double *vel, const double *mass)
{
    const int n = (int)c->cap;
    const double h = 0.5 * c->p.dt;
    CKS(forest_build(c, pos, mass, vel, h));
    return walk(c, n, c->acc, vel, h);
}

nbody_status begin_timing(nbody_ctx *c);
nbody_status end_timing(nbody_ctx *c);

// a^(k) at the current positions, unless kept from the previous call
nbody_status ensure_acc(nbody_ctx *c, const double *pos, const double *mass, int64_t n)
{
    if (c->acc_n == n) return NBODY_OK;
    CKS(build(c, pos, mass, (int)n, false));
    CKS(walk(c, (int)n, c->acc, nullptr, 0.0));
    c->acc_n = n;
    return NBODY_OK;
}

// One kick-drift-kick step (§2.4); `drifted` (may be null) is recorded on the context stream once
// the positions of this step are final (after the drift).
nbody_status step_once(nbody_ctx *c, double *pos, double *vel, const double *mass, int64_t n,
                       cudaEvent_t drifted)
{
    const double h = 0.5 * c->p.dt;
    CKS(begin_timing(c));
    launch_kick_drift_bbox(pos, vel, c->acc, mass, (int)n, h, c->p.dt, c->partials, c->nblk,
                           c->aos, !is_fp64(c->p.precision), c->stream);
    CKS(check_launch(c, "kick/drift"));
    if (drifted) CK(cudaEventRecord(drifted, c->stream));
    CKS(build(c, pos, mass, (int)n, true));
    CKS(walk(c, (int)n, c->acc, vel, h));
    return end_timing(c);
}

nbody_status begin_timing(nbody_ctx *c)
{
    if (!c->timing) return NBODY_OK;
    c->timing_pending = false;
    for (int k = 0; k < 5; ++k) c->ms[k] = 0.f;
    CK(cudaEventRecord(c->ev[0], c->stream));
    for (int k = 1; k < 5; ++k) CK(cudaEventRecord(c->ev[k], c->stream));
    return NBODY_OK;
}

nbody_status end_timing(nbody_ctx *c)
{
    if (!c->timing) return NBODY_OK;
    CK(cudaEventRecord(c->ev[5], c->stream));
    c->timing_pending = true;
    return NBODY_OK;
}

}  // namespace

extern "C" {

nbody_status nbody_create(nbody_ctx **out, int64_t n_capacity, const nbody_params *p,
                          void *cuda_stream)
{
    nbody_ctx *c = nullptr;
    if (!out) return NBODY_EINVAL;
    *out = nullptr;
    if (n_capacity < 0 || n_capacity > ((int64_t)1 << 30) || !params_ok(p)) return NBODY_EINVAL;
    c = new (std::nothrow) nbody_ctx;
    if (!c) return NBODY_ENOMEM;
    c->p = *p;
    c->cap = n_capacity;
    c->stream = (cudaStream_t)cuda_stream;
    nbody_status st = NBODY_OK;
    auto body = [&]() -> nbody_status {
        CK(cudaGetDevice(&c->device));
        CK(sort_prepare());
        CK(walk_prepare());
        const size_t cap = (size_t)std::max<int64_t>(n_capacity, 1);
        CK(dalloc(&c->keys, cap));
        CK(dalloc(&c->keys_alt, cap));
        CK(dalloc(&c->ids, cap));
        CK(dalloc(&c->ids_alt, cap));
        CK(dalloc(&c->sbody64, cap));
        CK(dalloc(&c->aos, cap));
        CK(dalloc(&c->sbody32, cap));
        CK(dalloc(&c->node_off, cap + 1));
        CK(dalloc(&c->hist, 14 * 256));
        CK(dalloc(&c->counts, (size_t)256 * sort_tiles((int)cap)));
        CK(dalloc(&c->block_sums, (size_t)scan_tiles((int)cap + 1) + 1));
        c->nblk = bbox_blocks((int64_t)cap);
        CK(dalloc(&c->partials, (size_t)bbox_partial_doubles() * c->nblk));
        CK(dalloc(&c->box, 2));
        CK(dalloc(&c->tab, 2));
        CK(dalloc(&c->acc, 3 * cap));
        CK(dalloc(&c->pp, cap));
        CK(dalloc(&c->pc, cap));
        CK(dalloc(&c->err, 1));
        CK(dalloc(&c->cgroups, cap + 1));
        CK(dalloc(&c->cgroups_n, 1));
        CK(dalloc(&c->work, 2));
        CK(dalloc(&c->chk, 1));
        CK(cudaMemset(c->err, 0, sizeof(int)));
        CK(cudaMallocHost((void **)&c->h_word, (2 + kOrderStats) * sizeof(uint32_t)));
        CK(dalloc(&c->info, 1));
        for (int k = 0; k < 6; ++k) CK(cudaEventCreate(&c->ev[k]));
        return NBODY_OK;
    };
    st = body();
    if (st != NBODY_OK) {
        nbody_destroy(c);
        return st;
    }
    *out = c;
    return NBODY_OK;
}

nbody_status nbody_destroy(nbody_ctx *c)
{
    if (!c) return NBODY_EINVAL;
    cudaStreamSynchronize(c->stream);
    dfree(c->keys);
    dfree(c->keys_alt);
    dfree(c->ids);
    dfree(c->ids_alt);
    dfree(c->sbody64);
    dfree(c->aos);
    dfree(c->sbody32);
    dfree(c->node_off);
    dfree(c->hist);
    dfree(c->counts);
    dfree(c->block_sums);
    dfree(c->partials);
    dfree(c->box);
    dfree(c->tab);
    dfree(c->acc);
    dfree(c->pp);
    dfree(c->pc);
    dfree(c->err);
    dfree(c->info);
    dfree(c->dscratch);
    dfree(c->cgroups);
    dfree(c->cgroups_n);
    dfree(c->work);
    dfree(c->chk);
    dfree(c->overflow);
    dfree(c->n_overflow);
    free_spans(c);
    dfree(c->sys);
    dfree(c->sys_start);
    dfree(c->sys_hist);
    dfree(c->groups);
    dfree(c->roots);
    dfree(c->nn);
    dfree(c->box_chunks);
    dfree(c->box_chunk_start);
    dfree(c->box_partials);
    free_order(c);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    for (int k = 0; k < 2; ++k)
        if (c->gev[k]) cudaEventDestroy(c->gev[k]);
    dfree(c->hpos);
    dfree(c->hvel);
    dfree(c->hmass);
    if (c->xdrift) cudaEventDestroy(c->xdrift);
    if (c->xstream) cudaStreamDestroy(c->xstream);
    free_nodes(c);
    if (c->h_word) cudaFreeHost(c->h_word);
    for (int k = 0; k < 6; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    delete c;
    return NBODY_OK;
}

nbody_status nbody_set_params(nbody_ctx *c, const nbody_params *p)
{
    if (!c) return NBODY_EINVAL;
    if (!params_ok(p)) return fail(c, NBODY_EINVAL, "invalid parameters");
    c->p = *p;
    c->acc_n = -1;
    CKS(ensure_quad(c));
    if (c->gexec) {  // the captured step holds the old parameters
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return NBODY_OK;
}

nbody_status nbody_build_tree(nbody_ctx *c, const double *d_pos, const double *d_mass, int64_t n)
{
    if (!c) return NBODY_EINVAL;
    if (c->n_sys) return fail(c, NBODY_ESTATE, "a forest context takes the forest entry points");
    CKS(check_n(c, n));
    if (n > 0 && (!d_pos || !d_mass)) return fail(c, NBODY_EINVAL, "null pointer");
    CKS(begin_timing(c));
    CKS(build(c, d_pos, d_mass, (int)n, false));
    return end_timing(c);
}

nbody_status nbody_forces(nbody_ctx *c, const double *d_pos, const double *d_mass, int64_t n,
                          double *d_acc)
{
    if (!c) return NBODY_EINVAL;
    if (c->n_sys) return fail(c, NBODY_ESTATE, "a forest context takes the forest entry points");
    CKS(check_n(c, n));
    if (n > 0 && (!d_pos || !d_mass || !d_acc)) return fail(c, NBODY_EINVAL, "null pointer");
    CKS(begin_timing(c));
    CKS(build(c, d_pos, d_mass, (int)n, false));
    CKS(walk(c, (int)n, d_acc, nullptr, 0.0));
    return end_timing(c);
}

nbody_status nbody_step(nbody_ctx *c, double *d_pos, double *d_vel, const double *d_mass,
                        int64_t n, int32_t nsteps)
{
    if (!c) return NBODY_EINVAL;
    if (c->n_sys) return fail(c, NBODY_ESTATE, "a forest context takes the forest entry points");
    CKS(check_n(c, n));
    if (nsteps < 0) return fail(c, NBODY_EINVAL, "nsteps < 0");
    if (n > 0 && (!d_pos || !d_vel || !d_mass)) return fail(c, NBODY_EINVAL, "null pointer");
    if (n == 0 || nsteps == 0) return NBODY_OK;
    CKS(ensure_acc(c, d_pos, d_mass, n));
    for (int32_t k = 0; k < nsteps; ++k) CKS(step_once(c, d_pos, d_vel, d_mass, n, nullptr));
    return NBODY_OK;
}

nbody_status nbody_step_host(nbody_ctx *c, double *h_pos, double *h_vel, double *h_acc,
                             const double *h_mass, int64_t n, int32_t nsteps)
{
    if (!c) return NBODY_EINVAL;
    if (c->n_sys) return fail(c, NBODY_ESTATE, "a forest context takes the forest entry points");
    CKS(check_n(c, n));
    if (nsteps < 0) return fail(c, NBODY_EINVAL, "nsteps < 0");
    if (n > 0 && (!h_pos || !h_vel || !h_mass)) return fail(c, NBODY_EINVAL, "null pointer");
    if (n == 0) return NBODY_OK;
    if (!c->hpos) {
        const size_t cap = (size_t)c->cap;
        CK(dalloc(&c->hpos, 3 * cap));
        CK(dalloc(&c->hvel, 3 * cap));
        CK(dalloc(&c->hmass, cap));
    }
    const size_t b3 = sizeof(double) * 3 * (size_t)n;
    CK(cudaMemcpyAsync(c->hpos, h_pos, b3, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->hvel, h_vel, b3, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->hmass, h_mass, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice,
                       c->stream));
    if (h_acc) {
        // the caller's a^(k) at h_pos: no force evaluation before the first kick
        CK(cudaMemcpyAsync(c->acc, h_acc, b3, cudaMemcpyHostToDevice, c->stream));
        c->acc_n = n;
    } else {
        c->acc_n = -1;
    }
    CKS(ensure_acc(c, c->hpos, c->hmass, n));
    if (nsteps > 0) {
        if (!c->xstream) {
            CK(cudaStreamCreateWithFlags(&c->xstream, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&c->xdrift, cudaEventDisableTiming));
        }
        for (int32_t k = 0; k + 1 < nsteps; ++k)
            CKS(step_once(c, c->hpos, c->hvel, c->hmass, n, nullptr));
        // the last step: its positions go back to the host while its tree and walk run
        CKS(step_once(c, c->hpos, c->hvel, c->hmass, n, c->xdrift));
        CK(cudaStreamWaitEvent(c->xstream, c->xdrift, 0));
        CK(cudaMemcpyAsync(h_pos, c->hpos, b3, cudaMemcpyDeviceToHost, c->xstream));
    } else {
        CK(cudaMemcpyAsync(h_pos, c->hpos, b3, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaMemcpyAsync(h_vel, c->hvel, b3, cudaMemcpyDeviceToHost, c->stream));
    if (h_acc) CK(cudaMemcpyAsync(h_acc, c->acc, b3, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->xstream) CK(cudaStreamSynchronize(c->xstream));
    c->acc_n = -1;  // the device copy belongs to this call only
    return NBODY_OK;
}

nbody_status nbody_direct_forces(nbody_ctx *c, const double *d_pos, const double *d_mass,
                                 int64_t n, const int64_t *d_targets, int64_t nt, double *d_acc)
{
    if (!c) return NBODY_EINVAL;
    if (c->n_sys) return fail(c, NBODY_ESTATE, "a forest context takes the forest entry points");
    CKS(check_n(c, n));
    if (!d_targets) nt = n;
    if (nt < 0 || nt > ((int64_t)1 << 30)) return fail(c, NBODY_EINVAL, "bad target count");
    if (n > 0 && (!d_pos || !d_mass || !d_acc)) return fail(c, NBODY_EINVAL, "null pointer");
    if (n == 0 || nt == 0) return NBODY_OK;
    launch_bbox_partials(d_pos, d_mass, (int)n, c->partials, c->nblk, nullptr, c->stream);
    launch_bbox_finalize(c->partials, c->nblk, c->box + 1, c->tab + 1, c->p.theta, c->stream);
    DirectScratch ds{nullptr, nullptr};
    if (!is_fp64(c->p.precision)) {
        // FP32 scratch, grown on demand: sources, then per-chunk partial sums
        const int64_t need = (int64_t)4 * n + (int64_t)direct32_chunks((int)n, (int)nt) * 3 * nt;
        if (need > c->dscratch_cap) {
            dfree(c->dscratch);
            c->dscratch_cap = 0;
            CK(dalloc(&c->dscratch, (size_t)need));
            c->dscratch_cap = need;
        }
        ds.src = reinterpret_cast<float4 *>(c->dscratch);
        ds.part = c->dscratch + 4 * n;
    }
    launch_direct(c->p.precision, d_pos, d_mass, (int)n, d_targets, (int)nt, c->p.G, c->p.eps,
                  c->box + 1, d_acc, ds, c->stream);
    return check_launch(c, "direct sum");
}

nbody_status nbody_sync(nbody_ctx *c)
{
    if (!c) return NBODY_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    int e = 0;
    CK(cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e == 0) return NBODY_OK;
    // reported once: the word is cleared, and the context stays usable
    CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    c->acc_n = -1;  // a kept acceleration may come from the failed walk
    if (e & kErrInput) return fail(c, NBODY_EINVAL, "a position or mass is NaN or infinite");
    if (e & kErrTimeout) return fail(c, NBODY_ETIMEOUT, "a device-side wait gave up");
    if (e & kErrNodeCap) return fail(c, NBODY_ENOMEM, "node capacity exceeded on the device");
    if (e & kErrStack)
        return fail(c, NBODY_ESTACK, "a walk ran out of stack entries or steps");
    return fail(c, NBODY_ECUDA, "device error word %d", e);
}

nbody_status nbody_get_keys(nbody_ctx *c, uint64_t *h_keys_sorted, uint32_t *h_ids_sorted)
{
    if (!c) return NBODY_EINVAL;
    if (c->n_built < 0) return fail(c, NBODY_ESTATE, "no tree built yet");
    const size_t n = (size_t)c->n_built;
    CK(cudaStreamSynchronize(c->stream));
    if (h_keys_sorted) CK(cudaMemcpy(h_keys_sorted, c->keys, 8 * n, cudaMemcpyDeviceToHost));
    if (h_ids_sorted) CK(cudaMemcpy(h_ids_sorted, c->ids, 4 * n, cudaMemcpyDeviceToHost));
    return NBODY_OK;
}

nbody_status nbody_get_box(nbody_ctx *c, double *h_box)
{
    if (!c || !h_box) return NBODY_EINVAL;
    if (c->n_built < 0) return fail(c, NBODY_ESTATE, "no tree built yet");
    Box b;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(&b, c->box, sizeof(Box), cudaMemcpyDeviceToHost));
    h_box[0] = b.o[0];
    h_box[1] = b.o[1];
    h_box[2] = b.o[2];
    h_box[3] = b.L;
    h_box[4] = b.s;
    return NBODY_OK;
}

nbody_status nbody_get_tree(nbody_ctx *c, int64_t *n_nodes, nbody_tree_record *h_records,
                            int64_t cap)
{
    if (!c || !n_nodes) return NBODY_EINVAL;
    if (c->n_built < 0) return fail(c, NBODY_ESTATE, "no tree built yet");
    if (c->n_sys) return fail(c, NBODY_ESTATE, "a forest's trees stay on the device");
    const int64_t nn = c->n_nodes, n = c->n_built;
    *n_nodes = nn;
    if (!h_records || cap < nn || nn == 0) return NBODY_OK;
    std::vector<WalkNode> wn((size_t)nn);
    std::vector<uint8_t> lev((size_t)nn), mask((size_t)nn);
    std::vector<uint64_t> keys((size_t)n);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(wn.data(), c->na.wn, sizeof(WalkNode) * nn, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(lev.data(), c->na.level, nn, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(mask.data(), c->na.mask, nn, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(keys.data(), c->keys, 8 * n, cudaMemcpyDeviceToHost));
    for (int64_t j = 0; j < nn; ++j) {
        const int l = lev[j];
        const int64_t first = wn[j].first;
        const uint64_t prefix = l == 0 ? 0ull : (keys[first] >> (3 * (kMaxLevel - l)));
        nbody_tree_record &r = h_records[j];
        r.key = (1ull << (3 * l)) | prefix;
        r.level = l;
        r.child_mask = mask[j];
        r.first = first;
        if (wn[j].count != 0) {
            r.count = wn[j].count;
        } else {
            const int64_t sk = wn[j].skip;
            r.count = (sk < nn ? (int64_t)wn[sk].first : n) - first;
        }
    }
    return NBODY_OK;
}

nbody_status nbody_get_moments(nbody_ctx *c, double *h_out, int64_t cap_nodes)
{
    if (!c || !h_out) return NBODY_EINVAL;
    if (c->n_built < 0) return fail(c, NBODY_ESTATE, "no tree built yet");
    if (c->n_sys) return fail(c, NBODY_ESTATE, "a forest's trees stay on the device");
    const int64_t nn = c->n_nodes;
    if (cap_nodes < nn) return fail(c, NBODY_EINVAL, "cap_nodes < node count %lld", (long long)nn);
    if (nn == 0) return NBODY_OK;
    std::vector<D4> m((size_t)nn);
    CK(cudaStreamSynchronize(c->stream));
    if (sums_moments(c)) {
        // the build keeps FP64 sums only where its own passes read them: the sums pass runs
        // again on the same tree with every node's sums kept (centre of mass = sums / mass)
        const Systems one{nullptr, nullptr, 1};
        launch_subtree_sums(c->keys, kMaxLevel, c->sbody64, c->sbody32, c->box, c->tab, one,
                            c->p.G, c->na, c->gn, true, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        std::vector<D4> sm((size_t)nn);
        std::vector<int> inv((size_t)nn);
        CK(cudaMemcpy(sm.data(), c->na.com_lo, sizeof(D4) * nn, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(inv.data(), c->na.inv, sizeof(int) * nn, cudaMemcpyDeviceToHost));
        for (int64_t b = 0; b < nn; ++b) {
            const D4 &q = sm[(size_t)b];
            D4 &o = m[(size_t)inv[(size_t)b]];
            o.w = q.w;
            o.x = q.x / q.w;
            o.y = q.y / q.w;
            o.z = q.z / q.w;
        }
    } else {
        CK(cudaMemcpy(m.data(), c->na.com64, sizeof(D4) * nn, cudaMemcpyDeviceToHost));
    }
    for (int64_t j = 0; j < nn; ++j) {
        h_out[4 * j] = m[j].w;
        h_out[4 * j + 1] = m[j].x;
        h_out[4 * j + 2] = m[j].y;
        h_out[4 * j + 3] = m[j].z;
    }
    return NBODY_OK;
}

nbody_status nbody_get_counters(nbody_ctx *c, uint32_t *h_pp, uint32_t *h_pc)
{
    if (!c || !h_pp || !h_pc) return NBODY_EINVAL;
    if (c->n_forces < 0 || c->n_forces != c->n_built)
        return fail(c, NBODY_ESTATE, "no force evaluation on the current tree");
    const size_t n = (size_t)c->n_forces;
    std::vector<uint32_t> ids(n), pp(n), pc(n);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(ids.data(), c->ids, 4 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(pp.data(), c->pp, 4 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(pc.data(), c->pc, 4 * n, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) {
        h_pp[ids[i]] = pp[i];
        h_pc[ids[i]] = pc[i];
    }
    return NBODY_OK;
}

nbody_status nbody_enable_timing(nbody_ctx *c, int32_t on)
{
    if (!c) return NBODY_EINVAL;
    c->timing = on != 0;
    return NBODY_OK;
}

nbody_status nbody_get_timings(nbody_ctx *c, float *h_ms5)
{
    if (!c || !h_ms5) return NBODY_EINVAL;
    if (c->timing_pending) {
        CK(cudaEventSynchronize(c->ev[5]));
        for (int k = 0; k < 4; ++k) CK(cudaEventElapsedTime(&c->ms[k], c->ev[k], c->ev[k + 1]));
        CK(cudaEventElapsedTime(&c->ms[4], c->ev[0], c->ev[5]));
        c->timing_pending = false;
    }
    for (int k = 0; k < 5; ++k) h_ms5[k] = c->ms[k];
    return NBODY_OK;
}

nbody_status nbody_get_launch_count(int64_t *out)
{
    if (!out) return NBODY_EINVAL;
    *out = launch_count();
    return NBODY_OK;
}

nbody_status nbody_last_error(nbody_ctx *c, char *buf, int64_t cap)
{
    if (!c || !buf || cap <= 0) return NBODY_EINVAL;
    snprintf(buf, (size_t)cap, "%s", c->msg);
    return NBODY_OK;
}

// ---------------------------------------------------------------- autotuning

nbody_status nbody_autotune(nbody_ctx *c, const double *d_pos, const double *d_mass, int64_t n,
                            float *h_ms, int32_t *chosen)
{
    if (!c) return NBODY_EINVAL;
    if (c->n_sys) n = c->cap;
    CKS(check_n(c, n));
    if (n > 0 && (!d_pos || !d_mass)) return fail(c, NBODY_EINVAL, "null pointer");
    int &shape = is_fp64(c->p.precision) ? c->shape64 : c->shape32;
    if (h_ms)
        for (int k = 0; k < kWalkShapes; ++k) h_ms[k] = 0.f;
    if (n == 0) {
        if (chosen) *chosen = shape;
        return NBODY_OK;
    }
    const bool timing = c->timing;
    c->timing = false;
    // one tree for every candidate, with the cell-following groups when a candidate uses them
    c->forced_shape = shape_applies(c, 7) ? 7 : shape;
    nbody_status st = c->n_sys ? forest_build(c, const_cast<double *>(d_pos), d_mass)
                               : build(c, d_pos, d_mass, (int)n, false);
    float ms[kWalkShapes] = {};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == NBODY_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = fail(c, NBODY_ECUDA, "event creation failed");
    const int reps = 3;
    for (int k = 0; k < kWalkShapes && st == NBODY_OK; ++k) {
        if (!shape_applies(c, k)) continue;
        c->forced_shape = k;
        st = walk(c, (int)n, c->acc, nullptr, 0.0);  // warm-up of this shape
        if (st == NBODY_OK && cudaEventRecord(e0, c->stream) != cudaSuccess)
            st = fail(c, NBODY_ECUDA, "event record failed");
        for (int r = 0; r < reps && st == NBODY_OK; ++r) st = walk(c, (int)n, c->acc, nullptr, 0.0);
        if (st == NBODY_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess ||
                               cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(&ms[k], e0, e1) != cudaSuccess))
            st = fail(c, NBODY_ECUDA, "timing the walk failed");
        ms[k] /= (float)reps;
    }
    c->forced_shape = -1;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->timing = timing;
    c->acc_n = -1;  // the walks above overwrote the kept acceleration
    if (st != NBODY_OK) return st;
    int best = -1;
    for (int k = 0; k < kWalkShapes; ++k)
        if (shape_applies(c, k) && (best < 0 || ms[k] < ms[best])) best = k;
    shape = best;
    // kept for this size bucket and theta; other sizes use it too until tuned themselves
    const int b = size_bucket(n);
    bool found = false;
    for (auto &e : c->shape_cache)
        if (e.bucket == b && e.theta == c->p.theta) {
            e.shape = best;
            found = true;
        }
    if (!found) c->shape_cache.push_back({b, c->p.theta, best});
    if (c->gexec) {  // a captured forest step holds the old shape
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (h_ms)
        for (int k = 0; k < kWalkShapes; ++k) h_ms[k] = ms[k];
    if (chosen) *chosen = best;
    return NBODY_OK;
}

nbody_status nbody_set_walk_shape(nbody_ctx *c, int32_t shape)
{
    if (!c) return NBODY_EINVAL;
    if (shape < 0 || shape >= kWalkShapes) return fail(c, NBODY_EINVAL, "shape %d", (int)shape);
    (is_fp64(c->p.precision) ? c->shape64 : c->shape32) = shape;
    c->shape_cache.clear();  // an explicit shape replaces the tuned choices
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return NBODY_OK;
}

nbody_status nbody_get_walk_shape(nbody_ctx *c, int32_t *shape, int32_t *threads_per_block)
{
    if (!c) return NBODY_EINVAL;
    const int k = is_fp64(c->p.precision) ? c->shape64 : c->shape32;
    if (shape) *shape = k;
    if (threads_per_block) *threads_per_block = walk_shape_threads(c->p.precision, k);
    return NBODY_OK;
}

nbody_status nbody_set_walk_limits(nbody_ctx *c, int32_t stack_entries, int64_t max_steps,
                                   int32_t fast_entries)
{
    if (!c) return NBODY_EINVAL;
    if (stack_entries != 0 && stack_entries < 33)
        return fail(c, NBODY_EINVAL, "stack_entries %d: 0 or at least 33", (int)stack_entries);
    if (max_steps < 0) return fail(c, NBODY_EINVAL, "max_steps < 0");
    if (fast_entries != 0 && fast_entries < 64)
        return fail(c, NBODY_EINVAL, "fast_entries %d: 0 or at least 64", (int)fast_entries);
    c->stack_limit = stack_entries == 0 ? (1 << 30) : stack_entries;
    c->step_limit = max_steps == 0 ? INT64_MAX : max_steps;
    c->fast_stack_limit = fast_entries == 0 ? (1 << 30) : fast_entries;
    if (c->gexec) {  // a captured forest step holds the old limits
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return NBODY_OK;
}

nbody_status nbody_measure_fp32_rate(void *cuda_stream, double *h_tflops)
{
    if (!h_tflops) return NBODY_EINVAL;
    *h_tflops = 0.0;
    const cudaError_t e = measure_fp32_rate((cudaStream_t)cuda_stream, h_tflops);
    if (e == cudaErrorMemoryAllocation) return NBODY_ENOMEM;
    return e == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
}

nbody_status nbody_measure_fp64_rate(void *cuda_stream, double *h_tflops)
{
    if (!h_tflops) return NBODY_EINVAL;
    *h_tflops = 0.0;
    const cudaError_t e = measure_fp64_rate((cudaStream_t)cuda_stream, h_tflops);
    if (e == cudaErrorMemoryAllocation) return NBODY_ENOMEM;
    return e == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
}

nbody_status nbody_set_sort_mode(nbody_ctx *c, int32_t mode)
{
    if (!c) return NBODY_EINVAL;
    if (mode < NBODY_SORT_AUTO || mode > NBODY_SORT_RESORT)
        return fail(c, NBODY_EINVAL, "sort mode %d not in 0..2", (int)mode);
    c->sort_mode = mode;
    return NBODY_OK;
}

nbody_status nbody_get_sort_stats(nbody_ctx *c, int32_t *path, int64_t *removed)
{
    if (!c) return NBODY_EINVAL;
    int32_t p = c->last_sort_path;
    int64_t r = -1;
    if (p == 2) {  // the device chose: read its words after the last build
        CK(cudaMemcpyAsync(c->h_word + 2, c->ord.stats, sizeof(uint32_t) * kOrderStats,
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        p = c->h_word[2 + kOrderResorted] ? 1 : 0;
        r = (int64_t)c->h_word[2 + kOrderRemoved];
    }
    if (path) *path = p;
    if (removed) *removed = r;
    return NBODY_OK;
}

// ---------------------------------------------------------------- forest

nbody_status nbody_forest_create(nbody_ctx **out, int32_t n_systems, const int64_t *h_offsets,
                                 const nbody_params *p, void *cuda_stream)
{
    if (!out) return NBODY_EINVAL;
    *out = nullptr;
    if (n_systems < 1 || n_systems > kMaxSystems || !h_offsets || !params_ok(p)) return NBODY_EINVAL;
    if (h_offsets[0] != 0) return NBODY_EINVAL;
    for (int32_t k = 0; k < n_systems; ++k)
        if (h_offsets[k + 1] < h_offsets[k]) return NBODY_EINVAL;
    const int64_t n = h_offsets[n_systems];
    if (n < 1 || n > ((int64_t)1 << 30)) return NBODY_EINVAL;
    nbody_status st = nbody_create(out, n, p, cuda_stream);
    if (st != NBODY_OK) return st;
    nbody_ctx *c = *out;
    auto body = [&]() -> nbody_status {
        const int S = n_systems;
        c->n_sys = S;
        std::vector<uint16_t> sys((size_t)n);
        std::vector<int> start((size_t)S + 1);
        std::vector<uint32_t> hist(2 * 256, 0u);
        std::vector<int4> groups, chunks;
        std::vector<int> chunk_start((size_t)S + 1);
        for (int k = 0; k < S; ++k) {
            const int64_t lo = h_offsets[k], hi = h_offsets[k + 1];
            start[k] = (int)lo;
            chunk_start[k] = (int)chunks.size();
            for (int64_t b = lo; b < hi; b += kForestBoxChunk)
                chunks.push_back(make_int4((int)b, (int)std::min<int64_t>(b + kForestBoxChunk, hi),
                                           k, 0));
            for (int64_t i = lo; i < hi; ++i) sys[(size_t)i] = (uint16_t)k;
            hist[k & 255] += (uint32_t)(hi - lo);
            hist[256 + ((k >> 8) & 255)] += (uint32_t)(hi - lo);
            for (int64_t b = lo; b < hi; b += 32)
                groups.push_back(make_int4((int)b, (int)std::min<int64_t>(32, hi - b), k, 0));
        }
        start[S] = (int)n;
        chunk_start[S] = (int)chunks.size();
        c->n_groups = (int)groups.size();
        c->n_box_chunks = (int)chunks.size();
        CK(dalloc(&c->box_chunks, chunks.size()));
        CK(dalloc(&c->box_chunk_start, (size_t)S + 1));
        CK(dalloc(&c->box_partials, (size_t)bbox_partial_doubles() * std::max<size_t>(1, chunks.size())));
        if (!chunks.empty())
            CK(cudaMemcpy(c->box_chunks, chunks.data(), sizeof(int4) * chunks.size(),
                          cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->box_chunk_start, chunk_start.data(), sizeof(int) * (S + 1),
                      cudaMemcpyHostToDevice));
        CK(dalloc(&c->sys, (size_t)n));
        CK(dalloc(&c->sys_start, (size_t)S + 1));
        CK(dalloc(&c->sys_hist, 2 * 256));
        CK(dalloc(&c->groups, groups.size()));
        CK(dalloc(&c->roots, (size_t)S));
        CK(dalloc(&c->nn, 1));
        CK(cudaMemcpy(c->sys, sys.data(), sizeof(uint16_t) * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->sys_start, start.data(), sizeof(int) * (S + 1), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->sys_hist, hist.data(), sizeof(uint32_t) * 512, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->groups, groups.data(), sizeof(int4) * groups.size(),
                      cudaMemcpyHostToDevice));
        // one root box and level table per system
        dfree(c->box);
        dfree(c->tab);
        CK(dalloc(&c->box, (size_t)std::max(2, S)));
        CK(dalloc(&c->tab, (size_t)std::max(2, S)));
        // the node count is only known on the device during a step: room for 4 nodes per body
        // (Plummer-like systems need about 1.5) plus a full chain of 22 levels per system
        CKS(ensure_nodes(c, 4 * n + 22 * (int64_t)S + 1024));
        CKS(ensure_quad(c));
        CKS(ensure_order(c));  // the re-sort's scratch: never allocated inside a (captured) step
        CKS(ensure_overflow(c));
        if (c->na.cap > kMaxGroupNodes)
            return fail(c, NBODY_EINVAL, "forest of %lld bodies exceeds the node index range",
                        (long long)n);
        return NBODY_OK;
    };
    st = body();
    if (st != NBODY_OK) {
        nbody_destroy(c);
        *out = nullptr;
        return st;
    }
    return NBODY_OK;
}

nbody_status nbody_forest_forces(nbody_ctx *c, const double *d_pos, const double *d_mass,
                                 double *d_acc)
{
    if (!c) return NBODY_EINVAL;
    if (c->n_sys == 0) return fail(c, NBODY_ESTATE, "not a forest context");
    if (!d_pos || !d_mass || !d_acc) return fail(c, NBODY_EINVAL, "null pointer");
    CKS(begin_timing(c));
    CKS(forest_build(c, const_cast<double *>(d_pos), d_mass));  // positions only read
    CKS(walk(c, (int)c->cap, d_acc, nullptr, 0.0));
    return end_timing(c);
}

nbody_status nbody_forest_step(nbody_ctx *c, double *d_pos, double *d_vel, const double *d_mass,
                               int32_t nsteps, int32_t use_graph)
{
    if (!c) return NBODY_EINVAL;
    if (c->n_sys == 0) return fail(c, NBODY_ESTATE, "not a forest context");
    if (nsteps < 0) return fail(c, NBODY_EINVAL, "nsteps < 0");
    if (!d_pos || !d_vel || !d_mass) return fail(c, NBODY_EINVAL, "null pointer");
    if (nsteps == 0) return NBODY_OK;
    const int64_t n = c->cap;
    if (c->acc_n != n) {
        CKS(forest_build(c, d_pos, d_mass));
        CKS(walk(c, (int)n, c->acc, nullptr, 0.0));
        c->acc_n = n;
    }
    if (!use_graph) {
        for (int32_t k = 0; k < nsteps; ++k) {
            CKS(begin_timing(c));
            CKS(forest_step_once(c, d_pos, d_vel, d_mass));
            CKS(end_timing(c));
        }
        return NBODY_OK;
    }
    if (!c->gstream) {
        CK(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) CK(cudaEventCreateWithFlags(&c->gev[k], cudaEventDisableTiming));
    }
    // the captured step depends on the buffers and on the sort mode (re-sort or full sort)
    const void *key[4] = {d_pos, d_vel, d_mass, reinterpret_cast<const void *>((intptr_t)c->sort_mode)};
    if (!c->gexec || memcmp(key, c->gkey, sizeof(key)) != 0) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        // the caller's stream must reach this point before the captured work may run
        CK(cudaEventRecord(c->gev[0], c->stream));
        CK(cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
        CK(cudaStreamSynchronize(c->gstream));
        cudaStream_t user = c->stream;
        const bool timing = c->timing;
        c->stream = c->gstream;
        c->timing = false;
        const int64_t l0 = launch_count();
        CK(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
        const nbody_status st = forest_step_once(c, d_pos, d_vel, d_mass);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->gstream, &g);
        c->stream = user;
        c->timing = timing;
        const int64_t k = launch_count() - l0;  // recorded, not launched
        count_launches((int)-k);
        if (st != NBODY_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (st != NBODY_OK) return st;
            return fail(c, NBODY_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            c->gexec = nullptr;
            return fail(c, NBODY_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
        }
        c->glaunches = k;
        memcpy(c->gkey, key, sizeof(key));
    }
    CK(cudaEventRecord(c->gev[0], c->stream));
    CK(cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
    for (int32_t s = 0; s < nsteps; ++s) {
        CK(cudaGraphLaunch(c->gexec, c->gstream));
        count_launches((int)c->glaunches);
    }
    CK(cudaEventRecord(c->gev[1], c->gstream));
    CK(cudaStreamWaitEvent(c->stream, c->gev[1], 0));
    c->n_forces = n;
    return NBODY_OK;
}

}  // extern "C"

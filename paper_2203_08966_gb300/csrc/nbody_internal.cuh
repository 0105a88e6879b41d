// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nbody.h"

namespace nb {

constexpr int kBits = 21;          // bits per axis of a Morton key (§4.4)
constexpr int kMaxLevel = 21;      // deepest octree level; cells there are buckets
constexpr int kLevels = 22;        // levels 0..21
constexpr uint32_t kQMax = 2097151u;

// Sorted body or tree node in FP64: (x, y, z, m).
struct alignas(32) D4 {
    double x, y, z, w;
};

// What the FP32 walk reads per node (32 bytes, two 16-byte loads).
//   c      centre of mass minus the box centre (FP32), c.w = G * m
//   skip   pre-order index of the first node after this node's subtree
//   first  sorted index of the node's first body
//   count  0 for an internal cell; number of bodies for a leaf (1, or > 1 for a level-21 bucket)
//   crit   internal cells: l^2 / theta^2 of the node's level, +inf when theta == 0
struct alignas(16) WalkNode {
    float4 c;
    int skip;
    int first;
    int count;
    float crit;
};

// Root box on the device.
struct Box {
    double o[3];      // min corner
    double L;         // cube side
    double s;         // 2^21 / L
    double c[3];      // origin of the FP32 coordinates: the centre of mass
};

// Morton keys (§4.4): q = clamp(floor((x - o) * s), 0, 2^21 - 1) per axis, then the bits of
// q_x, q_y, q_z interleaved with x most significant (a 63-bit key in one 64-bit word).
// floor((x - o) * s) clamped to [0, 2^21 - 1], the subtraction and the product each rounded to
// nearest.  The conversion rounds down and saturates (negative and NaN give 0, values past the
// unsigned range its maximum), so the clamp is one integer min.
__device__ __forceinline__ uint32_t quantise(double x, double o, double s)
{
    const double t = __dmul_rn(__dsub_rn(x, o), s);
    return min(__double2uint_rd(t), kQMax);
}

// Spreads the low 21 bits of v so that bit b lands on bit 3b.
__device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x001f00000000ffffull;
    v = (v | (v << 16)) & 0x001f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint64_t morton_key(double x, double y, double z, const Box &b)
{
    const double s = b.s;
    return (spread3(quantise(x, b.o[0], s)) << 2) | (spread3(quantise(y, b.o[1], s)) << 1) |
           spread3(quantise(z, b.o[2], s));
}

// Device error word bits.
enum : int { kErrNodeCap = 1, kErrTimeout = 2, kErrStack = 4, kErrInput = 8 };

// Per-level tables written with the box.
struct LevelTables {
    double l2[kLevels];      // (L / 2^level)^2
    float crit32[kLevels];   // l2 / theta^2 as FP32 (+inf when theta == 0)
};

// The systems of a forest.  sys[i] is the system of body i; the bodies of system k are
// start[k] .. start[k+1] - 1, both in the caller's order and in sorted order (the sort keeps every
// body inside its system's range).  A single system is {nullptr, nullptr, 1}.
struct Systems {
    const uint16_t *sys;
    const int *start;
    int count;
};
constexpr int kMaxSystems = 65535;

// FP64 precisions (the bit-exact and the fast form share the FP64 tree and acceptance test).
inline bool is_fp64(int precision)
{
    return precision == NBODY_FP64 || precision == NBODY_FP64_FAST;
}

// Process-wide count of kernel launches made by the library (every launcher adds its launches).
void count_launches(int k);
int64_t launch_count();

// ---------------------------------------------------------------- build_kernels.cu
int bbox_blocks(int64_t n);
int bbox_partial_doubles();  // doubles per block in the partials buffer
// aos: the bodies as (x, y, z, m) records in the caller's order, written for the permutation
// (may be null for launch_bbox_partials).
void launch_bbox_partials(const double *pos, const double *mass, int n, double *partials,
                          int nblk, D4 *aos, cudaStream_t s);
void launch_kick_drift_bbox(double *pos, double *vel, const double *acc, const double *mass,
                            int n, double h, double dt, double *partials, int nblk, D4 *aos,
                            bool fused, cudaStream_t s);
void launch_bbox_finalize(const double *partials, int nblk, Box *box, LevelTables *tab,
                          double theta, cudaStream_t s);
constexpr int kForestBoxChunk = 4096;  // forest: bodies per partial-box block
// Forest: a step's kick and drift (vel non-null) fused with the per-system root boxes (chunks of
// at most kForestBoxChunk bodies inside one system, partial boxes per chunk, then one block per
// system), writing the (x, y, z, m) records.
void launch_forest_boxes(double *pos, double *vel, const double *acc, const double *mass, int n,
                         const int4 *chunks, int nchunks, const int *chunk_start, int n_sys,
                         double h, double dt, double *partials, Box *box, LevelTables *tab,
                         double theta, D4 *aos, bool fused, cudaStream_t s);
// gate (may be null): a device count; the kernel does nothing when it is 0.
void launch_keys(const double *pos, int n, const Box *box, const Systems &ss, uint64_t *keys,
                 uint32_t *ids, cudaStream_t s, const int *gate = nullptr);

// Radix sort geometry (build_kernels.cu): keys per tile, key passes, and rows of digit totals
// (8 key passes, up to 4 passes on id bytes, 2 on the system of a forest's bodies).
constexpr int kSortTileKeys = 4096;
constexpr int kSortKeyPasses = 8;
constexpr int kSortHistRows = 14;

struct SortScratch {
    uint64_t *keys_alt;
    uint32_t *ids_alt;
    uint32_t *hist;       // 14 x 256 digit totals (8 key passes, up to 4 id passes, 2 system
                          // passes of a subset of a forest's bodies)
    uint32_t *counts;     // 256 x tiles
    int max_tiles;
    const uint16_t *sys;  // forest: two more stable passes on the system of every id
    const uint32_t *sys_hist;  // their digit totals (2 x 256, fixed per forest); null with sys:
                               // counted from the data (the sort of a subset of the bodies)
    const int *d_n = nullptr;  // non-null: the pair count is read on the device (at most n)
};
int sort_tiles(int n);
cudaError_t sort_prepare(); // one-time function attributes
void launch_radix_sort(uint64_t *keys, uint32_t *ids, int n, const SortScratch &sc,
                       cudaStream_t s);
// Sort of (key, id) pairs by key, then id, for ids in no particular order (ids < 2^id_bits):
// passes on the id bytes first, then the key passes.  The sorted pairs end in (keys, ids) or in
// (sc.keys_alt, sc.ids_alt); *out_keys / *out_ids say which.
void launch_radix_sort_key_id(uint64_t *keys, uint32_t *ids, int n, int id_bits,
                              const SortScratch &sc, cudaStream_t s, uint64_t **out_keys,
                              uint32_t **out_ids);

// Sets *flag (kErrInput bits, OR-ed) when a position or mass of the n bodies is NaN or infinite.
void launch_check_finite(const double *pos, const double *mass, int n, int *flag, cudaStream_t s);

void launch_permute(const D4 *aos, const uint32_t *ids, int n, const Box *box, const Systems &ss,
                    double G, D4 *sbody64, float4 *sbody32, cudaStream_t s);

struct ScanScratch {
    uint32_t *block_sums;  // tiles + 1
    int max_tiles;
};
int scan_tiles(int len);
void launch_count_nodes(const uint64_t *keys, int n, const Systems &ss, uint32_t *counts,
                        unsigned *max_level, cudaStream_t s);
void launch_exclusive_scan(const uint32_t *in, uint32_t *out, int len, const ScanScratch &sc,
                           cudaStream_t s);

// Node kind byte: the level of an internal cell, kLeafKind for a leaf.
constexpr uint8_t kLeafKind = 0x80;

// Nodes in pre-order (capacity `cap`).  The node count lives on the device (d_nn, the last
// entry of the node offsets); kernels that loop over nodes read it there.
struct NodeArrays {
    WalkNode *wn;
    D4 *com64;
    uint8_t *level;
    uint8_t *mask;
    uint8_t *kind;
    int *order;               // pre-order index -> level-order index
    int *inv;                 // level-order index -> pre-order index
    D4 *com_lo;               // FP64 moments in level order
    // quadrupoles about each node's centre of mass (null unless requested): 6 doubles per node
    // (xx, yy, zz, xy, xz, yz), in level order and in pre-order; FP32 G*Q for the group walk,
    // two float4 per node in level order: (xx, yy, zz, xy), (xz, yz, 0, 0)
    double *q_lo;
    double *q64;
    float4 *gq;
    int4 *lo_child;           // level order: (first child, child count, first body, 0); count 0 = leaf
    int4 *spine;              // FP32 sums: per (level, pre-order tile) the tile's spine cell
    uint32_t *tile_offsets;   // level-major (level, tile) offsets; level l starts at [l * tiles]
    uint32_t *block_sums;     // scan scratch for tile_offsets
    const uint32_t *d_nn;     // node count (device)
    int tiles;                // layout tiles for `cap` nodes
    int64_t cap;
};
// Node split; nodes past `cap` are not written and set kErrNodeCap in *err.
void launch_emit_nodes(const uint64_t *keys, int n, const Systems &ss, const uint32_t *node_off,
                       NodeArrays na, int *err, cudaStream_t s);
// Stable partition of the nodes by level (order, inv, per-level starts).
void launch_level_order(const NodeArrays &na, cudaStream_t s);
// Child masks, node kinds, leaf moments, then the internal cells level by level (levels
// max_level - 1 .. 0) up to the roots.
void launch_moments(const uint64_t *keys, int max_level, const D4 *sbody64, const Box *box,
                    const LevelTables *tab, const Systems &ss, double G, NodeArrays na,
                    cudaStream_t s);

// Level-order copy of the octree read by the FP32 group walk.  Nodes are ordered by level, and
// within a level in pre-order (= Morton order), so the children of a cell are contiguous:
// children of node b are child .. child + n - 1.
//   c      as WalkNode::c
//   child  internal: level-order index of the first child; leaf: sorted index of its first body
//   n      internal: number of children (1..8); leaf: -(number of bodies)
//   crit   internal: l^2 / theta^2 as FP32 (+inf when theta == 0); leaf: 0
//   pre    pre-order index of the same node
struct alignas(16) GroupNode {
    float4 c;
    int child;
    int n;
    float crit;
    int pre;
};

// Node indices of the group walk's stack entries have 28 bits.
constexpr int64_t kMaxGroupNodes = (int64_t)1 << 28;

int layout_tiles(int64_t n_nodes);
int layout_scan_len(int64_t n_nodes);
// GroupNode records at their level-order positions (after the moments); a cell's FP32 centre of
// mass relative to its system's origin and its level's FP32 threshold are made here.
void launch_group_nodes(const NodeArrays &na, const Box *box, const LevelTables *tab,
                        const Systems &ss, double G, GroupNode *gn, cudaStream_t s);
// FP32 contexts without quadrupoles: every node's FP64 sums (sum m x, sum m y, sum m z, sum m),
// its child mask, and its GroupNode record with the FP32 centre of mass formed from those sums
// (one FP64 reciprocal per node); one pass over pre-order tiles, then the tiles' spine cells
// level by level (levels max_level - 1 .. 0).  com_lo receives the sums the spine cells read, or
// every node's with all_sums (nbody_get_moments).  lo_child, kind and com64 are not written.
int subtree_tiles(int64_t cap);
void launch_subtree_sums(const uint64_t *keys, int max_level, const D4 *sbody64,
                         const float4 *sbody32, const Box *box, const LevelTables *tab,
                         const Systems &ss, double G, NodeArrays na, GroupNode *gn,
                         bool all_sums, cudaStream_t s);
// Walk groups that follow the tree: every cell of at most gmax bodies whose parent holds more
// (consecutive such siblings merged while they fit in gmax), buckets of more than gmax bodies cut
// into chunks.  (first body, count, system, 0) entries, *ngroups of them (zeroed by the caller);
// more than cap entries set kErrNodeCap.
void launch_cell_groups(const NodeArrays &na, const uint32_t *node_off, const Systems &ss, int n,
                        int gmax, int4 *groups, unsigned *ngroups, int64_t cap, int *err,
                        cudaStream_t s);
// Forest: *nn = *total when it fits in cap nodes, else 0 with kErrNodeCap set.
void launch_clamp_count(const uint32_t *total, int64_t cap, uint32_t *nn, int *err,
                        cudaStream_t s);
// Forest: level-order index of every system's root.
void launch_roots(const NodeArrays &na, const uint32_t *node_off, const Systems &ss, int *roots,
                  cudaStream_t s);

// ---------------------------------------------------------------- order_kernels.cu
// Re-sort from the previous step's order (§4.4): bodies move little in one step, so last step's
// sorted list is almost sorted.  The result equals the stable sort by (system, key, caller's
// index):
//   extract  keys of the bodies in the previous order (gathered through its permutation); every
//            body in a descent of that sequence is removed, repeatedly, until the rest ascends
//            (inside tiles in shared memory, then across tile seams); then the device decides:
//            re-sort, or (the seam repair gave up, or with auto_limit more than a quarter of the
//            bodies were removed) the full sort;
//   merge    the removed bodies are sorted by (system, key, id) and merged with the kept ones.
// Nothing is read back to the host: the kernels of the path not taken return at once, so a step
// can be captured in a CUDA graph.
struct OrderScratch {
    uint32_t *keep;      // one bit per position of the previous order: still in the ascending rest
    int2 *ends;          // per tile: first and last kept position (-1: none)
    uint32_t *seams;     // one bit per tile: the seam before it needs the fix-up
    uint32_t *kept_off;  // per tile: kept positions before it
    unsigned *stats;     // kOrder* words
    int *split;          // merge path: kept bodies before each merge tile
    uint64_t *rk, *xk;   // kept / removed keys
    uint32_t *ri, *xi;   // their ids
};
enum : int {
    kOrderKept = 0,      // kept positions
    kOrderSeams = 1,     // tile seams flagged for the repair
    kOrderGaveUp = 2,    // the repair ran out of steps
    kOrderRemoved = 3,   // removed positions
    kOrderXn = 4,        // removed positions when re-sorting, else 0 (count of the removed sort)
    kOrderFullN = 5,     // n when the full sort runs instead, else 0
    kOrderResorted = 6,  // 1: re-sorted
    kOrderStats = 8
};
int order_tiles(int n);        // extract tiles (entries of ends and kept_off)
int order_merge_tiles(int n);  // merge tiles (split has one more entry)
// keys: out, the keys in the previous order (read again by launch_order_merge).  prev: the
// previous sorted ids.  auto_limit: fall back to the full sort above a quarter removed.
void launch_order_extract(const D4 *aos, const uint32_t *prev, int n, const Box *box,
                          const Systems &ss, bool auto_limit, uint64_t *keys,
                          const OrderScratch &o, cudaStream_t s);
// Leaves the sorted keys and ids in (keys, ids) when the device chose the re-sort; sc is the
// radix sort's scratch (sorts the removed bodies).
void launch_order_merge(uint64_t *keys, uint32_t *ids, int n, const Systems &ss,
                        const OrderScratch &o, const SortScratch &sc, cudaStream_t s);
// Device count for the full sort's kernels: n when the device chose the full sort, else 0.
inline const int *order_full_count(const OrderScratch &o)
{
    return reinterpret_cast<const int *>(o.stats + kOrderFullN);
}

// ---------------------------------------------------------------- probe_kernels.cu
// The FP32 fused multiply-add rate of the current device in TFLOP/s (a timed kernel of
// independent FMA chains on every SM; the call waits for it).
cudaError_t measure_fp32_rate(cudaStream_t s, double *tflops);
// The same for FP64 fused multiply-adds.
cudaError_t measure_fp64_rate(cudaStream_t s, double *tflops);

// ---------------------------------------------------------------- walk_kernels.cu
struct WalkArgs {
    const WalkNode *wn;
    const D4 *com64;
    const uint8_t *level;
    const LevelTables *tab;
    const D4 *sbody64;
    const float4 *sbody32;
    const uint32_t *ids;
    int n;
    double G, eps, theta;
    double *acc;          // 3n, user order (written)
    double *vel;          // 3n, user order, kicked by acc*h when non-null
    double h;
    uint32_t *pp, *pc;    // n, sorted order
    const GroupNode *gn;  // level-order tree (FP32 walks)
    int *err;             // device error word (kErrStack)
    const uint32_t *d_nn; // node count (device)
    // forest: the walk runs over groups of <= 32 bodies of one system each
    const int4 *groups;   // (first body, count, system, 0); null for a single system
    int n_groups;
    const int *roots;     // level-order index of each system's root
    const uint32_t *node_off;  // pre-order: nodes of system k are node_off[start[k]] ..
    const int *start;     // system starts (bodies)
    bool group_mac;       // FP32 walks: grouped acceptance test (NBODY_FLAG_GROUP_MAC)
    const double *q64;    // quadrupoles (pre-order) for the FP64 walk, null without them
    const float4 *gq;     // G * quadrupoles (level order) for the FP32 walk, null without them
    const unsigned *d_ngroups;  // groups built on the device: their count (n_groups = capacity)
    unsigned *work;       // FP32 walk: group counters of the persistent warps (2, zeroed per launch)
    // spans of kSpanBodies consecutive bodies sharing one far walk (single systems, per-body
    // test, monopole cells); span_meta null: every group walks from the root
    int4 *span_meta;      // per span: far count (-1: walk from the root), frontier count, far
                          // leaves, far cells
    uint32_t *span_off;   // per span: offset of its far list (then its frontier) in span_pool
    uint32_t *span_pool;  // level-order node indices
    int64_t span_pool_cap;
    uint32_t *span_tmp;   // per far-walk warp: kSpanFarTmp + 2 kSpanFrTmp words
    unsigned *span_next;  // [0] pool words handed out, [1] span counter (zeroed per launch)
    int span_bodies;      // bodies per span (a multiple of 32)
    // test aid (nbody_set_walk_limits): stack entries a group walk may use (at most the
    // kernel's capacity) and steps per group or span (at most the node count)
    int stack_limit;
    int64_t step_limit;
    int fast_stack_limit; // test aid: stack entries of the fast per-body walk (at least 64)
    // FP32 per-body walk: groups whose stack outgrew the fast walk's, walked afterwards with the
    // full stack ((first body, count, system, 0), as many entries as groups); null: none
    int4 *overflow;
    unsigned *n_overflow;
};
// Spans of the shared far walk: groups of 32 bodies, span_bodies (128, 256 or 512) per span.  A
// span's far list holds at most kSpanFarTmp nodes and its frontier at most kSpanFrTmp (else its
// groups walk from the root).
constexpr int kSpanMinBodies = 128;
constexpr int kSpanFarTmp = 8192;
constexpr int kSpanFrTmp = 2048;
// Far-walk warps launched (the span_tmp slices needed), for n bodies in spans of span_bodies.
int span_far_warps(int n, int span_bodies);
// Launch shapes of the walks; results do not depend on the shape.  FP64 walks: shapes 0, 1, 2
// are 64, 128, 256 threads per block (the others run as 1).  FP32 walks: walk_shape32; the
// grouped acceptance test and quadrupole cells use only its warps per block, forests neither
// spans nor (shapes 3..5) anything but shape 1.
struct WalkShape {
    int warps;         // warps (groups) per block
    int span_bodies;   // bodies per span of the shared far walk; 0: every group from the root
    int buf;           // interaction-buffer entries (64 or 128)
    bool cell_groups;  // groups follow the tree's cells (as NBODY_FLAG_CELL_GROUPS)
};
constexpr int kWalkShapes = 8;
constexpr int kDefaultWalkShape = 1;
WalkShape walk_shape32(int shape);
int walk_shape_threads(int precision, int shape);
cudaError_t walk_prepare();  // one-time function attributes (dynamic shared memory)
void launch_walk(int precision, const WalkArgs &a, int shape, cudaStream_t s);

// FP32 direct sum scratch: FP32 sources (n) and per-chunk partial sums
// (direct32_chunks(n, nt) x 3 x nt floats).
struct DirectScratch {
    float4 *src;
    float *part;
};
int direct32_chunks(int n, int nt);
void launch_direct(int precision, const double *pos, const double *mass, int n,
                   const int64_t *targets, int nt, double G, double eps, const Box *box,
                   double *acc, const DirectScratch &sc, cudaStream_t s);

}  // namespace nb

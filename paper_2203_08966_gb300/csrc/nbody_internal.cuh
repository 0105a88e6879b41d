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

// Device error word bits.
enum : int { kErrNodeCap = 1, kErrTimeout = 2, kErrStack = 4 };

// Per-level tables written with the box.
struct LevelTables {
    double l2[kLevels];      // (L / 2^level)^2
    float crit32[kLevels];   // l2 / theta^2 as FP32 (+inf when theta == 0)
};

// Process-wide count of kernel launches made by the library (every launcher adds its launches).
void count_launches(int k);
int64_t launch_count();

// ---------------------------------------------------------------- build_kernels.cu
int bbox_blocks(int64_t n);
int bbox_partial_doubles();  // doubles per block in the partials buffer
void launch_bbox_partials(const double *pos, const double *mass, int n, double *partials,
                          int nblk, cudaStream_t s);
void launch_kick_drift_bbox(double *pos, double *vel, const double *acc, const double *mass,
                            int n, double h, double dt, double *partials, int nblk,
                            cudaStream_t s);
void launch_bbox_finalize(const double *partials, int nblk, Box *box, LevelTables *tab,
                          double theta, cudaStream_t s);
void launch_keys(const double *pos, int n, const Box *box, uint64_t *keys, uint32_t *ids,
                 cudaStream_t s);

struct SortScratch {
    uint64_t *keys_alt;
    uint32_t *ids_alt;
    uint32_t *hist;       // 8 x 256 digit totals
    uint32_t *counts;     // 256 x tiles
    int max_tiles;
};
int sort_tiles(int n);
cudaError_t sort_prepare(); // one-time function attributes
void launch_radix_sort(uint64_t *keys, uint32_t *ids, int n, const SortScratch &sc,
                       cudaStream_t s);

void launch_permute(const double *pos, const double *mass, const uint32_t *ids, int n,
                    const Box *box, double G, D4 *sbody64, float4 *sbody32, cudaStream_t s);

struct ScanScratch {
    uint32_t *block_sums;  // tiles + 1
    int max_tiles;
};
int scan_tiles(int len);
void launch_count_nodes(const uint64_t *keys, int n, uint32_t *counts, unsigned *max_level,
                        cudaStream_t s);
void launch_exclusive_scan(const uint32_t *in, uint32_t *out, int len, const ScanScratch &sc,
                           cudaStream_t s);

// Node kind byte: the level of an internal cell, kLeafKind for a leaf.
constexpr uint8_t kLeafKind = 0x80;

struct NodeArrays {
    WalkNode *wn;
    D4 *com64;
    uint8_t *level;
    uint8_t *mask;
    uint8_t *kind;
    int *level_list;          // internal cells grouped by level (cap entries)
    unsigned *level_count;    // kLevels counters
    unsigned *level_start;    // kLevels + 1 offsets into level_list
    unsigned *level_cursor;   // kLevels scatter cursors
    int64_t cap;
};
void launch_emit_nodes(const uint64_t *keys, int n, const uint32_t *node_off, NodeArrays na,
                       cudaStream_t s);
// Child masks, node kinds, leaf moments, then the internal cells level by level up to the root.
void launch_moments(const uint64_t *keys, int n_nodes, int max_level, const D4 *sbody64,
                    const Box *box, const LevelTables *tab, double G, NodeArrays na,
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

struct LayoutScratch {
    uint32_t *tile_offsets;  // kLevels x tiles (+1), level-major
    uint32_t *block_sums;    // scan scratch for the tile offsets
    int *order;              // pre-order index -> level-order index
    int max_tiles;
};
int layout_tiles(int64_t n_nodes);
int layout_scan_len(int64_t n_nodes);
// Stable partition of the nodes by level, then the GroupNode records.
void launch_level_order(const NodeArrays na, int n_nodes, const LayoutScratch &ls,
                        GroupNode *gn, cudaStream_t s);

// ---------------------------------------------------------------- walk_kernels.cu
struct WalkArgs {
    const WalkNode *wn;
    const D4 *com64;
    const uint8_t *level;
    const LevelTables *tab;
    int n_nodes;
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
};
void launch_walk(int precision, const WalkArgs &a, cudaStream_t s);

void launch_direct(int precision, const double *pos, const double *mass, int n,
                   const int64_t *targets, int nt, double G, double eps, const Box *box,
                   double *acc, cudaStream_t s);

}  // namespace nb

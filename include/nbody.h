/*
 * nbody.h -- C ABI of the GB300 Barnes-Hut timestep library (libnbody.so).
 *
 * Method: A. Brandt, "On Distributed Gravitational N-Body Simulations" (arXiv 2203.08966).
 * One call advances or evaluates one gravitational system on one GPU:
 *   octree build  (§3 and Algorithm 2 "Build Tree"; Morton keys of §4.4; the tree is the
 *                  uncompressed octree whose leaves hold one body, or several bodies that share
 *                  one level-21 cell),
 *   moments       (Algorithm 2: total mass and centre of mass from the leaves to the root;
 *                  eq. `approxforce` of §2.1),
 *   traversal     (Algorithm 2 "Compute Cell Force": for every body, the children of each
 *                  opened cell are visited in Morton order; a leaf gives particle-particle
 *                  interactions, a cell with side l and centre-of-mass distance d is accepted
 *                  when l/d < theta, evaluated as l*l < theta*theta*d*d, else it is opened;
 *                  the root itself is never tested),
 *   softened pair kernel  (eq. `motion` of §2.1 with |r|^2 replaced by |r|^2 + eps^2),
 *   leapfrog      (kick-drift-kick, eqs. `leapkick1`, `leapdrift`, `leapkick2` of §2.4).
 *
 * Conventions shared by every entry point
 *   - Array layout is structure-of-arrays float64: pos = [x_0..x_{N-1} | y_0.. | z_0..] (3N
 *     doubles), vel likewise, mass[N], acc[3N].  Bodies are in the caller's order ("user
 *     order") on input and output; the library reorders internally.
 *   - Pointers named d_* are DEVICE pointers on the context's device; h_* are HOST pointers.
 *     The caller owns every buffer it passes and must keep it alive until the call's work on
 *     the context stream has completed; the library never frees caller memory.
 *   - All work is enqueued on the context's CUDA stream.  Entry points that must read a
 *     device-side size (the node count of the tree) synchronise that stream once per build,
 *     and once more when the build re-sorts from the previous order (the device's choice of
 *     path, see nbody_set_sort_mode); every other call returns without waiting.  Results in device buffers are valid once the
 *     stream has reached the call; nbody_sync() waits for it and reports device-side errors.
 *   - Errors are returned as nbody_status codes; nbody_last_error() gives a one-line message.
 *     A failed call leaves caller buffers in an unspecified state but the context usable,
 *     except after NBODY_ECUDA, after which the context should be destroyed.
 *   - Preconditions: n <= n_capacity; masses positive and finite; positions finite;
 *     theta >= 0, eps >= 0, G and dt finite.  Violations found on the host give NBODY_EINVAL.
 *   - Contexts are not thread-safe: one host thread at a time per context.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nbody_ctx nbody_ctx;

typedef enum {
    NBODY_OK = 0,
    NBODY_EINVAL = 1,    /* bad argument (null pointer, size, parameter) */
    NBODY_ENOMEM = 2,    /* device or host allocation failed */
    NBODY_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    NBODY_ESTACK = 4,    /* a walk ran out of stack entries or steps (reported by nbody_sync) */
    NBODY_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    NBODY_ESTATE = 6     /* call out of order (e.g. introspection before any build) */
} nbody_status;

typedef enum {
    NBODY_FP64 = 0,        /* pair interactions, walk and accumulation in FP64 */
    NBODY_FP32 = 1,        /* FP32 pair interactions, MAC and accumulation */
    NBODY_FP32_KAHAN = 2,  /* FP32 pair interactions with compensated (Kahan) accumulation */
    NBODY_FP64_FAST = 3    /* FP64 with the FP64 acceptance test of NBODY_FP64 (the same
                            * interaction lists and counters) but each pair term evaluated with
                            * fused multiply-adds and one reciprocal square root (rsqrt) instead
                            * of separately rounded operations, a square root and a division:
                            * results differ from NBODY_FP64 by rounding */
    /* FP64 sums each body's terms in the order of its own recursive walk.  The FP32 forms give
     * every body the interaction list that the per-body FP32 acceptance test decides, but
     * evaluate the walk for 32 Morton-consecutive bodies at a time and sum the terms in another
     * order; their trees may hold at most 2^28 nodes (EINVAL beyond). */
} nbody_precision;

/* Physical and numerical parameters.  G: gravitational constant; eps: Plummer softening length
 * (§2.1); theta: opening angle of the acceptance test l/d < theta (§3); dt: leapfrog time step
 * (§2.4); precision: nbody_precision; flags: a combination of NBODY_FLAG_GROUP_MAC and
 * NBODY_FLAG_CELL_GROUPS (FP32 forms only), NBODY_FLAG_QUADRUPOLE and NBODY_FLAG_CHECK_FINITE,
 * or 0. */
/* Flag: the grouped acceptance test of Barnes (1990) instead of the paper's per-body test
 * (FP32 forms only; EINVAL with NBODY_FP64).  Bodies are taken in Morton order in groups of 32;
 * a cell is accepted for all bodies of a group when l/d_min < theta, d_min being the distance
 * from its centre of mass to the group's bounding box, and opened for all of them otherwise.
 * Every body then sums a superset-refinement of its own per-body list: at least as many
 * interactions, a smaller force error, different results and counters. */
#define NBODY_FLAG_GROUP_MAC 1u

/* Flag: the FP32 walk groups bodies by the tree's cells instead of in consecutive chunks of 32
 * (FP32 forms only).  A group is a cell of at most 32 bodies whose parent holds more, with
 * consecutive such siblings merged while they fit in 32, so a group never straddles a jump of
 * the Morton curve.  Results are unchanged (each body keeps its own interaction list); only the
 * summation order and the speed differ.  Always on with NBODY_FLAG_GROUP_MAC, whose shared lists
 * need compact groups. */
#define NBODY_FLAG_CELL_GROUPS 2u

/* Flag: accepted cells add their quadrupole term (§2.2, the truncated multipole expansion about
 * the cell's centre of mass, where the dipole vanishes), softened like the monopole: with
 * d = r_J - r_i and r_s^2 = |d|^2 + eps^2,
 *   a_i += G (M d / r_s^3 - Q d / r_s^5 + 5/2 (d.Q.d) d / r_s^7),
 *   Q_ab = sum_j m_j (3 x_a,j x_b,j - r_j^2 delta_ab) over the cell's bodies.
 * All precisions.  The same cells are accepted (counters unchanged); forces are more accurate.
 * Quadrupoles are built bottom-up (parallel-axis sums), so the FP64 path matches a body-by-body
 * evaluation to rounding rather than bit for bit. */
#define NBODY_FLAG_QUADRUPOLE 4u

/* Flag: every build first checks that all positions and masses are finite (one extra pass over
 * them).  A single-system call that finds a NaN or an infinity returns NBODY_EINVAL before the
 * node split and the walk; a forest step, which never waits on the host, reports it at the next
 * nbody_sync.  Without the flag non-finite inputs are a precondition violation: the library
 * still keeps every access in bounds, but the results are undefined. */
#define NBODY_FLAG_CHECK_FINITE 8u

typedef struct {
    double G;
    double eps;
    double theta;
    double dt;
    int32_t precision;
    uint32_t flags;
} nbody_params;

/* One node of the octree in the paper's pre-order serialisation (§4.2) with its hashed-octree
 * key (§4.7: root key 1, child key = parent key << 3 | octant, octant digit = 4x + 2y + z).
 * first = rank of the node's first body in Morton order, count = bodies in its subtree. */
typedef struct {
    uint64_t key;
    int32_t level;
    int32_t child_mask;   /* bit c set when octant c has a child */
    int64_t first;
    int64_t count;
} nbody_tree_record;

/* Creates a context on the current CUDA device for systems of up to n_capacity bodies.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).  Allocates the per-body
 * working set (about 120 bytes per body plus the tree, which is grown on demand).
 * Errors: EINVAL (out == NULL, n_capacity < 0 or > 2^30, bad params), ENOMEM, ECUDA. */
nbody_status nbody_create(nbody_ctx **out, int64_t n_capacity, const nbody_params *p,
                          void *cuda_stream);

/* Releases all device and host memory of the context after its stream has drained. */
nbody_status nbody_destroy(nbody_ctx *c);

/* Replaces the parameters; the next nbody_step recomputes the starting acceleration. */
nbody_status nbody_set_params(nbody_ctx *c, const nbody_params *p);

/* Builds the octree of d_pos/d_mass (n bodies): root box, Morton keys, sort, node split and
 * moments (Algorithm 2, "Build Tree" and the leaves-to-root pass).  Synchronises the stream
 * once to learn the node count (twice when it re-sorts from the previous build's order).
 * Errors: EINVAL, ENOMEM (tree larger than the device can hold), ECUDA. */
nbody_status nbody_build_tree(nbody_ctx *c, const double *d_pos, const double *d_mass,
                              int64_t n);

/* Barnes-Hut accelerations of all bodies (Algorithm 2): builds the tree of d_pos/d_mass and
 * writes d_acc (3n doubles, user order) in the context's precision.  Per-body interaction
 * counters (pp: particle-particle, pc: particle-cell; Algorithm 9 counts pp + 2 pc) are kept
 * for nbody_get_counters.  Errors as nbody_build_tree. */
nbody_status nbody_forces(nbody_ctx *c, const double *d_pos, const double *d_mass, int64_t n,
                          double *d_acc);

/* Advances d_pos/d_vel in place by nsteps kick-drift-kick steps of the context's dt (§2.4):
 * v += a dt/2; r += v dt; a = BH(r); v += a dt/2, in FP64 (FP64 contexts round every product
 * and sum separately, as the oracle does; FP32 contexts take the first kick and the drift as
 * FP64 fused multiply-adds).  The acceleration at the current positions
 * is kept in the context between calls; the first call after create, set_params or a change
 * of n computes it first.  Synchronises once per step (node count), twice when the step
 * re-sorts from the previous order.  nsteps >= 0. */
nbody_status nbody_step(nbody_ctx *c, double *d_pos, double *d_vel, const double *d_mass,
                        int64_t n, int32_t nsteps);

/* nbody_step on HOST buffers (the call is synchronous).  Copies h_pos, h_vel, h_mass (and
 * h_acc) to the device, runs nsteps kick-drift-kick steps and copies h_pos, h_vel (and h_acc)
 * back before returning.  h_acc (3n doubles, in/out, may be NULL): on entry the acceleration
 * at h_pos, as left by the previous call, so the first kick needs no force evaluation; on exit
 * the acceleration at the new positions.  With h_acc == NULL the acceleration at h_pos is
 * computed first.  Page-locked host buffers give the fastest copies.  The device copies are
 * scratch owned by the context and allocated on the first call. */
nbody_status nbody_step_host(nbody_ctx *c, double *h_pos, double *h_vel, double *h_acc,
                             const double *h_mass, int64_t n, int32_t nsteps);

/* Direct-sum accelerations (Algorithm 1) of nt target bodies against all n sources, in the
 * context's precision (FP32_KAHAN runs as FP32).  d_targets: device int64 user indices, or NULL
 * for all n bodies (then nt is ignored).  d_acc: 3*nt doubles, row-major (x row, y row, z row).
 * Sources are summed in ascending index order; a target never interacts with itself. */
nbody_status nbody_direct_forces(nbody_ctx *c, const double *d_pos, const double *d_mass,
                                 int64_t n, const int64_t *d_targets, int64_t nt, double *d_acc);

/* Waits for the context stream and reports the device-side error word set since the last
 * report: EINVAL (NBODY_FLAG_CHECK_FINITE found a NaN or infinite input in a forest step),
 * ENOMEM (a forest's trees outgrew the node arrays), ESTACK (a walk ran out of stack entries or
 * steps: a malformed tree, or limits lowered by nbody_set_walk_limits).  The word is cleared once
 * reported; the context stays usable, and the next nbody_step recomputes its starting
 * acceleration. */
nbody_status nbody_sync(nbody_ctx *c);

/* ---- introspection (copies to caller-provided HOST buffers; synchronous) ---- */

/* Sorted Morton keys and the user index of each sorted body, from the last build
 * (n entries each).  Errors: ESTATE before any build. */
nbody_status nbody_get_keys(nbody_ctx *c, uint64_t *h_keys_sorted, uint32_t *h_ids_sorted);

/* Root box of the last build: h_box[0..2] = min corner, [3] = side L, [4] = 2^21 / L. */
nbody_status nbody_get_box(nbody_ctx *c, double *h_box);

/* Pre-order node records of the last build.  Writes *n_nodes; fills h_records when
 * h_records != NULL and cap >= *n_nodes (else only *n_nodes is written). */
nbody_status nbody_get_tree(nbody_ctx *c, int64_t *n_nodes, nbody_tree_record *h_records,
                            int64_t cap);

/* FP64 moments of the last build, pre-order: h_out[4*k .. 4*k+3] = (m, x, y, z) of node k.
 * FP64 contexts (and quadrupole contexts) form every cell's centre of mass from its children's
 * as the oracle does, bit for bit; the other FP32 contexts build from FP64 sums (sum m, sum m r,
 * a cell adding its children's in octant order), so their masses are the oracle's bit for bit
 * and their centres of mass, sum m r / sum m, differ from its means by rounding.  Those contexts
 * keep only the sums their build reads, so this call runs the sums pass again on the same tree
 * (on the context's stream, synchronised) before copying them. */
nbody_status nbody_get_moments(nbody_ctx *c, double *h_out, int64_t cap_nodes);

/* Interaction counters of the last force evaluation, user order (n entries each). */
nbody_status nbody_get_counters(nbody_ctx *c, uint32_t *h_pp, uint32_t *h_pc);

/* Device time in milliseconds of the phases of the last build/force/step call (for
 * nbody_step: of its last step; for a forest, of its last nbody_forest_forces), measured with
 * CUDA events recorded on the context stream: [0] kick/drift + box + keys (re-sort: + the
 * extract phase), [1] sort (radix sort, or the re-sort's merge phase), [2] permutation + node
 * split + moments, [3] walk, [4] whole call.  Recorded only while timing is enabled with
 * nbody_enable_timing; nbody_get_timings waits for the last call's final event. */
nbody_status nbody_enable_timing(nbody_ctx *c, int32_t on);
nbody_status nbody_get_timings(nbody_ctx *c, float *h_ms5);

/* Number of kernel launches the library has made in this process (all contexts), so callers
 * can count the launches inside a timed region.  Errors: EINVAL when out == NULL. */
nbody_status nbody_get_launch_count(int64_t *out);

/* ---- launch-shape autotuning of the walk ---- */

/* Number of launch shapes of the walk.  Every shape gives every body the same interaction list
 * (the same counters); FP64 results are identical in every shape, while the FP32 forms' sums can
 * differ in rounding between shapes that group or buffer the terms differently (3 .. 7).
 * FP64 forms: shapes 0, 1, 2 are 64, 128, 256 threads per block (the other shapes run as 1).
 * FP32 forms (one warp per group of 32 bodies; interaction buffers of 128 entries unless noted):
 *   0, 1, 2  2, 4, 8 warps per block, spans of 256 bodies sharing one walk of the far field
 *   3        4 warps per block, no shared far walk (every group walks from the root)
 *   4, 5     4 warps per block, spans of 128 and 512 bodies
 *   6        4 warps per block, spans of 256 bodies, interaction buffers of 64 entries
 *   7        4 warps per block, groups that follow the tree's cells (as NBODY_FLAG_CELL_GROUPS)
 * The grouped acceptance test and quadrupole cells take only the warps per block of a shape;
 * forests and NBODY_FLAG_CELL_GROUPS never share far walks. */
#define NBODY_WALK_SHAPES 8

/* Builds the tree of d_pos/d_mass (n bodies; for a forest context n is ignored and the whole
 * forest is used), times the walk in every launch shape that makes a difference for this
 * context (3 walks each after a warm-up, CUDA events on the context stream; the call waits for
 * them) and keeps the fastest: for later walks of n' bodies with floor(log2 n') == floor(log2 n)
 * at the same theta, and as the context's shape for every other size.  h_ms (host, may be NULL):
 * receives the mean time of each shape in ms (NBODY_WALK_SHAPES floats, 0 for the shapes not
 * timed); chosen (may be NULL): the shape kept.  The kept acceleration of nbody_step is
 * recomputed by the next step.  Errors as nbody_forces; on error the shapes are unchanged. */
nbody_status nbody_autotune(nbody_ctx *c, const double *d_pos, const double *d_mass, int64_t n,
                            float *h_ms, int32_t *chosen);

/* Sets the walk shape (0 .. NBODY_WALK_SHAPES - 1) for the context's precision class without
 * timing anything, and forgets the autotuner's choices.  Errors: EINVAL for a shape out of
 * range. */
nbody_status nbody_set_walk_shape(nbody_ctx *c, int32_t shape);

/* The walk shape in use for the context's precision and its threads per block. */
nbody_status nbody_get_walk_shape(nbody_ctx *c, int32_t *shape, int32_t *threads_per_block);

/* Test aid with no counterpart in the paper: lowers the walk's resources so that its guards and
 * its overflow path can be exercised.  stack_entries: stack ranges an FP32 group walk may hold
 * (at least 33; the kernels' own capacity when larger; 0 = that capacity); max_steps: steps one
 * group, span or FP64 warp may take (0 = no limit beyond the node count); fast_entries: stack
 * ranges of the per-body FP32 walk's fast kernel (at least 64; 0 = its 256), past which a group
 * is handed, untouched, to a second walk with the full stack (its sums are then taken in another
 * order; its interaction list is the same).  A walk that reaches stack_entries or max_steps
 * stops before any further memory access, its bodies' forces are left incomplete, and the next
 * nbody_sync returns NBODY_ESTACK.  With the defaults, no valid tree reaches them (the stack holds
 * at most 32 ranges per level, a walk at most one step per node).  Errors: EINVAL (stack_entries
 * in 1..32, max_steps < 0, fast_entries in 1..63). */
nbody_status nbody_set_walk_limits(nbody_ctx *c, int32_t stack_entries, int64_t max_steps,
                                   int32_t fast_entries);

/* ---- re-sort from the previous step's order (temporal coherence, §4.4) ---- */

/* How a build sorts the bodies by (key, index) (forests: by (system, key, index)).  Every mode
 * gives the same order, bit for bit; they differ only in cost.
 *   NBODY_SORT_AUTO    (default) when the context's last build was of the same n, start from
 *                      its sorted order: bodies move little in one step (§4.4), so that order
 *                      is almost sorted.  Every body in a descent of it is taken out (until the
 *                      rest ascends), the bodies taken out are radix-sorted and merged back.
 *                      Used from 65,536 bodies (a forest: in total); when more than a quarter of
 *                      the bodies are taken out the build runs the full sort instead.
 *   NBODY_SORT_FULL    always the full radix sort of the keys.
 *   NBODY_SORT_RESORT  as AUTO from any n > 0 and any number taken out (for tests).
 * Either re-sort falls back to the full sort when its repair of tile seams exceeds its step
 * limit.  The choice between re-sort and full sort is made on the device, so a forest step
 * stays capturable as a CUDA graph (a change of mode recaptures it).  Errors: EINVAL for an
 * unknown mode. */
#define NBODY_SORT_AUTO 0
#define NBODY_SORT_FULL 1
#define NBODY_SORT_RESORT 2
nbody_status nbody_set_sort_mode(nbody_ctx *c, int32_t mode);

/* How the last build sorted: *path (may be NULL) 1 when it re-sorted from the previous order,
 * 0 for the full sort, -1 before any build; *removed (may be NULL) the bodies the re-sort took
 * out of the previous order (-1 when the build ran the full sort without trying).  Waits for the
 * context's stream when the device made the choice. */
nbody_status nbody_get_sort_stats(nbody_ctx *c, int32_t *path, int64_t *removed);

/* ---- forest: many independent systems advanced together ---- */

/* Creates a context for n_systems independent systems packed into one set of arrays: system k
 * owns bodies h_offsets[k] .. h_offsets[k+1] - 1 of every SoA row (h_offsets: HOST array of
 * n_systems + 1 entries, h_offsets[0] == 0, non-decreasing; empty systems are allowed).  Bodies
 * of different systems never interact; each system gets its own root box, octree and walk
 * (§3, Algorithm 2), with the shared parameters p.  All systems are handled by the same kernel
 * launches, and a step synchronises nothing on the host, so it can be replayed as a CUDA graph.
 * The node arrays are sized here for 4 nodes per body plus 22 per system; a step whose trees
 * need more reports ENOMEM at the next nbody_sync.  Errors: EINVAL (bad offsets, n_systems
 * outside 1..65535, total bodies outside 1..2^30, bad params), ENOMEM, ECUDA.  Destroy with
 * nbody_destroy.  The single-system entry points (build_tree, forces, step, step_host,
 * direct_forces, get_tree, get_moments) return ESTATE on a forest context. */
nbody_status nbody_forest_create(nbody_ctx **out, int32_t n_systems, const int64_t *h_offsets,
                                 const nbody_params *p, void *cuda_stream);

/* Barnes-Hut accelerations of every system (d_pos 3N, d_mass N, d_acc 3N doubles, device, user
 * order, N = h_offsets[n_systems]).  Per-body counters and sorted keys are available through
 * nbody_get_counters / nbody_get_keys (keys sorted by system, then key, then index). */
nbody_status nbody_forest_forces(nbody_ctx *c, const double *d_pos, const double *d_mass,
                                 double *d_acc);

/* nsteps kick-drift-kick steps of every system (§2.4), in place on d_pos / d_vel.  The first
 * call (and the first after nbody_set_params) computes the starting accelerations.  use_graph:
 * 0 launches every kernel of every step; 1 captures one step as a CUDA graph on a stream the
 * context owns (again whenever d_pos, d_vel or d_mass differ from the captured ones, after
 * nbody_set_params, or after a change of sort mode) and replays it nsteps times, ordered after the work already on the
 * context stream, with the context stream waiting for the replays.  Timing events are not
 * recorded by replayed steps. */
nbody_status nbody_forest_step(nbody_ctx *c, double *d_pos, double *d_vel, const double *d_mass,
                               int32_t nsteps, int32_t use_graph);

/* ---- allocation-free keys + sort ---- */

/* Largest n accepted by nbody_sort_keys_noalloc. */
#define NBODY_NOALLOC_MAX_N 262144

/* The paper has no counterpart to this entry point: it exists for callers that cannot call
 * cudaMalloc -- runtimes that own a fixed device-memory budget, real-time loops that must not
 * block in the allocator, hosts that forbid allocation after start-up.  It computes what nbody_build_tree
 * followed by nbody_get_keys returns (root box, Morton keys, stable sort by key then id) without
 * a context and without allocating: its working memory is one file-scope device array of about
 * 3.2 MB, which every GPU that loads the library holds until the process exits.
 *   d_pos (3n doubles, SoA) and d_mass (n doubles): device inputs, caller-owned.
 *   d_keys_sorted (n uint64) and d_ids_sorted (n uint32): device outputs, caller-owned; on
 *   return (once the stream reaches the work) they hold the sorted Morton keys and the user
 *   index of every sorted body.
 *   cuda_stream: a cudaStream_t (NULL = the legacy default stream); the call is asynchronous.
 * Errors: NBODY_EINVAL when n < 0, n > NBODY_NOALLOC_MAX_N or a pointer is NULL (n == 0 is a
 * no-op); NBODY_ECUDA when a CUDA call fails, including a CUDA error that earlier work left
 * pending on the calling thread (the call reads and clears the thread's last error).
 * Every call looks up the array's device address (cudaGetSymbolAddress, which enqueues nothing);
 * the first call on each device, and the first after a device reset, also sets a kernel
 * attribute, so make that first call before any stream capture.  Every call on a
 * device shares the one array and leaves its last contents there: calls whose work overlaps on
 * the GPU (different streams, or host threads without ordering) race and must be serialised by
 * the caller. */
nbody_status nbody_sort_keys_noalloc(const double *d_pos, const double *d_mass, int64_t n,
                                     uint64_t *d_keys_sorted, uint32_t *d_ids_sorted,
                                     void *cuda_stream);

/* ---- measurement aid ---- */

/* No counterpart in the paper: the FP32 fused multiply-add rate the current device sustains,
 * in TFLOP/s (2 flops per FMA), from a timed kernel of independent FMA chains on every SM
 * (about 10 ms; enqueued on cuda_stream, NULL = the legacy default stream; the call waits for
 * it).  It is the measured counterpart of the nominal FP32 peak against which the walk's useful
 * FP32 rate is read.  Errors: EINVAL when h_tflops is NULL; ENOMEM, ECUDA. */
nbody_status nbody_measure_fp32_rate(void *cuda_stream, double *h_tflops);

/* No counterpart in the paper: the FP64 fused multiply-add rate of the current device in
 * TFLOP/s (2 flops per FMA), measured like nbody_measure_fp32_rate; the denominator of the FP64
 * walk's and direct sum's useful rates.  Errors: EINVAL when h_tflops is NULL; ENOMEM, ECUDA. */
nbody_status nbody_measure_fp64_rate(void *cuda_stream, double *h_tflops);

/* Copies the last error message (NUL-terminated, truncated to cap bytes). */
nbody_status nbody_last_error(nbody_ctx *c, char *buf, int64_t cap);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */

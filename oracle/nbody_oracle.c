/*
 * CPU oracle for the Barnes-Hut timestep -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-precision-free (FP64 throughout) restatement of what the paper's method
 * computes.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * this library; the product path never calls it and shares no code with it.
 *
 * Built with -ffp-contract=off so every multiply and add is a separately rounded IEEE-754
 * operation in the order written here.
 *
 * Paper: A. Brandt, "On Distributed Gravitational N-Body Simulations" (arXiv 2203.08966).
 *   - Pair acceleration, eq. `motion` (§2.1), with Plummer softening (§2.1, after eq. `motion`).
 *   - Cell (monopole) approximation, eq. `approxforce` (§2.1); centre of mass read as
 *     r_J = sum_j m_j r_j / m_J (the printed formula drops the division by m_J).
 *   - Direct sum, Algorithm 1.
 *   - Barnes-Hut loop body, Algorithm 2: insertion build with splitting, moments leaves->root,
 *     per-particle walk over the children of each opened node with the test l/d < theta.
 *   - Work counters: +1 per particle-particle, +2 per particle-cell interaction (Algorithm 9);
 *     kept here as the two separate counts pp and pc.
 *   - Morton keys: 21 bits per axis, bit interleave with x most significant (§4.4, Fig. `hot`).
 *   - Hashed-octree cell keys: root 1, child = parent << 3 | digit (§4.7).
 *   - Pre-order serialisation with an 8-bit child mask (§4.2).
 *   - Kick-drift-kick leapfrog, eqs. `leapkick1`, `leapdrift`, `leapkick2` (§2.4).
 *   - Energy, §2.3 (pair sum taken over i < j, softened like the force).
 *   - Quadrupole cell terms, eq. `truncmultipole` (§2.2), softened like the monopole.
 *   - Re-sort of last step's sorted order by insertion sort (§4.4, end: bodies move little in
 *     one step, so the list stays almost sorted).
 *   - Grouped acceptance test (Barnes 1990; not in the paper): one interaction list per group of
 *     bodies, cells tested against the group's bounding box.
 *
 * Readings where the paper is silent or garbled (all mirrored in the project's design notes):
 *   root box = tight FP64 min corner, side = largest extent (1 if all bodies coincide);
 *   quantisation q = clamp(floor((x - o) * s), 0, 2^21 - 1), s = 2^21 / L, subtract and multiply
 *   separately rounded; cell membership is decided on q (so tree and Morton order agree);
 *   bodies sharing one level-21 cell form a bucket leaf; the root is never MAC-tested; the MAC is
 *   the strict test l*l < theta*theta*d*d; cells use the same softened kernel as pairs;
 *   a pair at zero softened distance contributes nothing.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BITS 21
#define ORC_QMAX 2097151u           /* 2^21 - 1 */
#define ORC_CELLS 2097152.0         /* 2^21 */

static int g_threads = 1;

void orc_set_threads(int t) { g_threads = t < 1 ? 1 : t; }
int orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------ */
/* Root box and quantisation (§4.4: map the domain onto [0, 2^21)).     */
/* ------------------------------------------------------------------ */

/* box[0..2] = min corner o, box[3] = side L, box[4] = scale s = 2^21 / L. */
void orc_bbox(const double *pos, int64_t n, double *box)
{
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double *x = pos + (size_t)d * (size_t)n;
        double lo = 0.0, hi = 0.0;
        if (n > 0) { lo = x[0]; hi = x[0]; }
        for (int64_t i = 1; i < n; ++i) {
            if (x[i] < lo) lo = x[i];
            if (x[i] > hi) hi = x[i];
        }
        box[d] = lo;
        double e = hi - lo;
        if (e > ext) ext = e;
    }
    if (!(ext > 0.0)) ext = 1.0;
    box[3] = ext;
    box[4] = ORC_CELLS / ext;
}

static uint32_t quantise(double x, double o, double s)
{
    double t = (x - o) * s;
    if (!(t > 0.0)) return 0u;
    double f = floor(t);
    if (f >= (double)ORC_QMAX) return ORC_QMAX;
    return (uint32_t)f;
}

void orc_quantise(const double *pos, int64_t n, const double *box, uint32_t *q /* 3n */)
{
    for (int d = 0; d < 3; ++d)
        for (int64_t i = 0; i < n; ++i)
            q[(size_t)d * n + i] = quantise(pos[(size_t)d * n + i], box[d], box[4]);
}

/* Bit interleave of d coordinates of `bits` bits each, coordinate 0 most significant
 * within every group (the paper's x > y ordering, §4.4). */
uint64_t orc_interleave(const uint32_t *c, int d, int bits)
{
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int k = 0; k < d; ++k)
            key = (key << 1) | (uint64_t)((c[k] >> b) & 1u);
    return key;
}

void orc_keys(const double *pos, int64_t n, const double *box, uint64_t *keys)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t c[3];
        for (int d = 0; d < 3; ++d) c[d] = quantise(pos[(size_t)d * n + i], box[d], box[4]);
        keys[i] = orc_interleave(c, 3, ORC_BITS);
    }
}

/* ------------------------------------------------------------------ */
/* Sort of (key, id) pairs: ascending key, ties by ascending id.        */
/* ------------------------------------------------------------------ */

typedef struct { uint64_t key; int64_t id; } orc_pair;

static int pair_cmp(const void *a, const void *b)
{
    const orc_pair *x = (const orc_pair *)a, *y = (const orc_pair *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

void orc_sort_pairs(const uint64_t *keys, int64_t n, uint64_t *keys_out, int64_t *ids_out)
{
    orc_pair *p = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { p[i].key = keys[i]; p[i].id = i; }
    qsort(p, (size_t)n, sizeof(orc_pair), pair_cmp);
    for (int64_t i = 0; i < n; ++i) { keys_out[i] = p[i].key; ids_out[i] = p[i].id; }
    free(p);
}

/* ------------------------------------------------------------------ */
/* Re-sort from the previous order (§4.4, end: bodies move little in  */
/* one step, so last step's sorted list is almost sorted and an       */
/* insertion sort finishes it with few exchanges).                    */
/* ------------------------------------------------------------------ */

/* Insertion sort of the bodies taken in the order prev[0..n-1] (a permutation of 0..n-1, e.g. last
 * step's sorted ids) by (keys[id], id) ascending: each element sinks left past every element that
 * must follow it, one exchange of neighbours at a time.  Writes the sorted ids and keys; returns
 * the number of exchanges, which equals the number of inverted pairs of the starting order. */
int64_t orc_resort_insertion(const uint64_t *keys, const int64_t *prev, int64_t n,
                             uint64_t *keys_out, int64_t *ids_out)
{
    int64_t swaps = 0;
    for (int64_t i = 0; i < n; ++i) {
        ids_out[i] = prev[i];
        keys_out[i] = keys[prev[i]];
    }
    for (int64_t i = 1; i < n; ++i) {
        for (int64_t j = i; j > 0; --j) {
            const uint64_t ka = keys_out[j - 1], kb = keys_out[j];
            const int64_t ia = ids_out[j - 1], ib = ids_out[j];
            if (ka < kb || (ka == kb && ia < ib)) break;
            keys_out[j - 1] = kb;
            keys_out[j] = ka;
            ids_out[j - 1] = ib;
            ids_out[j] = ia;
            ++swaps;
        }
    }
    return swaps;
}

/* ------------------------------------------------------------------ */
/* Softened pair kernel (eq. `motion` + softening; eq. `approxforce`). */
/* ------------------------------------------------------------------ */

static inline void accumulate(double xp, double yp, double zp, double xj, double yj, double zj,
                              double mj, double G, double eps2, double *a)
{
    double dx = xj - xp;
    double dy = yj - yp;
    double dz = zj - zp;
    double r2 = dx * dx + dy * dy + dz * dz + eps2;
    if (r2 > 0.0) {
        double rinv = 1.0 / sqrt(r2);
        double rinv3 = rinv * rinv * rinv;
        double s = G * mj * rinv3;
        a[0] += s * dx;
        a[1] += s * dy;
        a[2] += s * dz;
    }
}

/* Algorithm 1: a_i = G sum_{j != i} m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^(3/2), j ascending.
 * targets == NULL means every body; acc is (3, nt) row-major. */
void orc_direct(const double *pos, const double *mass, int64_t n, const int64_t *targets,
                int64_t nt, double G, double eps, double *acc)
{
    const double eps2 = eps * eps;
    const double *X = pos, *Y = pos + n, *Z = pos + 2 * n;
    if (targets == NULL) nt = n;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double a[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j)
            if (j != i) accumulate(X[i], Y[i], Z[i], X[j], Y[j], Z[j], mass[j], G, eps2, a);
        acc[t] = a[0];
        acc[nt + t] = a[1];
        acc[2 * nt + t] = a[2];
    }
}

/* ------------------------------------------------------------------ */
/* Pointer octree by one-at-a-time insertion (Algorithm 2, "Build Tree"). */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t child[8];     /* -1: no child in that octant */
    int32_t level;        /* root 0; side = L / 2^level */
    uint32_t cell[3];     /* integer cell coordinates at this level */
    int32_t is_leaf;
    int32_t head;         /* leaf: first body of its list (-1 while the root is empty) */
    int32_t tail;
    int64_t nbody;        /* bodies in the subtree */
    double m, x, y, z;    /* total mass and centre of mass */
    double q[6];          /* quadrupole about the centre of mass: xx, yy, zz, xy, xz, yz */
} orc_node;

typedef struct {
    orc_node *nodes;
    int64_t n_nodes, cap;
    int has_quad;         /* quadrupoles computed (on first request) */
    int64_t n;
    int32_t *next;        /* body linked lists inside leaves (bucket members in id order) */
    uint32_t *q;          /* quantised coordinates, (3, n) */
    const double *pos;    /* borrowed, valid while the tree is used */
    const double *mass;
    double box[5];
} orc_tree;

static int32_t new_node(orc_tree *t, int32_t level, const uint32_t *qb)
{
    if (t->n_nodes == t->cap) {
        t->cap = t->cap ? t->cap * 2 : 1024;
        t->nodes = (orc_node *)realloc(t->nodes, sizeof(orc_node) * (size_t)t->cap);
    }
    orc_node *nd = &t->nodes[t->n_nodes];
    for (int c = 0; c < 8; ++c) nd->child[c] = -1;
    nd->level = level;
    for (int d = 0; d < 3; ++d) nd->cell[d] = level == 0 ? 0u : (qb[d] >> (ORC_BITS - level));
    nd->is_leaf = 1;
    nd->head = -1;
    nd->tail = -1;
    nd->nbody = 0;
    nd->m = nd->x = nd->y = nd->z = 0.0;
    return (int32_t)(t->n_nodes++);
}

/* Octant of body p inside a cell at `level` (its child at level+1): x > y > z (Fig. `hot`). */
static int octant(const orc_tree *t, int64_t p, int level)
{
    int b = ORC_BITS - 1 - level;
    uint32_t qx = t->q[p], qy = t->q[t->n + p], qz = t->q[2 * t->n + p];
    return (int)((((qx >> b) & 1u) << 2) | (((qy >> b) & 1u) << 1) | ((qz >> b) & 1u));
}

static void body_q(const orc_tree *t, int64_t p, uint32_t *qb)
{
    qb[0] = t->q[p];
    qb[1] = t->q[t->n + p];
    qb[2] = t->q[2 * t->n + p];
}

static void leaf_push(orc_tree *t, int32_t nd, int32_t p)
{
    orc_node *L = &t->nodes[nd];
    t->next[p] = -1;
    if (L->head < 0) L->head = p; else t->next[L->tail] = p;
    L->tail = p;
    L->nbody += 1;
}

static void insert(orc_tree *t, int32_t p)
{
    uint32_t qb[3];
    body_q(t, p, qb);
    int32_t nd = 0;
    for (;;) {
        orc_node *N = &t->nodes[nd];
        if (!N->is_leaf) {
            int c = octant(t, p, N->level);
            int32_t ch = N->child[c];
            if (ch < 0) {
                int32_t lv = N->level + 1;
                int32_t leaf = new_node(t, lv, qb);
                t->nodes[nd].child[c] = leaf;
                leaf_push(t, leaf, p);
                return;
            }
            nd = ch;
            continue;
        }
        if (N->nbody == 0) { leaf_push(t, nd, p); return; }          /* empty root */
        if (N->level == ORC_BITS) { leaf_push(t, nd, p); return; }   /* bucket */
        /* A leaf already holding one body: split it, push that body one level down, and go on
         * inserting p from this (now internal) node. */
        int32_t q = N->head;
        int lv = N->level;
        N->is_leaf = 0;
        N->head = N->tail = -1;
        N->nbody = 0;
        uint32_t qq[3];
        body_q(t, q, qq);
        int c = octant(t, q, lv);
        int32_t leaf = new_node(t, lv + 1, qq);
        t->nodes[nd].child[c] = leaf;
        leaf_push(t, leaf, q);
    }
}

/* Moments from the leaves to the root (Algorithm 2, "Compute mass distribution approximations"). */
static void moments(orc_tree *t, int32_t nd)
{
    orc_node *N = &t->nodes[nd];
    const double *X = t->pos, *Y = t->pos + t->n, *Z = t->pos + 2 * t->n;
    if (N->is_leaf) {
        if (N->nbody == 1) {
            int32_t p = N->head;
            N->m = t->mass[p]; N->x = X[p]; N->y = Y[p]; N->z = Z[p];
        } else if (N->nbody > 1) {
            double m = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
            for (int32_t p = N->head; p >= 0; p = t->next[p]) {
                m += t->mass[p];
                mx += t->mass[p] * X[p];
                my += t->mass[p] * Y[p];
                mz += t->mass[p] * Z[p];
            }
            N->m = m; N->x = mx / m; N->y = my / m; N->z = mz / m;
        }
        return;
    }
    double m = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    int64_t cnt = 0;
    for (int c = 0; c < 8; ++c) {
        int32_t ch = t->nodes[nd].child[c];
        if (ch < 0) continue;
        moments(t, ch);
        const orc_node *C = &t->nodes[ch];
        m += C->m;
        mx += C->m * C->x;
        my += C->m * C->y;
        mz += C->m * C->z;
        cnt += C->nbody;
    }
    N = &t->nodes[nd];
    N->m = m; N->x = mx / m; N->y = my / m; N->z = mz / m;
    N->nbody = cnt;
}

void *orc_tree_build(const double *pos, const double *mass, int64_t n)
{
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    t->n = n;
    t->pos = pos;
    t->mass = mass;
    orc_bbox(pos, n, t->box);
    t->q = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(3 * (n > 0 ? n : 1)));
    orc_quantise(pos, n, t->box, t->q);
    t->next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint32_t zero[3] = {0, 0, 0};
    new_node(t, 0, zero);
    for (int64_t p = 0; p < n; ++p) insert(t, (int32_t)p);
    if (n > 0) moments(t, 0);
    return t;
}

void orc_tree_free(void *h)
{
    orc_tree *t = (orc_tree *)h;
    if (!t) return;
    free(t->nodes);
    free(t->next);
    free(t->q);
    free(t);
}

/* stats[0] nodes, [1] max level, [2] buckets (leaves with > 1 body), [3] leaves */
void orc_tree_stats(void *h, int64_t *stats)
{
    orc_tree *t = (orc_tree *)h;
    int64_t depth = 0, buckets = 0, leaves = 0;
    for (int64_t i = 0; i < t->n_nodes; ++i) {
        const orc_node *N = &t->nodes[i];
        if (N->level > depth) depth = N->level;
        if (N->is_leaf) { leaves++; if (N->nbody > 1) buckets++; }
    }
    stats[0] = t->n > 0 ? t->n_nodes : 0;
    stats[1] = depth;
    stats[2] = buckets;
    stats[3] = t->n > 0 ? leaves : 0;
}

void orc_tree_box(void *h, double *box) { memcpy(box, ((orc_tree *)h)->box, 5 * sizeof(double)); }

void orc_tree_root(void *h, double *out)
{
    orc_tree *t = (orc_tree *)h;
    const orc_node *R = &t->nodes[0];
    out[0] = R->m; out[1] = R->x; out[2] = R->y; out[3] = R->z;
}

/* Pre-order serialisation (§4.2) with the hashed-octree key of each cell (§4.7).
 * Record r (5 int64): [key, level, child mask, first body rank, body count].
 * The body rank counts bodies in the order the traversal meets them in leaves. */
static void emit(const orc_tree *t, int32_t nd, int64_t *rec, int64_t *k, int64_t *rank,
                 int64_t *leaf_ids)
{
    const orc_node *N = &t->nodes[nd];
    int64_t *r = rec + 5 * (*k);
    (*k)++;
    uint64_t prefix = orc_interleave(N->cell, 3, N->level);
    uint64_t key = ((uint64_t)1 << (3 * N->level)) | prefix;
    int mask = 0;
    for (int c = 0; c < 8; ++c) if (N->child[c] >= 0) mask |= 1 << c;
    r[0] = (int64_t)key;
    r[1] = N->level;
    r[2] = mask;
    r[3] = *rank;
    r[4] = N->nbody;
    if (N->is_leaf) {
        for (int32_t p = N->head; p >= 0; p = t->next[p]) {
            if (leaf_ids) leaf_ids[*rank] = p;
            (*rank)++;
        }
        return;
    }
    for (int c = 0; c < 8; ++c)
        if (N->child[c] >= 0) emit(t, N->child[c], rec, k, rank, leaf_ids);
}

/* rec: 5 * n_nodes int64; leaf_ids: n int64 (may be NULL). Returns the record count. */
int64_t orc_tree_records(void *h, int64_t *rec, int64_t *leaf_ids)
{
    orc_tree *t = (orc_tree *)h;
    if (t->n == 0) return 0;
    int64_t k = 0, rank = 0;
    emit(t, 0, rec, &k, &rank, leaf_ids);
    return k;
}

/* Moments of every node in the pre-order of orc_tree_records: out[4k..4k+3] = (m, x, y, z). */
static void emit_moments(const orc_tree *t, int32_t nd, double *out, int64_t *k)
{
    const orc_node *N = &t->nodes[nd];
    double *r = out + 4 * (*k);
    (*k)++;
    r[0] = N->m; r[1] = N->x; r[2] = N->y; r[3] = N->z;
    if (N->is_leaf) return;
    for (int c = 0; c < 8; ++c)
        if (N->child[c] >= 0) emit_moments(t, N->child[c], out, k);
}

int64_t orc_tree_moments(void *h, double *out)
{
    orc_tree *t = (orc_tree *)h;
    if (t->n == 0) return 0;
    int64_t k = 0;
    emit_moments(t, 0, out, &k);
    return k;
}

/* ------------------------------------------------------------------ */
/* Quadrupole moments (§2.2, eq. `truncmultipole` and the coefficients below it): about the     */
/* cell's centre of mass, where the dipole vanishes,                                            */
/*   Q_aa = sum_j m_j (3 x_a,j^2 - r_j^2),   Q_ab = sum_j m_j 3 x_a,j x_b,j  (a != b),          */
/* x_j = r_j - r_J.  Computed here from that definition, body by body, for every cell.          */
/* ------------------------------------------------------------------ */

static void quad_add_bodies(const orc_tree *t, int32_t nd, const orc_node *J, double *q)
{
    const orc_node *N = &t->nodes[nd];
    const double *X = t->pos, *Y = t->pos + t->n, *Z = t->pos + 2 * t->n;
    if (N->is_leaf) {
        for (int32_t j = N->head; j >= 0; j = t->next[j]) {
            const double m = t->mass[j];
            const double x = X[j] - J->x, y = Y[j] - J->y, z = Z[j] - J->z;
            const double r2 = x * x + y * y + z * z;
            q[0] += m * (3.0 * x * x - r2);
            q[1] += m * (3.0 * y * y - r2);
            q[2] += m * (3.0 * z * z - r2);
            q[3] += m * (3.0 * x * y);
            q[4] += m * (3.0 * x * z);
            q[5] += m * (3.0 * y * z);
        }
        return;
    }
    for (int c = 0; c < 8; ++c)
        if (N->child[c] >= 0) quad_add_bodies(t, N->child[c], J, q);
}

static void quads(orc_tree *t)
{
    if (t->has_quad) return;
#pragma omp parallel for schedule(dynamic, 64) num_threads(g_threads)
    for (int64_t k = 0; k < t->n_nodes; ++k) {
        orc_node *J = &t->nodes[k];
        for (int a = 0; a < 6; ++a) J->q[a] = 0.0;
        quad_add_bodies(t, (int32_t)k, J, J->q);
    }
    t->has_quad = 1;
}

/* Cell term with the quadrupole: the acceleration -grad Phi of the softened truncated expansion
 * Phi = -G (M / r_s + (x.Q.x) / (2 r_s^5)), x = r_p - r_J, r_s^2 = |x|^2 + eps^2, i.e. with
 * d = r_J - r_p:  a += G (M d / r_s^3 - Q d / r_s^5 + 5/2 (d.Q.d) d / r_s^7). */
static inline void accumulate_quad(double xp, double yp, double zp, const orc_node *C, double G,
                                   double eps2, double *a)
{
    double dx = C->x - xp;
    double dy = C->y - yp;
    double dz = C->z - zp;
    double r2 = dx * dx + dy * dy + dz * dz + eps2;
    if (r2 > 0.0) {
        const double *q = C->q;
        double rinv = 1.0 / sqrt(r2);
        double rinv2 = rinv * rinv;
        double rinv3 = rinv * rinv2;
        double rinv5 = rinv3 * rinv2;
        double rinv7 = rinv5 * rinv2;
        double qx = q[0] * dx + q[3] * dy + q[4] * dz;
        double qy = q[3] * dx + q[1] * dy + q[5] * dz;
        double qz = q[4] * dx + q[5] * dy + q[2] * dz;
        double dqd = dx * qx + dy * qy + dz * qz;
        double s = G * (C->m * rinv3 + 2.5 * dqd * rinv7);
        double u = G * rinv5;
        a[0] += s * dx - u * qx;
        a[1] += s * dy - u * qy;
        a[2] += s * dz - u * qz;
    }
}

/* ------------------------------------------------------------------ */
/* Barnes-Hut walk (Algorithm 2, "Compute Cell Force"; counters of Algorithm 9). */
/* ------------------------------------------------------------------ */

typedef struct {
    double xp, yp, zp;
    int64_t p;
    double G, eps2, th2;
    double a[3];
    uint32_t pp, pc;
    int quad;             /* accepted cells add the quadrupole term */
} walk_state;

static void walk(const orc_tree *t, int32_t nd, walk_state *w)
{
    const double *X = t->pos, *Y = t->pos + t->n, *Z = t->pos + 2 * t->n;
    for (int c = 0; c < 8; ++c) {
        int32_t ch = t->nodes[nd].child[c];
        if (ch < 0) continue;
        const orc_node *C = &t->nodes[ch];
        if (C->is_leaf) {
            for (int32_t j = C->head; j >= 0; j = t->next[j]) {
                if (j == w->p) continue;
                accumulate(w->xp, w->yp, w->zp, X[j], Y[j], Z[j], t->mass[j], w->G, w->eps2, w->a);
                w->pp += 1;
            }
        } else {
            double l = ldexp(t->box[3], -C->level);
            double dx = C->x - w->xp;
            double dy = C->y - w->yp;
            double dz = C->z - w->zp;
            double d2 = dx * dx + dy * dy + dz * dz;
            if (l * l < w->th2 * d2) {
                if (w->quad)
                    accumulate_quad(w->xp, w->yp, w->zp, C, w->G, w->eps2, w->a);
                else
                    accumulate(w->xp, w->yp, w->zp, C->x, C->y, C->z, C->m, w->G, w->eps2, w->a);
                w->pc += 1;
            } else {
                walk(t, ch, w);
            }
        }
    }
}

/* Accelerations of the given targets (user ids; NULL = all bodies, nt ignored) on the tree.
 * acc is (3, nt) row-major; pp/pc (nt) may be NULL.  quad != 0: accepted cells add their
 * quadrupole term. */
void orc_tree_forces_q(void *h, const int64_t *targets, int64_t nt, double G, double eps,
                       double theta, int quad, double *acc, uint32_t *pp, uint32_t *pc)
{
    orc_tree *t = (orc_tree *)h;
    if (quad) quads(t);
    if (targets == NULL) nt = t->n;
    const double *X = t->pos, *Y = t->pos + t->n, *Z = t->pos + 2 * t->n;
    const double eps2 = eps * eps, th2 = theta * theta;
#pragma omp parallel for schedule(dynamic, 64) num_threads(g_threads)
    for (int64_t k = 0; k < nt; ++k) {
        int64_t p = targets ? targets[k] : k;
        walk_state w;
        w.xp = X[p]; w.yp = Y[p]; w.zp = Z[p];
        w.p = p;
        w.G = G; w.eps2 = eps2; w.th2 = th2;
        w.a[0] = w.a[1] = w.a[2] = 0.0;
        w.pp = w.pc = 0;
        w.quad = quad;
        if (!t->nodes[0].is_leaf) walk(t, 0, &w);
        acc[k] = w.a[0];
        acc[nt + k] = w.a[1];
        acc[2 * nt + k] = w.a[2];
        if (pp) pp[k] = w.pp;
        if (pc) pc[k] = w.pc;
    }
}

void orc_tree_forces(void *h, const int64_t *targets, int64_t nt, double G, double eps,
                     double theta, double *acc, uint32_t *pp, uint32_t *pc)
{
    orc_tree_forces_q(h, targets, nt, G, eps, theta, 0, acc, pp, pc);
}

/* Quadrupole moments of every node in the pre-order of orc_tree_records:
 * out[6k .. 6k+5] = (xx, yy, zz, xy, xz, yz). */
static void emit_quads(const orc_tree *t, int32_t nd, double *out, int64_t *k)
{
    memcpy(out + 6 * (*k), t->nodes[nd].q, 6 * sizeof(double));
    *k += 1;
    if (t->nodes[nd].is_leaf) return;
    for (int c = 0; c < 8; ++c)
        if (t->nodes[nd].child[c] >= 0) emit_quads(t, t->nodes[nd].child[c], out, k);
}

int64_t orc_tree_quads(void *h, double *out)
{
    orc_tree *t = (orc_tree *)h;
    quads(t);
    int64_t k = 0;
    if (t->n > 0) emit_quads(t, 0, out, &k);
    return k;
}

/* One-shot Barnes-Hut accelerations of all bodies (build + walk + free). */
void orc_bh(const double *pos, const double *mass, int64_t n, double G, double eps, double theta,
            double *acc, uint32_t *pp, uint32_t *pc)
{
    void *t = orc_tree_build(pos, mass, n);
    orc_tree_forces(t, NULL, n, G, eps, theta, acc, pp, pc);
    orc_tree_free(t);
}

/* ------------------------------------------------------------------ */
/* Group walk: NOT in the paper.  The grouped acceptance test of Barnes (1990): bodies close in  */
/* space form groups; a cell is accepted for the whole group when its side l                    */
/* and the distance d_min from its centre of mass to the group's bounding box satisfy           */
/* l*l < theta*theta*d_min*d_min, else it is opened; leaves interact with every member but the   */
/* body itself.  Every member then uses the group's interaction list.  With groups of one body   */
/* the box is a point, d_min is the per-body distance and this is the walk above, term for term. */
/* ------------------------------------------------------------------ */

typedef struct {
    const int64_t *ids;   /* members (user ids) */
    int64_t ng;
    double lo[3], hi[3];  /* bounding box of the members */
    double G, eps2, th2;
    double *acc;          /* (3, n) user order */
    int64_t n;
    uint32_t *pp, *pc;
} group_state;

static double axis_gap(double c, double lo, double hi)
{
    if (c < lo) return lo - c;
    if (c > hi) return c - hi;
    return 0.0;
}

static void group_walk(const orc_tree *t, int32_t nd, group_state *g)
{
    const double *X = t->pos, *Y = t->pos + t->n, *Z = t->pos + 2 * t->n;
    for (int c = 0; c < 8; ++c) {
        int32_t ch = t->nodes[nd].child[c];
        if (ch < 0) continue;
        const orc_node *C = &t->nodes[ch];
        if (C->is_leaf) {
            for (int32_t j = C->head; j >= 0; j = t->next[j]) {
                for (int64_t k = 0; k < g->ng; ++k) {
                    const int64_t p = g->ids[k];
                    if (j == p) continue;
                    double a[3] = {g->acc[p], g->acc[g->n + p], g->acc[2 * g->n + p]};
                    accumulate(X[p], Y[p], Z[p], X[j], Y[j], Z[j], t->mass[j], g->G, g->eps2, a);
                    g->acc[p] = a[0];
                    g->acc[g->n + p] = a[1];
                    g->acc[2 * g->n + p] = a[2];
                    if (g->pp) g->pp[p] += 1;
                }
            }
        } else {
            double l = ldexp(t->box[3], -C->level);
            double dx = axis_gap(C->x, g->lo[0], g->hi[0]);
            double dy = axis_gap(C->y, g->lo[1], g->hi[1]);
            double dz = axis_gap(C->z, g->lo[2], g->hi[2]);
            double d2 = dx * dx + dy * dy + dz * dz;
            if (l * l < g->th2 * d2) {
                for (int64_t k = 0; k < g->ng; ++k) {
                    const int64_t p = g->ids[k];
                    double a[3] = {g->acc[p], g->acc[g->n + p], g->acc[2 * g->n + p]};
                    accumulate(X[p], Y[p], Z[p], C->x, C->y, C->z, C->m, g->G, g->eps2, a);
                    g->acc[p] = a[0];
                    g->acc[g->n + p] = a[1];
                    g->acc[2 * g->n + p] = a[2];
                    if (g->pc) g->pc[p] += 1;
                }
            } else {
                group_walk(t, ch, g);
            }
        }
    }
}

/* Groups that follow the tree's cells: a cell of more than gmax bodies hands out its children
 * in octant order, consecutive children of at most gmax bodies merged while the group stays
 * within gmax, larger children handled the same way in turn (buckets of more than gmax bodies cut
 * into chunks of gmax in their list order); a root of at most gmax bodies is one group.
 * members receives the user ids group after group (each in Morton order), offsets the group
 * starts (n_groups + 1 entries).  Returns the number of groups. */
typedef struct {
    int64_t *members, *offsets;
    int64_t nm, ng, cur;     /* members written, groups closed, members in the open group */
    int64_t gmax;
} cell_groups_state;

static void cg_flush(cell_groups_state *s)
{
    if (s->cur == 0) return;
    s->ng += 1;
    s->offsets[s->ng] = s->nm;
    s->cur = 0;
}

static void cg_add_subtree(const orc_tree *t, int32_t nd, cell_groups_state *s)
{
    const orc_node *N = &t->nodes[nd];
    if (N->is_leaf) {
        for (int32_t j = N->head; j >= 0; j = t->next[j]) {
            s->members[s->nm++] = j;
            s->cur += 1;
        }
        return;
    }
    for (int c = 0; c < 8; ++c)
        if (N->child[c] >= 0) cg_add_subtree(t, N->child[c], s);
}

static void cg_visit(const orc_tree *t, int32_t nd, cell_groups_state *s)
{
    for (int c = 0; c < 8; ++c) {
        const int32_t ch = t->nodes[nd].child[c];
        if (ch < 0) continue;
        const orc_node *C = &t->nodes[ch];
        if (C->nbody > s->gmax) {
            cg_flush(s);
            if (C->is_leaf) {
                for (int32_t j = C->head; j >= 0; j = t->next[j]) {
                    s->members[s->nm++] = j;
                    if (++s->cur == s->gmax) cg_flush(s);
                }
                cg_flush(s);
            } else {
                cg_visit(t, ch, s);
            }
            continue;
        }
        if (s->cur > 0 && s->cur + C->nbody > s->gmax) cg_flush(s);
        cg_add_subtree(t, ch, s);
    }
    cg_flush(s);
}

int64_t orc_tree_cell_groups(void *h, int64_t gmax, int64_t *members, int64_t *offsets)
{
    orc_tree *t = (orc_tree *)h;
    cell_groups_state s = {members, offsets, 0, 0, 0, gmax};
    offsets[0] = 0;
    if (t->n == 0) return 0;
    if (t->nodes[0].nbody <= gmax) {
        cg_add_subtree(t, 0, &s);
        cg_flush(&s);
    } else {
        cg_visit(t, 0, &s);
    }
    return s.ng;
}

/* Group-walk accelerations of all bodies.  Group k is members[offsets[k] .. offsets[k+1] - 1]
 * (user ids).  acc (3, n) user order; pp, pc (n) may be NULL. */
void orc_tree_forces_group(void *h, const int64_t *members, const int64_t *offsets,
                           int64_t ngroups, double G, double eps, double theta, double *acc,
                           uint32_t *pp, uint32_t *pc)
{
    orc_tree *t = (orc_tree *)h;
    const int64_t n = t->n;
    const double *X = t->pos, *Y = t->pos + n, *Z = t->pos + 2 * n;
    memset(acc, 0, sizeof(double) * 3 * n);
    if (pp) memset(pp, 0, sizeof(uint32_t) * n);
    if (pc) memset(pc, 0, sizeof(uint32_t) * n);
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int64_t k = 0; k < ngroups; ++k) {
        group_state g;
        g.ids = members + offsets[k];
        g.ng = offsets[k + 1] - offsets[k];
        for (int d = 0; d < 3; ++d) {
            g.lo[d] = INFINITY;
            g.hi[d] = -INFINITY;
        }
        for (int64_t m = 0; m < g.ng; ++m) {
            const int64_t p = g.ids[m];
            const double v[3] = {X[p], Y[p], Z[p]};
            for (int d = 0; d < 3; ++d) {
                if (v[d] < g.lo[d]) g.lo[d] = v[d];
                if (v[d] > g.hi[d]) g.hi[d] = v[d];
            }
        }
        g.G = G;
        g.eps2 = eps * eps;
        g.th2 = theta * theta;
        g.acc = acc;
        g.n = n;
        g.pp = pp;
        g.pc = pc;
        if (!t->nodes[0].is_leaf) group_walk(t, 0, &g);
    }
}

/* ------------------------------------------------------------------ */
/* Kick-drift-kick leapfrog (§2.4, eqs. leapkick1, leapdrift, leapkick2). */
/* ------------------------------------------------------------------ */

/* Advances nsteps steps.  On entry acc holds a^(k) at the entry positions; on exit it holds the
 * acceleration at the final positions.  method 0 = direct sum, 1 = Barnes-Hut. */
void orc_kdk(double *pos, double *vel, const double *mass, int64_t n, double *acc, double G,
             double eps, double theta, double dt, int32_t nsteps, int32_t method)
{
    const double h = 0.5 * dt;
    const int64_t m3 = 3 * n;
    for (int32_t s = 0; s < nsteps; ++s) {
        for (int64_t i = 0; i < m3; ++i) vel[i] = vel[i] + acc[i] * h;
        for (int64_t i = 0; i < m3; ++i) pos[i] = pos[i] + vel[i] * dt;
        if (method == 0) orc_direct(pos, mass, n, NULL, n, G, eps, acc);
        else orc_bh(pos, mass, n, G, eps, theta, acc, NULL, NULL);
        for (int64_t i = 0; i < m3; ++i) vel[i] = vel[i] + acc[i] * h;
    }
}

/* ------------------------------------------------------------------ */
/* Energy (§2.3): E_kin = sum m v^2 / 2, E_pot = -sum_{i<j} G m_i m_j / sqrt(r_ij^2 + eps^2). */
/* ------------------------------------------------------------------ */

void orc_energy(const double *pos, const double *vel, const double *mass, int64_t n, double G,
                double eps, double *out)
{
    const double eps2 = eps * eps;
    const double *X = pos, *Y = pos + n, *Z = pos + 2 * n;
    double ekin = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double v2 = vel[i] * vel[i] + vel[n + i] * vel[n + i] + vel[2 * n + i] * vel[2 * n + i];
        ekin += 0.5 * mass[i] * v2;
    }
    double *row = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = X[j] - X[i], dy = Y[j] - Y[i], dz = Z[j] - Z[i];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 > 0.0) s += G * mass[i] * mass[j] / sqrt(r2);
        }
        row[i] = s;
    }
    double epot = 0.0;
    for (int64_t i = 0; i < n; ++i) epot -= row[i];
    free(row);
    out[0] = ekin;
    out[1] = epot;
    out[2] = ekin + epot;
}

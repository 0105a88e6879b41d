// Force kernels: the Barnes-Hut walk (Algorithm 2, "Compute Cell Force") and the direct sum
// (Algorithm 1), both with the softened pair kernel of eq. `motion` (§2.1).
//
// FP64 walk.  The nodes are stored in pre-order, each with `skip` = the index of the first node
// after its subtree.  A body's recursive walk over the children of every opened cell then
// becomes a monotone scan over node indices: at node j the body either opens j (next node j + 1,
// its first child) or is done with j's subtree (next node skip[j]: a leaf, or a cell accepted by
// l/d < theta).  One warp owns 32 Morton-consecutive bodies; every lane keeps its own `next`, and
// the warp visits the minimum `next` over its lanes, so each lane sees exactly its own sequence
// of nodes in its own order: interaction list and summation order are those of the per-particle
// recursive walk.
//
// FP32 walk: the group walk below (same interaction lists, terms summed in another order).
#include <math.h>

#include <algorithm>

#include "nbody_internal.cuh"

namespace nb {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 ldg4(const float4 *p) { return __ldg(p); }

// 1/sqrt(x) from the hardware approximation (the one rsqrtf uses) with subnormal inputs taken as
// zero: skips the rescaling of subnormal arguments, which never occur here (x >= eps^2 > 0, or
// x == 0 under kGuard).
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// FP64 pair term with every operation separately rounded in the order of the plain definition:
// dx = xj - xi, r2 = ((dx dx + dy dy) + dz dz) + eps^2, 1 / sqrt(r2), (G m) (1/r)^3.
__device__ __forceinline__ void pair64(double xj, double yj, double zj, double mj, double xi,
                                       double yi, double zi, double G, double eps2, double &ax,
                                       double &ay, double &az)
{
    const double dx = __dsub_rn(xj, xi), dy = __dsub_rn(yj, yi), dz = __dsub_rn(zj, zi);
    const double r2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                          __dmul_rn(dz, dz)), eps2);
    if (r2 > 0.0) {
        const double rinv = __ddiv_rn(1.0, __dsqrt_rn(r2));
        const double rinv3 = __dmul_rn(__dmul_rn(rinv, rinv), rinv);
        const double f = __dmul_rn(__dmul_rn(G, mj), rinv3);
        ax = __dadd_rn(ax, __dmul_rn(f, dx));
        ay = __dadd_rn(ay, __dmul_rn(f, dy));
        az = __dadd_rn(az, __dmul_rn(f, dz));
    }
}

// The same pair term, fast form (NBODY_FP64_FAST): fused multiply-adds and one reciprocal
// square root; the result differs from pair64 by rounding only.
__device__ __forceinline__ void pair64_fast(double xj, double yj, double zj, double mj, double xi,
                                            double yi, double zi, double G, double eps2,
                                            double &ax, double &ay, double &az)
{
    const double dx = xj - xi, dy = yj - yi, dz = zj - zi;
    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    if (r2 > 0.0) {
        const double ri = rsqrt(r2);
        const double f = (G * mj) * (ri * ri * ri);
        ax = fma(f, dx, ax);
        ay = fma(f, dy, ay);
        az = fma(f, dz, az);
    }
}

template <bool kFast>
__device__ __forceinline__ void pair64_any(double xj, double yj, double zj, double mj, double xi,
                                           double yi, double zi, double G, double eps2,
                                           double &ax, double &ay, double &az)
{
    if (kFast) pair64_fast(xj, yj, zj, mj, xi, yi, zi, G, eps2, ax, ay, az);
    else pair64(xj, yj, zj, mj, xi, yi, zi, G, eps2, ax, ay, az);
}

// FP64 cell term with the quadrupole (§2.2, eq. `truncmultipole`): the acceleration of the
// softened expansion Phi = -G (M / r_s + (x.Q.x) / (2 r_s^5)), x = r_i - r_J,
// r_s^2 = |x|^2 + eps^2; with d = r_J - r_i:
//   a += G (M d / r_s^3 - Q d / r_s^5 + 5/2 (d.Q.d) d / r_s^7),
// q = (xx, yy, zz, xy, xz, yz); every operation separately rounded.
__device__ __forceinline__ void cell64q(double xj, double yj, double zj, double mj,
                                        const double *__restrict__ q, double xi, double yi,
                                        double zi, double G, double eps2, double &ax, double &ay,
                                        double &az)
{
    const double dx = __dsub_rn(xj, xi), dy = __dsub_rn(yj, yi), dz = __dsub_rn(zj, zi);
    const double r2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                          __dmul_rn(dz, dz)), eps2);
    if (!(r2 > 0.0)) return;
    const double rinv = __ddiv_rn(1.0, __dsqrt_rn(r2));
    const double rinv2 = __dmul_rn(rinv, rinv);
    const double rinv3 = __dmul_rn(rinv, rinv2);
    const double rinv5 = __dmul_rn(rinv3, rinv2);
    const double rinv7 = __dmul_rn(rinv5, rinv2);
    const double qx = __dadd_rn(__dadd_rn(__dmul_rn(q[0], dx), __dmul_rn(q[3], dy)), __dmul_rn(q[4], dz));
    const double qy = __dadd_rn(__dadd_rn(__dmul_rn(q[3], dx), __dmul_rn(q[1], dy)), __dmul_rn(q[5], dz));
    const double qz = __dadd_rn(__dadd_rn(__dmul_rn(q[4], dx), __dmul_rn(q[5], dy)), __dmul_rn(q[2], dz));
    const double dqd = __dadd_rn(__dadd_rn(__dmul_rn(dx, qx), __dmul_rn(dy, qy)), __dmul_rn(dz, qz));
    const double s = __dmul_rn(G, __dadd_rn(__dmul_rn(mj, rinv3), __dmul_rn(__dmul_rn(2.5, dqd), rinv7)));
    const double u = __dmul_rn(G, rinv5);
    ax = __dadd_rn(ax, __dsub_rn(__dmul_rn(s, dx), __dmul_rn(u, qx)));
    ay = __dadd_rn(ay, __dsub_rn(__dmul_rn(s, dy), __dmul_rn(u, qy)));
    az = __dadd_rn(az, __dsub_rn(__dmul_rn(s, dz), __dmul_rn(u, qz)));
}

// One step of Kahan's compensated summation (Kahan 1965): s + c tracks the exact running sum.
__device__ __forceinline__ void kahan_add(float &s, float &c, float t)
{
    const float yv = t - c;
    const float u = s + yv;
    c = (u - s) - yv;
    s = u;
}

__device__ __forceinline__ void write_out(const WalkArgs &a, int i, double ax, double ay, double az,
                                          uint32_t pp, uint32_t pc)
{
    const uint32_t id = a.ids[i];
    const size_t n = (size_t)a.n;
    a.acc[id] = ax;
    a.acc[n + id] = ay;
    a.acc[2 * n + id] = az;
    if (a.vel) {
        // second kick of the leapfrog (eq. leapkick2): v += a dt/2, separately rounded
        a.vel[id] = __dadd_rn(a.vel[id], __dmul_rn(ax, a.h));
        a.vel[n + id] = __dadd_rn(a.vel[n + id], __dmul_rn(ay, a.h));
        a.vel[2 * n + id] = __dadd_rn(a.vel[2 * n + id], __dmul_rn(az, a.h));
    }
    if (a.pp) {
        a.pp[i] = pp;
        a.pc[i] = pc;
    }
}

// ------------------------------------------------------------------------------------------
// FP32 group walk with the grouped acceptance test or quadrupole cells (the per-body test with
// monopole cells, the default, runs the span-shared form further down, pb_walk32_kernel, built on
// the same classification).  One warp owns a group of 32 Morton-consecutive bodies and walks the
// level-order tree for all of them at once, 32 nodes per step (one node per lane).  Each node is
// tested against the group's bounding box first.  Per body the acceptance test is
// d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > crit with dx = c.x - x in FP32 (MAC l/d < theta of
// §3, crit = l^2 / theta^2); every step of that expression is monotone in |dx|, |dy|, |dz|, so
// the same expression over the per-axis distances from c to the box gives a lower bound of every
// body's d2, and over the farthest box corner an upper bound.  Hence:
//   lower bound > crit  -> every body of the group accepts the cell,
//   upper bound <= crit -> every body opens it,
// both exactly as the per-body test decides; only the cells in between ("mixed") are tested body
// by body (one lane per body).  A node on the stack carries the mask of the bodies that opened
// all its ancestors, so each body ends up with exactly the interaction list of its own walk
// (Algorithm 2, "Compute Cell Force"): the same cells accepted, the same leaves, itself left
// out.  Only the order of the terms differs.
//
// Interactions are collected per warp in shared memory, full-group ones (every live body of
// the group) and partial ones (with a body mask), and evaluated in a dense loop with one lane per
// body reading each source by broadcast.
// ------------------------------------------------------------------------------------------

// Stack of child ranges.  Every step pops <= 32 nodes and pushes <= 1 range per popped node, all
// one level deeper than the shallowest popped node; so the ranges pushed by one step lie
// strictly deeper than everything left below them, and at most 21 such groups (levels 1..21) of
// <= 32 ranges are ever on the stack.
constexpr int kStackCap = 22 * 32;
constexpr int kFCap = 64;    // full-group interaction buffer
constexpr int kPCap = 64;    // partial interaction buffer
constexpr uint32_t kIdxMask = 0x0fffffffu;  // node index bits of a stack entry; 3 bits count - 1

// Interaction buffers hold sources in pairs for the packed (2 x FP32) pair kernel: entries
// 2k and 2k+1 are f[2k] = (x0, x1, y0, y1) and f[2k+1] = (z0, z1, w0, w1).
struct GroupSmem {
    uint32_t st_node[kStackCap];  // first node | (count - 1) << 28
    uint32_t st_mask[kStackCap];  // bodies of the group that still need these nodes
    float4 f[kFCap];              // full-group sources, paired
    float4 p[kPCap];              // partial sources, paired
    uint2 pm[kPCap];              // (body mask, 1 for a leaf body / 0 for a cell) per entry
};

// With quadrupoles, accepted cells go to their own buffers (their term needs G Q), in pairs for
// the packed kernel: cells 2k and 2k+1 occupy five float4, (x0, x1, y0, y1), (z0, z1, w0, w1),
// (xx0, xx1, yy0, yy1), (zz0, zz1, xy0, xy1), (xz0, xz1, yz0, yz1) with w = G M and the
// quadrupole components times G; the partial ones with a body mask each.
constexpr int kQCap = 32;
struct QuadSmem {
    float4 f[5 * kQCap / 2];
    float4 p[5 * kQCap / 2];
    uint32_t pm[kQCap];
};

__device__ __forceinline__ void put_quad_entry(float4 *buf, int e, const float4 &c,
                                               const float4 &q0, const float4 &q1)
{
    float *q = reinterpret_cast<float *>(buf + 5 * (e >> 1)) + (e & 1);
    q[0] = c.x;
    q[2] = c.y;
    q[4] = c.z;
    q[6] = c.w;
    q[8] = q0.x;    // xx
    q[10] = q0.y;   // yy
    q[12] = q0.z;   // zz
    q[14] = q0.w;   // xy
    q[16] = q1.x;   // xz
    q[18] = q1.y;   // yz
}

// Two quadrupole cell terms at once with packed FP32 arithmetic (the expansion of cell32q);
// on = (on0, on1) drops a term with 0.
template <bool kGuard>
__device__ __forceinline__ void cell32q_x2(const float4 *e, float2 nx, float2 ny, float2 nz,
                                           float2 eps2, float2 on, float2 &ax, float2 &ay,
                                           float2 &az)
{
    const float4 a = e[0], b = e[1], q0 = e[2], q1 = e[3], q2 = e[4];
    const float2 dx = __fadd2_rn(make_float2(a.x, a.y), nx);
    const float2 dy = __fadd2_rn(make_float2(a.z, a.w), ny);
    const float2 dz = __fadd2_rn(make_float2(b.x, b.y), nz);
    float2 r2 = __ffma2_rn(dz, dz, eps2);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dx, dx, r2);
    float2 ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
    if (kGuard) {
        ri.x = r2.x > 0.f ? ri.x : 0.f;
        ri.y = r2.y > 0.f ? ri.y : 0.f;
    }
    ri = __fmul2_rn(ri, on);
    const float2 ri2 = __fmul2_rn(ri, ri);
    const float2 ri3 = __fmul2_rn(ri, ri2);
    const float2 ri5 = __fmul2_rn(ri3, ri2);
    const float2 ri7 = __fmul2_rn(ri5, ri2);
    const float2 qxx = make_float2(q0.x, q0.y), qyy = make_float2(q0.z, q0.w);
    const float2 qzz = make_float2(q1.x, q1.y), qxy = make_float2(q1.z, q1.w);
    const float2 qxz = make_float2(q2.x, q2.y), qyz = make_float2(q2.z, q2.w);
    const float2 qx = __ffma2_rn(qxx, dx, __ffma2_rn(qxy, dy, __fmul2_rn(qxz, dz)));
    const float2 qy = __ffma2_rn(qxy, dx, __ffma2_rn(qyy, dy, __fmul2_rn(qyz, dz)));
    const float2 qz = __ffma2_rn(qxz, dx, __ffma2_rn(qyz, dy, __fmul2_rn(qzz, dz)));
    const float2 dqd = __ffma2_rn(dx, qx, __ffma2_rn(dy, qy, __fmul2_rn(dz, qz)));
    const float2 s = __ffma2_rn(make_float2(b.z, b.w), ri3,
                                __fmul2_rn(__fmul2_rn(make_float2(2.5f, 2.5f), dqd), ri7));
    const float2 nri5 = __fmul2_rn(make_float2(-1.f, -1.f), ri5);
    ax = __ffma2_rn(s, dx, __ffma2_rn(nri5, qx, ax));
    ay = __ffma2_rn(s, dy, __ffma2_rn(nri5, qy, ay));
    az = __ffma2_rn(s, dz, __ffma2_rn(nri5, qz, az));
}
template <bool kQuad>
__host__ __device__ constexpr size_t group_smem_bytes()
{
    return kQuad ? sizeof(GroupSmem) + sizeof(QuadSmem) : sizeof(GroupSmem);
}

__device__ __forceinline__ void put_entry(float4 *buf, int e, const float4 &c)
{
    float *q = reinterpret_cast<float *>(buf + 2 * (e >> 1)) + (e & 1);
    q[0] = c.x;
    q[2] = c.y;
    q[4] = c.z;
    q[6] = c.w;
}

// Two softened pair terms at once with packed FP32 arithmetic (each component rounded exactly
// as the scalar fmaf / add / mul): sources a = (x0, x1, y0, y1), b = (z0, z1, w0, w1); the
// target's coordinates come negated.  The terms are added to two interleaved partial sums.
template <bool kGuard>
__device__ __forceinline__ void pair32x2(const float4 &a, const float4 &b, float2 nx, float2 ny,
                                         float2 nz, float2 eps2, float2 &ax, float2 &ay,
                                         float2 &az)
{
    const float2 dx = __fadd2_rn(make_float2(a.x, a.y), nx);
    const float2 dy = __fadd2_rn(make_float2(a.z, a.w), ny);
    const float2 dz = __fadd2_rn(make_float2(b.x, b.y), nz);
    float2 r2 = __ffma2_rn(dz, dz, eps2);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dx, dx, r2);
    float2 ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
    if (kGuard) {
        ri.x = r2.x > 0.f ? ri.x : 0.f;
        ri.y = r2.y > 0.f ? ri.y : 0.f;
    }
    const float2 f = __fmul2_rn(__fmul2_rn(make_float2(b.z, b.w), __fmul2_rn(ri, ri)), ri);
    ax = __ffma2_rn(f, dx, ax);
    ay = __ffma2_rn(f, dy, ay);
    az = __ffma2_rn(f, dz, az);
}

// Packed accumulator: two interleaved FP32 partial sums per component.  Compensated form: the
// partials are folded into a Kahan sum every kFold terms and at the end.
template <bool kKahan>
struct Acc3x2 {
    static constexpr int kFold = 64;
    float2 x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f), z = make_float2(0.f, 0.f);
    float sx = 0.f, sy = 0.f, sz = 0.f;  // compensated total
    float cx = 0.f, cy = 0.f, cz = 0.f;  // its compensation
    __device__ __forceinline__ void fold()
    {
        if (kKahan) {
            kahan_add(sx, cx, x.x + x.y);
            kahan_add(sy, cy, y.x + y.y);
            kahan_add(sz, cz, z.x + z.y);
            x = y = z = make_float2(0.f, 0.f);
        }
    }
    __device__ __forceinline__ float3 result()
    {
        if (kKahan) {
            fold();
            return make_float3(sx, sy, sz);
        }
        return make_float3(x.x + x.y, y.x + y.y, z.x + z.y);
    }
};

enum : int { kNone = 0, kFullLeaf, kFullCell, kPartLeaf, kPartCell, kOpen, kMixed, kBucket };

__device__ __forceinline__ unsigned lanemask_lt_w()
{
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

__device__ __forceinline__ float warp_fmin(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ float warp_fmax(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Distance along one axis from c to [lo, hi], as the per-body expression rounds it: the smallest
// |c - x| (0 inside) and the largest.
__device__ __forceinline__ void axis_bounds(float c, float lo, float hi, float &dmin, float &dmax)
{
    const float a = c - lo, b = c - hi;   // a >= b
    dmin = b > 0.f ? b : (a < 0.f ? a : 0.f);
    dmax = fmaxf(fabsf(a), fabsf(b));
}

// Group gi: its first sorted body, its size (1..32) and the level-order index of its system's
// root.  Without a table a single system is cut into groups of 32 from body 0; a table lists
// the groups (none crosses a system boundary): a forest's fixed chunks, or groups that follow
// the tree's cells, built on the device (count in *d_ngroups).
__device__ __forceinline__ bool group_of(const WalkArgs &a, int gi, int &g0, int &count,
                                         int &root)
{
    if (a.groups) {
        const int ng = a.d_ngroups ? (int)min(*a.d_ngroups, (unsigned)a.n_groups) : a.n_groups;
        if (gi >= ng) return false;
        const int4 g = a.groups[gi];
        g0 = g.x;
        count = g.y;
        root = a.roots ? a.roots[g.z] : 0;
        return true;
    }
    g0 = gi * 32;
    if (g0 >= a.n) return false;
    count = min(32, a.n - g0);
    root = 0;
    return true;
}

template <bool kKahan, bool kGuard>
struct GroupEval {
    Acc3x2<kKahan> acc;
    uint32_t pp = 0, pc = 0;      // partial entries of this lane's body: leaves, all
    int terms = 0;                // terms in the current partial (warp-uniform)
    __device__ __forceinline__ void settle(int cnt)
    {
        terms += cnt;
        if (terms >= Acc3x2<kKahan>::kFold) {
            acc.fold();
            terms = 0;
        }
    }
    // quadrupole cells, two at a time (counts padded to even by the caller): every live body of
    // the group (full) or the masked ones (part)
    __device__ __forceinline__ void full_quad(const QuadSmem &Q, int cnt, const float2 *nme,
                                              float2 eps2)
    {
        const int np = (cnt + 1) >> 1;
#pragma unroll 2
        for (int k = 0; k < np; ++k)
            cell32q_x2<kGuard>(Q.f + 5 * k, nme[0], nme[1], nme[2], eps2, make_float2(1.f, 1.f),
                               acc.x, acc.y, acc.z);
        settle(cnt);
    }
    __device__ __forceinline__ void part_quad(const QuadSmem &Q, int cnt, const float2 *nme,
                                              float2 eps2, int lane)
    {
        const int np = (cnt + 1) >> 1;
        const uint2 *pm2 = reinterpret_cast<const uint2 *>(Q.pm);
        for (int k = 0; k < np; ++k) {
            const uint2 m = pm2[k];
            const uint32_t on0 = (m.x >> lane) & 1u, on1 = (m.y >> lane) & 1u;
            cell32q_x2<kGuard>(Q.p + 5 * k, nme[0], nme[1], nme[2], eps2,
                               make_float2((float)on0, (float)on1), acc.x, acc.y, acc.z);
            pc += on0 + on1;
        }
        settle(cnt);
    }
    // cnt entries, padded to an even count by the caller (a zero-weight entry)
    __device__ __forceinline__ void full(const GroupSmem &S, int cnt, const float2 *nme,
                                         float2 eps2)
    {
        const int np = (cnt + 1) >> 1;
#pragma unroll 2
        for (int k = 0; k < np; ++k)
            pair32x2<kGuard>(S.f[2 * k], S.f[2 * k + 1], nme[0], nme[1], nme[2], eps2, acc.x,
                             acc.y, acc.z);
        settle(cnt);
    }
    __device__ __forceinline__ void part(const GroupSmem &S, int cnt, const float2 *nme,
                                         float2 eps2, int lane)
    {
        const int np = (cnt + 1) >> 1;
        const uint4 *pm2 = reinterpret_cast<const uint4 *>(S.pm);
#pragma unroll 2
        for (int k = 0; k < np; ++k) {
            const float4 a = S.p[2 * k];
            float4 b = S.p[2 * k + 1];
            const uint4 q = pm2[k];   // (mask0, leaf0, mask1, leaf1)
            const uint32_t on0 = (q.x >> lane) & 1u, on1 = (q.z >> lane) & 1u;
            b.z = on0 ? b.z : 0.f;
            b.w = on1 ? b.w : 0.f;
            pair32x2<kGuard>(a, b, nme[0], nme[1], nme[2], eps2, acc.x, acc.y, acc.z);
            pp += (on0 & q.y) + (on1 & q.w);  // leaf bodies
            pc += on0 + on1;                  // all partial entries; the cells are pc - pp
        }
        settle(cnt);
    }
};

// kWarps warps per block (a launch shape the autotuner chooses; results do not depend on it).
// kQuad: accepted cells add their quadrupole term (§2.2).
// kGroup: the grouped acceptance test (Barnes 1990; not in the paper): a cell is accepted for
// the whole group when the lower bound of the group's distances passes the test, else it is
// opened for the whole group; no body masks, no per-body tests.  A body meets its own leaf and
// interacts with itself there, which adds exactly zero (zero separation), and is not counted.
// The walk of one group (bodies g0 .. g0 + gcount - 1, its system's root at level-order index
// root) by one warp with its shared-memory slice S.
template <bool kKahan, bool kGuard, bool kGroup, bool kQuad>
__device__ __forceinline__ void walk_group(const WalkArgs &a, GroupSmem &S, QuadSmem &Q, int lane,
                                           int g0, int gcount, int root)
{
    const int i = g0 + lane;
    const bool live = lane < gcount;
    const int n_nodes = (int)*a.d_nn;
    const unsigned lt = lanemask_lt_w();
    const unsigned live_mask = __ballot_sync(kFull, live);
    // lanes past the group's end stand on its last body so that they do not widen its box
    const float4 me = ldg4(a.sbody32 + g0 + min(lane, gcount - 1));
    const float lox = warp_fmin(me.x), loy = warp_fmin(me.y), loz = warp_fmin(me.z);
    const float hix = warp_fmax(me.x), hiy = warp_fmax(me.y), hiz = warp_fmax(me.z);
    const float eps2s = (float)(a.eps * a.eps);
    const float2 eps2 = make_float2(eps2s, eps2s);
    const float2 nme[3] = {make_float2(-me.x, -me.x), make_float2(-me.y, -me.y),
                           make_float2(-me.z, -me.z)};

    GroupEval<kKahan, kGuard> ev;
    uint32_t upp = 0, upc = 0;    // full-entry counts (the same for every live body)
    unsigned self_seen = 0u;      // group walk: bodies whose own leaf entered the list
    int sp = 0, fn = 0, pn = 0;   // stack depth and buffer fills (warp-uniform)
    int qfn = 0, qpn = 0;         // quadrupole-cell buffer fills (warp-uniform)

    // the root is never tested: the walk starts with the root's children (none when the root
    // is a leaf, i.e. a single body)
    if (root >= 0 && root < n_nodes) {
        const int4 r = __ldg(reinterpret_cast<const int4 *>(&a.gn[root].child));
        if (r.y > 0) {
            if (lane == 0) {
                S.st_node[0] = (uint32_t)r.x | ((uint32_t)(r.y - 1) << 28);
                S.st_mask[0] = live_mask;
            }
            sp = 1;
        }
    }

    // appends one entry per lane whose kind says so: full-group entries to f, others to p;
    // with quadrupoles accepted cells go to their own buffers, with their G Q (node: level-order
    // index of the cell)
    auto emit = [&](int kind, const float4 &c, unsigned m, const float4 &q0, const float4 &q1) {
        if (kQuad) {
            const bool qf = kind == kFullCell, qp = kind == kPartCell;
            const unsigned qfb = __ballot_sync(kFull, qf), qpb = __ballot_sync(kFull, qp);
            if (qf || qp) {
                if (qf) {
                    put_quad_entry(Q.f, qfn + __popc(qfb & lt), c, q0, q1);
                } else {
                    const int o = qpn + __popc(qpb & lt);
                    put_quad_entry(Q.p, o, c, q0, q1);
                    Q.pm[o] = m;
                }
            }
            qfn += __popc(qfb);
            qpn += __popc(qpb);
            upc += __popc(qfb);
            if (qf || qp) kind = kNone;
        }
        const bool isf = kind == kFullLeaf || kind == kFullCell;
        const unsigned fb = __ballot_sync(kFull, isf);
        if (isf) put_entry(S.f, fn + __popc(fb & lt), c);
        fn += __popc(fb);
        const unsigned fl = __ballot_sync(kFull, kind == kFullLeaf);
        upp += __popc(fl);
        upc += __popc(fb & ~fl);
        const bool isp = kind == kPartLeaf || kind == kPartCell;
        const unsigned pb = __ballot_sync(kFull, isp);
        if (isp) {
            const int o = pn + __popc(pb & lt);
            put_entry(S.p, o, c);
            S.pm[o] = make_uint2(m, kind == kPartLeaf ? 1u : 0u);
        }
        pn += __popc(pb);
    };
    // evaluates and empties both buffers (an odd count is padded with a zero-weight source)
    auto drain = [&]() {
        if (lane == 0) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (fn & 1) put_entry(S.f, fn, z);
            if (pn & 1) {
                put_entry(S.p, pn, z);
                S.pm[pn] = make_uint2(0u, 0u);
            }
            if (kQuad && (qfn & 1)) put_quad_entry(Q.f, qfn, z, z, z);
            if (kQuad && (qpn & 1)) {
                put_quad_entry(Q.p, qpn, z, z, z);
                Q.pm[qpn] = 0u;
            }
        }
        __syncwarp();
        if (fn > 0) ev.full(S, fn, nme, eps2);
        if (pn > 0) ev.part(S, pn, nme, eps2, lane);
        if (kQuad) {
            if (qfn > 0) ev.full_quad(Q, qfn, nme, eps2);
            if (qpn > 0) ev.part_quad(Q, qpn, nme, eps2, lane);
            qfn = qpn = 0;
        }
        fn = pn = 0;
        __syncwarp();
    };

    // every node is popped at most once per group, so more steps than nodes means a malformed
    // tree: stop with the error word set rather than loop
    const int stack_cap = min(kStackCap, a.stack_limit);
    int64_t steps_left = min((int64_t)n_nodes, a.step_limit);
    while (sp > 0) {
        if (sp > stack_cap - 32 || --steps_left < 0) {  // cannot happen (see kStackCap)
            if (lane == 0) atomicOr(a.err, kErrStack);
            break;
        }
        __syncwarp();
        // ---- pop up to 32 nodes from the top ranges (lane k reads the k-th range from the top)
        const int ne = min(sp, 32);
        uint32_t pk = 0, pmk = 0;
        unsigned cm1 = 0;  // range size - 1 (0..7)
        if (lane < ne) {
            pk = S.st_node[sp - 1 - lane];
            pmk = S.st_mask[sp - 1 - lane];
            cm1 = pk >> 28;
        }
        // exclusive prefix sum of the range sizes: one per range before this lane's plus the
        // sizes - 1 from their bits, one ballot per bit
        const unsigned b0 = __ballot_sync(kFull, cm1 & 1u), b1 = __ballot_sync(kFull, cm1 & 2u);
        const unsigned b2 = __ballot_sync(kFull, cm1 & 4u);
        const int excl = min(lane, ne) + __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
        const int total = ne + __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
        const bool touched = lane < ne && excl < 32;
        const int nt = __popc(__ballot_sync(kFull, touched));       // ranges touched: 0 .. nt-1
        const int last_excl = __shfl_sync(kFull, excl, nt - 1);
        const uint32_t last_pk = __shfl_sync(kFull, pk, nt - 1);
        const int last_incl = last_excl + (int)(last_pk >> 28) + 1;
        const int items = min(total, 32);
        const unsigned starts = __reduce_or_sync(kFull, touched ? (1u << excl) : 0u);
        const unsigned le = starts & (lane == 31 ? kFull : ((2u << lane) - 1u));
        const int k = __popc(le) - 1;
        const int off = lane - (31 - __clz(le));
        const uint32_t ek = __shfl_sync(kFull, pk, k & 31);
        const uint32_t em = __shfl_sync(kFull, pmk, k & 31);
        __syncwarp();  // every popped entry is read before the stack is written again
        if (last_incl > 32) {
            // the deepest touched range is split: its first (32 - last_excl) nodes are taken
            const int taken = 32 - last_excl;
            sp -= nt - 1;
            if (lane == 0)
                S.st_node[sp - 1] = ((last_pk & kIdxMask) + (uint32_t)taken) |
                                    ((uint32_t)((int)(last_pk >> 28) - taken) << 28);
        } else {
            sp -= nt;
        }

        // ---- load the popped nodes (one per lane)
        const int node0 = (int)(ek & kIdxMask) + off;
        const bool bad = lane < items && node0 >= n_nodes;
        if (bad) atomicOr(a.err, kErrStack);
        const bool has = lane < items && !bad;
        const int node = has ? node0 : 0;
        const unsigned m = has ? em : 0u;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        int4 meta = make_int4(0, 0, 0, 0);
        float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
        if (has) {
            c = ldg4(&a.gn[node].c);
            meta = __ldg(reinterpret_cast<const int4 *>(&a.gn[node].child));
        }
        if (kQuad && has) {  // the quadrupole (every node has one), in case it is accepted
            q0 = ldg4(a.gq + 2 * (size_t)node);
            q1 = ldg4(a.gq + 2 * (size_t)node + 1);
        }

        // ---- while the loads are in flight: evaluate what the previous step buffered
        drain();

        // ---- classify
        int kind = kNone;
        unsigned emask = m;     // bodies that take this node's entry
        if (has) {
            if (meta.y < 0) {
                if (meta.y == -1) {
                    const unsigned d = (unsigned)(meta.x - g0);
                    if (kGroup) {
                        kind = kFullLeaf;
                    } else {
                        if (d < 32u) emask &= ~(1u << d);   // the body itself
                        kind = emask == 0u ? kNone : (emask == live_mask ? kFullLeaf : kPartLeaf);
                    }
                } else {
                    kind = kBucket;
                }
            } else if (kGroup) {
                const float crit = __int_as_float(meta.z);
                float nx, ny, nz, fx, fy, fz;
                axis_bounds(c.x, lox, hix, nx, fx);
                axis_bounds(c.y, loy, hiy, ny, fy);
                axis_bounds(c.z, loz, hiz, nz, fz);
                const float dmin2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
                kind = dmin2 > crit ? kFullCell : kOpen;
            } else {
                const float crit = __int_as_float(meta.z);
                float nx, ny, nz, fx, fy, fz;
                axis_bounds(c.x, lox, hix, nx, fx);
                axis_bounds(c.y, loy, hiy, ny, fy);
                axis_bounds(c.z, loz, hiz, nz, fz);
                const float dmin2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
                const float dmax2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
                if (dmin2 > crit) kind = m == live_mask ? kFullCell : kPartCell;
                else if (dmax2 <= crit) kind = kOpen;
                else kind = kMixed;
            }
        }

        if (kGroup) {  // the bodies whose own leaf is among this step's entries
            const unsigned d = (unsigned)(meta.x - g0);
            self_seen |= __reduce_or_sync(kFull, (kind == kFullLeaf && d < 32u) ? 1u << d : 0u);
        }

        // ---- mixed cells: every body tests its own acceptance, two cells per pass
        // (the cells' x, y, z, crit go through the full-entry buffer and the bodies' acceptance
        // masks back through the mask buffer: both are empty between the drain and the emit)
        const unsigned mx = kGroup ? 0u : __ballot_sync(kFull, kind == kMixed);
        unsigned myA = 0u;
        if (mx) {
            const int nm = __popc(mx);
            const int r = __popc(mx & lt);
            if (kind == kMixed)
                put_entry(S.f, r, make_float4(c.x, c.y, c.z, __int_as_float(meta.z)));
            __syncwarp();
            uint32_t *A = reinterpret_cast<uint32_t *>(S.pm);
            for (int k = 0; k < nm; k += 2) {
                const float4 u = S.f[k], v = S.f[k + 1];
                const float2 dx = __fadd2_rn(make_float2(u.x, u.y), nme[0]);
                const float2 dy = __fadd2_rn(make_float2(u.z, u.w), nme[1]);
                const float2 dz = __fadd2_rn(make_float2(v.x, v.y), nme[2]);
                const float2 q = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                const unsigned A1 = __ballot_sync(kFull, q.x > v.z);
                const unsigned A2 = __ballot_sync(kFull, q.y > v.w);
                if (lane == 0) {
                    A[k] = A1;
                    A[k + 1] = A2;
                }
            }
            __syncwarp();
            if (kind == kMixed) myA = A[r];
            __syncwarp();
        }
        unsigned pmask = kind == kOpen ? m : 0u;   // bodies that need this cell's children
        if (kind == kMixed) {
            emask = myA & m;
            pmask = m & ~emask;
            kind = emask == 0u ? kNone : (emask == live_mask ? kFullCell : kPartCell);
        }

        // ---- buffer the entries, push the children
        emit(kind, c, emask, q0, q1);
        {
            const bool isp = pmask != 0u;
            const unsigned ob = __ballot_sync(kFull, isp);
            if (isp) {
                const int o = sp + __popc(ob & lt);
                S.st_node[o] = (uint32_t)meta.x | ((uint32_t)(meta.y - 1) << 28);
                S.st_mask[o] = pmask;
            }
            sp += __popc(ob);
        }

        // ---- level-21 buckets (rare): every member but the body itself, 32 members at a time
        unsigned bk = __ballot_sync(kFull, kind == kBucket);
        while (bk) {
            const int src = __ffs(bk) - 1;
            bk &= bk - 1u;
            const int b0i = __shfl_sync(kFull, meta.x, src);
            const int nb = -__shfl_sync(kFull, meta.y, src);
            const unsigned sm = __shfl_sync(kFull, m, src);
            for (int base = 0; base < nb; base += 32) {
                if (fn > kFCap - 32 || pn > kPCap - 32) drain();
                const bool h = base + lane < nb;
                const int b = min(b0i + base + lane, b0i + nb - 1);
                const float4 s = h ? ldg4(a.sbody32 + b) : make_float4(0.f, 0.f, 0.f, 0.f);
                unsigned mb = sm;
                const unsigned d = (unsigned)(b - g0);
                int kb;
                if (kGroup) {
                    kb = h ? kFullLeaf : kNone;
                    self_seen |= __reduce_or_sync(kFull, (h && d < 32u) ? 1u << d : 0u);
                } else {
                    if (d < 32u) mb &= ~(1u << d);
                    kb = (!h || mb == 0u) ? kNone : (mb == live_mask ? kFullLeaf : kPartLeaf);
                }
                emit(kb, s, mb, s, s);
            }
        }
    }
    drain();
    const float3 r = ev.acc.result();
    const uint32_t self_term = kGroup ? (self_seen >> lane) & 1u : 0u;
    if (live)
        write_out(a, i, (double)r.x, (double)r.y, (double)r.z, ev.pp + upp - self_term,
                  ev.pc - ev.pp + upc);
}

template <int kWarps, bool kKahan, bool kGuard, bool kGroup, bool kQuad>
__global__ void __launch_bounds__(kWarps * 32) group_walk32_kernel(WalkArgs a)
{
    extern __shared__ __align__(16) unsigned char group_smem[];
    unsigned char *slice = group_smem + group_smem_bytes<kQuad>() * (threadIdx.x >> 5);
    GroupSmem &S = *reinterpret_cast<GroupSmem *>(slice);
    QuadSmem &Q = *reinterpret_cast<QuadSmem *>(slice + sizeof(GroupSmem));  // used with kQuad
    const int lane = threadIdx.x & 31;
    // persistent warps: each takes the next group from the shared counter until none is left
    for (;;) {
        unsigned gi = 0;
        if (lane == 0) gi = atomicAdd(a.work, 1u);
        gi = __shfl_sync(kFull, gi, 0);
        int g0, gcount, root;
        if (!group_of(a, (int)gi, g0, gcount, root)) break;  // uniform per warp
        walk_group<kKahan, kGuard, kGroup, kQuad>(a, S, Q, lane, g0, gcount, root);
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------
// Per-body acceptance test, monopole cells: the default FP32 walk of a single system, in two
// kernels.
//
// Neighbouring groups share most of their walks: a cell far from a span of 256 consecutive bodies
// (eight groups) is accepted by every body of the span, and the cells above it are opened by every
// body.  far_walk32_kernel walks the tree once per span and tests cells against the span's
// bounding box with the bounds of the group walk (below): cells that every body of the span
// accepts and leaves outside the span go to the span's far list, one entry for all its bodies;
// cells that every body opens are descended; every other node (a cell that the span's bodies
// decide differently, a leaf holding a body of the span, a bucket) goes to the span's frontier,
// sorted deepest level first.  Each body's own walk reaches exactly these nodes, with all their
// ancestors opened, so a group evaluates the far list as full-group entries and walks on from the
// frontier with its own bounding box and body masks (walk_group_pb): every body keeps exactly its
// own interaction list.  A span whose lists do not fit in the scratch is marked, and its groups
// walk from the root.
//
// The group walk is arranged for few instructions per step:
//   - a stack entry is one 8-byte pair (child range, body mask): one load per popped range;
//   - the interaction buffers are evaluated only when the next step might not fit in them;
//   - partial entries are kept apart by kind, leaves from the front of their buffer and cells
//     from its back, so the per-body counts need no per-entry kind flag;
//   - a mixed cell's per-body acceptance masks stay in registers.
// Stack bound.  Children are pushed in reverse lane order.  Popped nodes reach the lanes in stack
// order, so while the stack is sorted by level (deepest on top) the lane order is non-increasing
// in level and the reversed pushes keep the stack sorted.  A step that pops a level-l node then has
// popped every deeper entry, so after it the stack holds only the level-(l+1) ranges that this
// step pushed (at most 32), a count that only falls until the next such step: at most 32 ranges
// for each level 1..21.  Frontier chunks (deepest first) are taken only when the stack is empty.
// ------------------------------------------------------------------------------------------

constexpr int kPbStack = 22 * 32;  // at least 32 ranges for each level 1..21 (see above)
// The walk runs with a stack of kPbFast entries (walks rarely go deeper: the two-cluster
// benchmark peaks near 120), which leaves room for more warps per SM.  A group whose stack would
// overflow it writes nothing and goes to the overflow list, walked afterwards with kPbStack.
constexpr int kPbFast = 8 * 32;

// kBuf entries in each interaction buffer (a launch shape: 128 or 64); kStackN stack entries.
template <int kBuf, int kStackN>
struct PbSmem {
    uint2 st[kStackN];    // (first node | (count - 1) << 28, bodies that still need the range)
    float4 f[kBuf];       // full-group sources, pair-interleaved (put_entry)
    float4 p[kBuf];       // partial sources, pair-interleaved: leaves at 0.., cells at ..kBuf-1
    uint32_t pm[kBuf];    // their body masks
    float4 mx[32];        // this step's mixed cells (x, y, z, crit), pair-interleaved
};

// Along one axis: the smallest |c - x| over x in [lo, hi] as the FP32 subtraction rounds it (0
// inside; rounding is monotone, so the ends bound every body), and the largest.
__device__ __forceinline__ void axis_bounds_pb(float c, float lo, float hi, float &dmin,
                                               float &dmax)
{
    const float a = c - lo, b = c - hi;  // a >= b
    dmin = fmaxf(fmaxf(b, -a), 0.f);
    dmax = fmaxf(fabsf(a), fabsf(b));
}

// d^2 bounds of a cell at c from the bodies in the box [lo, hi] (the per-body expression
// fmaf(dx, dx, fmaf(dy, dy, dz * dz)) is monotone in |dx|, |dy|, |dz|).
__device__ __forceinline__ void box_d2(const float4 &c, float lox, float loy, float loz, float hix,
                                       float hiy, float hiz, float &dmin2, float &dmax2)
{
    float nx, ny, nz, fx, fy, fz;
    axis_bounds_pb(c.x, lox, hix, nx, fx);
    axis_bounds_pb(c.y, loy, hiy, ny, fy);
    axis_bounds_pb(c.z, loz, hiz, nz, fz);
    dmin2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
    dmax2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
}

// Partial entries k0 .. k1-1 (pairs): the bodies outside an entry's mask take it with weight 0.
// Returns how many of them this lane's body takes.
template <bool kKahan, bool kGuard>
__device__ __forceinline__ uint32_t eval_partial(const float4 *__restrict__ p,
                                                 const uint32_t *__restrict__ pm, int k0, int k1,
                                                 unsigned lanebit, const float2 *nme, float2 eps2,
                                                 Acc3x2<kKahan> &acc)
{
    uint32_t cnt = 0;
    const uint2 *pm2 = reinterpret_cast<const uint2 *>(pm);
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
        const float4 a = p[2 * k];
        float4 b = p[2 * k + 1];
        const uint2 q = pm2[k];
        const bool on0 = (q.x & lanebit) != 0u, on1 = (q.y & lanebit) != 0u;
        b.z = on0 ? b.z : 0.f;
        b.w = on1 ? b.w : 0.f;
        pair32x2<kGuard>(a, b, nme[0], nme[1], nme[2], eps2, acc.x, acc.y, acc.z);
        cnt += (uint32_t)on0 + (uint32_t)on1;
    }
    return cnt;
}

template <bool kKahan, bool kGuard, int kBuf, int kStackN>
__device__ __forceinline__ void walk_group_pb(const WalkArgs &a, PbSmem<kBuf, kStackN> &S,
                                              int lane, int g0, int gcount, int root, int sys)
{
    constexpr int kPbF = kBuf, kPbP = kBuf;
    const int i = g0 + lane;
    const int n_nodes = (int)*a.d_nn;
    const unsigned lt = lanemask_lt_w();
    const unsigned lanebit = 1u << lane;
    const unsigned live = gcount >= 32 ? kFull : ((1u << gcount) - 1u);
    // lanes past the group's end stand on its last body so that they do not widen its box
    const float4 me = ldg4(a.sbody32 + g0 + min(lane, gcount - 1));
    const float lox = warp_fmin(me.x), loy = warp_fmin(me.y), loz = warp_fmin(me.z);
    const float hix = warp_fmax(me.x), hiy = warp_fmax(me.y), hiz = warp_fmax(me.z);
    const float eps2s = (float)(a.eps * a.eps);
    const float2 eps2 = make_float2(eps2s, eps2s);
    const float2 nme[3] = {make_float2(-me.x, -me.x), make_float2(-me.y, -me.y),
                           make_float2(-me.z, -me.z)};

    Acc3x2<kKahan> acc;
    int terms = 0;                 // terms in the current FP32 partials (warp-uniform)
    uint32_t ufl = 0, ufc = 0;     // full-group leaves / cells (the same for every live body)
    uint32_t npl = 0, npc = 0;     // partial leaves / cells taken by this lane's body
    int sp = 0, fn = 0, pl = 0, pc = 0;  // stack depth and buffer fills (warp-uniform)

    auto fold_if_due = [&](int added) {
        terms += added;
        if (terms >= Acc3x2<kKahan>::kFold) {
            acc.fold();
            terms = 0;
        }
    };
    // evaluates and empties the buffers (odd counts padded with a zero-weight source)
    auto drain = [&]() {
        if (lane == 0) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (fn & 1) put_entry(S.f, fn, z);
            if (pl & 1) {
                put_entry(S.p, pl, z);
                S.pm[pl] = 0u;
            }
            if (pc & 1) {
                put_entry(S.p, kPbP - 1 - pc, z);
                S.pm[kPbP - 1 - pc] = 0u;
            }
        }
        __syncwarp();
        const int nf = (fn + 1) >> 1;
#pragma unroll 2
        for (int k = 0; k < nf; ++k)
            pair32x2<kGuard>(S.f[2 * k], S.f[2 * k + 1], nme[0], nme[1], nme[2], eps2, acc.x,
                             acc.y, acc.z);
        fold_if_due(2 * nf);
        const int nl = (pl + 1) >> 1;
        npl += eval_partial<kKahan, kGuard>(S.p, S.pm, 0, nl, lanebit, nme, eps2, acc);
        fold_if_due(2 * nl);
        const int c0 = (kPbP - ((pc + 1) & ~1)) >> 1;
        npc += eval_partial<kKahan, kGuard>(S.p, S.pm, c0, kPbP / 2, lanebit, nme, eps2, acc);
        fold_if_due(kPbP - 2 * c0);
        fn = pl = pc = 0;
        __syncwarp();
    };
    // appends one entry per lane with a nonzero mask: to f when every live body takes it, else
    // to the partial leaves or cells
    auto emit = [&](bool leaf, const float4 &c, unsigned emask) {
        const bool full = emask == live;
        const bool part = emask != 0u && !full;
        const unsigned fb = __ballot_sync(kFull, full);
        const unsigned pb = __ballot_sync(kFull, part);
        const unsigned lb = __ballot_sync(kFull, leaf);
        const unsigned plb = pb & lb, pcb = pb & ~lb;
        if (full) put_entry(S.f, fn + __popc(fb & lt), c);
        if (part) {
            const int o = leaf ? pl + __popc(plb & lt) : kPbP - 1 - pc - __popc(pcb & lt);
            put_entry(S.p, o, c);
            S.pm[o] = emask;
        }
        const int nf = __popc(fb), nfl = __popc(fb & lb);
        fn += nf;
        pl += __popc(plb);
        pc += __popc(pcb);
        ufl += nfl;
        ufc += nf - nfl;
    };

    // start: the span's far list and frontier, or the root's children (the root is never
    // tested; none when the root is a leaf, i.e. a single body)
    int far_n = -1, fr_n = 0, fr_next = 0;
    const uint32_t *far = nullptr;
    if (a.span_meta && !a.groups) {
        const int si = g0 / a.span_bodies;
        const int4 m = a.span_meta[si];
        if (m.x >= 0) {
            far = a.span_pool + a.span_off[si];
            far_n = m.x;
            fr_n = m.y;
            ufl = (uint32_t)m.z;
            ufc = (uint32_t)m.w;
        }
    }
    if (far) {
        for (int base = 0; base < far_n; base += 32) {
            const int cnt = min(32, far_n - base);
            if (fn > kPbF - 32) drain();
            if (lane < cnt) put_entry(S.f, fn + lane, ldg4(&a.gn[__ldg(far + base + lane)].c));
            fn += cnt;
        }
    } else if (root >= 0 && root < n_nodes) {
        const int4 r = __ldg(reinterpret_cast<const int4 *>(&a.gn[root].child));
        if (r.y > 0) {
            if (lane == 0) S.st[0] = make_uint2((uint32_t)r.x | ((uint32_t)(r.y - 1) << 28), live);
            sp = 1;
        }
    }
    const uint32_t *fr = far ? far + far_n : nullptr;

    // every node is popped at most once per group, so more steps than nodes means a malformed
    // tree: stop with the error word set rather than loop
    // the fast kernel hands a group that would overflow its stack to the overflow walk (the
    // test aid lowers that point); the full-stack walk reports it (cannot happen: stack bound)
    constexpr bool kFast = kStackN < kPbStack;
    const int stack_cap = min(kStackN, kFast ? min(a.stack_limit, a.fast_stack_limit)
                                             : a.stack_limit);
    int64_t steps_left = min((int64_t)n_nodes, a.step_limit);
    bool handed = false;  // the group went to the overflow walk: write nothing
    while (sp > 0 || fr_next < fr_n) {
        if (sp > stack_cap - 32 || --steps_left < 0) {
            handed = kFast && a.overflow && sp > stack_cap - 32;
            if (!handed && lane == 0) atomicOr(a.err, kErrStack);  // cannot happen
            break;
        }
        __syncwarp();
        uint32_t ek, em;
        int off, items;
        if (sp > 0) {
            // ---- pop up to 32 nodes from the top ranges (lane k reads the k-th from the top)
            const int ne = min(sp, 32);
            uint2 e = make_uint2(0u, 0u);
            if (lane < ne) e = S.st[sp - 1 - lane];
            const unsigned cm1 = e.x >> 28;  // range size - 1 (0..7); 0 past ne
            // exclusive prefix sum of the range sizes: one per range before this lane's plus
            // the sizes - 1 from their bits, one ballot per bit
            const unsigned b0 = __ballot_sync(kFull, cm1 & 1u), b1 = __ballot_sync(kFull, cm1 & 2u);
            const unsigned b2 = __ballot_sync(kFull, cm1 & 4u);
            const int excl =
                min(lane, ne) + __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
            const int total = ne + __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
            const bool touched = lane < ne && excl < 32;
            const int nt = __popc(__ballot_sync(kFull, touched));  // ranges touched: 0 .. nt-1
            const int end = excl + (int)cm1 + 1;
            const bool split = __shfl_sync(kFull, end, nt - 1) > 32;  // the deepest is cut
            const unsigned starts = __reduce_or_sync(kFull, touched ? (1u << excl) : 0u);
            const unsigned le = starts & (lane == 31 ? kFull : ((2u << lane) - 1u));
            const int k = __popc(le) - 1;
            off = lane - (31 - __clz(le));
            ek = __shfl_sync(kFull, e.x, k & 31);
            em = __shfl_sync(kFull, e.y, k & 31);
            __syncwarp();  // every popped entry is read before the stack is written again
            if (split && lane == nt - 1) {  // its first (32 - excl) nodes are taken
                const int taken = 32 - excl;
                S.st[sp - nt] = make_uint2(((e.x & kIdxMask) + (uint32_t)taken) |
                                               ((uint32_t)((int)cm1 - taken) << 28),
                                           e.y);
            }
            sp -= nt - (split ? 1 : 0);
            items = min(total, 32);
        } else {
            // ---- the next frontier chunk (deepest first), for every live body
            items = min(32, fr_n - fr_next);
            ek = lane < items ? __ldg(fr + fr_next + lane) : 0u;
            em = live;
            off = 0;
            fr_next += items;
        }

        // ---- load the popped nodes (one per lane; idle lanes read node 0 and take nothing)
        const int node0 = (int)(ek & kIdxMask) + off;
        const bool has0 = lane < items;
        const bool bad = has0 && node0 >= n_nodes;
        if (bad) atomicOr(a.err, kErrStack);
        const bool has = has0 && !bad;
        const int node = has ? node0 : 0;
        const unsigned m = has ? em : 0u;
        const float4 c = ldg4(&a.gn[node].c);
        const int4 meta = __ldg(reinterpret_cast<const int4 *>(&a.gn[node].child));

        // ---- while the loads are in flight: evaluate the buffers if this step might not fit
        if (fn > kPbF - 32 || pl + pc > kPbP - 34) drain();

        // ---- classify
        const bool leaf = meta.y < 0;
        const float crit = __int_as_float(meta.z);
        float dmin2, dmax2;
        box_d2(c, lox, loy, loz, hix, hiy, hiz, dmin2, dmax2);
        const bool acc_all = dmin2 > crit;    // every body of the group accepts the cell
        const bool open_all = dmax2 <= crit;  // every body opens it
        const unsigned d = (unsigned)(meta.x - g0);
        const unsigned self = d < 32u ? (1u << d) : 0u;
        unsigned emask, pmask;
        if (leaf) {
            emask = meta.y == -1 ? (m & ~self) : 0u;  // buckets below
            pmask = 0u;
        } else {
            emask = acc_all ? m : 0u;
            pmask = open_all ? m : 0u;
        }
        const bool mixed = !leaf && !acc_all && !open_all && m != 0u;

        // ---- mixed cells: every body tests its own acceptance, two cells per pass
        const unsigned mxb = __ballot_sync(kFull, mixed);
        if (mxb) {
            const int nm = __popc(mxb);
            const int r = __popc(mxb & lt);
            if (mixed) put_entry(S.mx, r, make_float4(c.x, c.y, c.z, crit));
            __syncwarp();
            unsigned myA = 0u;
            for (int t = 0; t < nm; t += 2) {
                const float4 u = S.mx[t], v = S.mx[t + 1];
                const float2 dx = __fadd2_rn(make_float2(u.x, u.y), nme[0]);
                const float2 dy = __fadd2_rn(make_float2(u.z, u.w), nme[1]);
                const float2 dz = __fadd2_rn(make_float2(v.x, v.y), nme[2]);
                const float2 q = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                const unsigned A1 = __ballot_sync(kFull, q.x > v.z);
                const unsigned A2 = __ballot_sync(kFull, q.y > v.w);
                myA = r == t ? A1 : (r == t + 1 ? A2 : myA);
            }
            __syncwarp();  // the cells are read before the next step writes them
            if (mixed) {
                emask = m & myA;
                pmask = m & ~myA;
            }
        }

        // ---- buffer the entries, push the children (reverse lane order: deepest on top)
        emit(leaf, c, emask);
        {
            const unsigned ob = __ballot_sync(kFull, pmask != 0u);
            const int no = __popc(ob);
            if (pmask)
                S.st[sp + no - 1 - __popc(ob & lt)] =
                    make_uint2((uint32_t)meta.x | ((uint32_t)(meta.y - 1) << 28), pmask);
            sp += no;
        }

        // ---- level-21 buckets (rare): every member but the body itself, 32 members at a time
        unsigned bk = __ballot_sync(kFull, leaf && meta.y < -1 && m != 0u);
        while (bk) {
            const int src = __ffs(bk) - 1;
            bk &= bk - 1u;
            const int b0i = __shfl_sync(kFull, meta.x, src);
            const int nb = -__shfl_sync(kFull, meta.y, src);
            const unsigned sm = __shfl_sync(kFull, m, src);
            for (int base = 0; base < nb; base += 32) {
                if (fn > kPbF - 32 || pl + pc > kPbP - 34) drain();
                const bool h = base + lane < nb;
                const int b = min(b0i + base + lane, b0i + nb - 1);
                const float4 s = ldg4(a.sbody32 + b);
                const unsigned db = (unsigned)(b - g0);
                const unsigned mb = h ? (sm & ~(db < 32u ? (1u << db) : 0u)) : 0u;
                emit(true, s, mb);
            }
        }
    }
    if (handed) {  // nothing written: the overflow walk does this group
        if (lane == 0) a.overflow[atomicAdd(a.n_overflow, 1u)] = make_int4(g0, gcount, sys, 0);
        return;
    }
    drain();
    const float3 r = acc.result();
    if (lane < gcount)
        write_out(a, i, (double)r.x, (double)r.y, (double)r.z, ufl + npl, ufc + npc);
}

template <int kWarps, bool kKahan, bool kGuard, int kBuf, int kStackN>
__global__ void __launch_bounds__(kWarps * 32) pb_walk32_kernel(WalkArgs a)
{
    extern __shared__ __align__(16) unsigned char pb_smem[];
    PbSmem<kBuf, kStackN> &S = reinterpret_cast<PbSmem<kBuf, kStackN> *>(pb_smem)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    // persistent warps: each takes the next group from the shared counter until none is left
    for (;;) {
        unsigned gi = 0;
        if (lane == 0) gi = atomicAdd(a.work, 1u);
        gi = __shfl_sync(kFull, gi, 0);
        int g0, gcount, root;
        if (!group_of(a, (int)gi, g0, gcount, root)) break;  // uniform per warp
        const int sys = a.groups ? a.groups[gi].z : 0;
        walk_group_pb<kKahan, kGuard, kBuf, kStackN>(a, S, lane, g0, gcount, root, sys);
        __syncwarp();
    }
}

// ---- the far walk of the spans (see above) ------------------------------------------------

struct FarSmem {
    uint2 st[kPbStack];   // (first node | (count - 1) << 28, level of the range's nodes)
    uint32_t cnt[kLevels];
};

// One warp per span, persistent.  Far list and frontier go to the warp's own scratch first
// (span_tmp: kSpanFarTmp + 2 kSpanFrTmp words per warp), then to the shared pool at an offset
// reserved from span_next, the frontier sorted by level, deepest first (counting sort, stable).
// A span whose lists exceed the scratch or the pool gets far count -1: its groups walk from the root.
template <int kWarps>
__global__ void __launch_bounds__(kWarps * 32) far_walk32_kernel(WalkArgs a)
{
    __shared__ FarSmem smem[kWarps];
    FarSmem &S = smem[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt_w();
    const size_t wg = (size_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    uint32_t *tfar = a.span_tmp + wg * (kSpanFarTmp + 2 * kSpanFrTmp);
    uint32_t *tfr = tfar + kSpanFarTmp;   // frontier nodes
    uint32_t *tlev = tfr + kSpanFrTmp;    // their levels
    const int n_nodes = (int)*a.d_nn;
    const int span = a.span_bodies;
    const int n_spans = (a.n + span - 1) / span;
    for (;;) {
        unsigned si = 0;
        if (lane == 0) si = atomicAdd(a.span_next + 1, 1u);
        si = __shfl_sync(kFull, si, 0);
        if ((int)si >= n_spans) break;
        const int s0 = (int)si * span, s1 = min(s0 + span, a.n);
        float lx = INFINITY, ly = INFINITY, lz = INFINITY;
        float hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
        for (int b = s0 + lane; b < s1; b += 32) {
            const float4 q = ldg4(a.sbody32 + b);
            lx = fminf(lx, q.x);
            ly = fminf(ly, q.y);
            lz = fminf(lz, q.z);
            hx = fmaxf(hx, q.x);
            hy = fmaxf(hy, q.y);
            hz = fmaxf(hz, q.z);
        }
        lx = warp_fmin(lx);
        ly = warp_fmin(ly);
        lz = warp_fmin(lz);
        hx = warp_fmax(hx);
        hy = warp_fmax(hy);
        hz = warp_fmax(hz);

        int sp = 0, fn = 0, frn = 0;
        uint32_t nfl = 0, nfc = 0;
        bool over = false;
        {
            const int4 r = __ldg(reinterpret_cast<const int4 *>(&a.gn[0].child));
            if (r.y > 0) {
                if (lane == 0) S.st[0] = make_uint2((uint32_t)r.x | ((uint32_t)(r.y - 1) << 28), 1u);
                sp = 1;
            }
        }
        const int stack_cap = min(kPbStack, a.stack_limit);
        int64_t steps_left = min((int64_t)n_nodes, a.step_limit);
        while (sp > 0) {
            if (sp > stack_cap - 32 || --steps_left < 0) {  // cannot happen (see the stack bound)
                if (lane == 0) atomicOr(a.err, kErrStack);
                over = true;
                break;
            }
            __syncwarp();
            // ---- pop up to 32 nodes (as in walk_group_pb)
            const int ne = min(sp, 32);
            uint2 e = make_uint2(0u, 0u);
            if (lane < ne) e = S.st[sp - 1 - lane];
            const unsigned cm1 = e.x >> 28;
            const unsigned b0 = __ballot_sync(kFull, cm1 & 1u), b1 = __ballot_sync(kFull, cm1 & 2u);
            const unsigned b2 = __ballot_sync(kFull, cm1 & 4u);
            const int excl =
                min(lane, ne) + __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
            const int total = ne + __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
            const bool touched = lane < ne && excl < 32;
            const int nt = __popc(__ballot_sync(kFull, touched));
            const int end = excl + (int)cm1 + 1;
            const bool split = __shfl_sync(kFull, end, nt - 1) > 32;
            const unsigned starts = __reduce_or_sync(kFull, touched ? (1u << excl) : 0u);
            const unsigned le = starts & (lane == 31 ? kFull : ((2u << lane) - 1u));
            const int k = __popc(le) - 1;
            const int off = lane - (31 - __clz(le));
            const uint32_t ek = __shfl_sync(kFull, e.x, k & 31);
            const uint32_t lev = __shfl_sync(kFull, e.y, k & 31);
            __syncwarp();
            if (split && lane == nt - 1) {
                const int taken = 32 - excl;
                S.st[sp - nt] = make_uint2(((e.x & kIdxMask) + (uint32_t)taken) |
                                               ((uint32_t)((int)cm1 - taken) << 28),
                                           e.y);
            }
            sp -= nt - (split ? 1 : 0);

            const int node0 = (int)(ek & kIdxMask) + off;
            const bool has0 = lane < min(total, 32);
            const bool bad = has0 && node0 >= n_nodes;
            if (bad) atomicOr(a.err, kErrStack);
            const bool has = has0 && !bad;
            const int node = has ? node0 : 0;
            const float4 c = ldg4(&a.gn[node].c);
            const int4 meta = __ldg(reinterpret_cast<const int4 *>(&a.gn[node].child));

            // ---- classify against the span's box
            const bool leaf = meta.y < 0;
            float dmin2, dmax2;
            box_d2(c, lx, ly, lz, hx, hy, hz, dmin2, dmax2);
            const float crit = __int_as_float(meta.z);
            bool to_far, to_push;
            if (leaf) {  // a single body outside the span: every body of the span takes it
                to_far = meta.y == -1 && (meta.x < s0 || meta.x >= s1);
                to_push = false;
            } else {
                to_far = dmin2 > crit;
                to_push = !to_far && dmax2 <= crit;
            }
            to_far = to_far && has;
            to_push = to_push && has;
            const bool to_fr = has && !to_far && !to_push;

            const unsigned fb = __ballot_sync(kFull, to_far), rb = __ballot_sync(kFull, to_fr);
            const unsigned lfb = fb & __ballot_sync(kFull, leaf);
            if (fn + __popc(fb) > kSpanFarTmp || frn + __popc(rb) > kSpanFrTmp) {
                over = true;
                break;
            }
            if (to_far) tfar[fn + __popc(fb & lt)] = (uint32_t)node;
            if (to_fr) {
                const int o = frn + __popc(rb & lt);
                tfr[o] = (uint32_t)node;
                tlev[o] = lev;
            }
            fn += __popc(fb);
            frn += __popc(rb);
            nfl += __popc(lfb);
            nfc += __popc(fb & ~lfb);
            const unsigned ob = __ballot_sync(kFull, to_push);
            const int no = __popc(ob);
            if (to_push)
                S.st[sp + no - 1 - __popc(ob & lt)] =
                    make_uint2((uint32_t)meta.x | ((uint32_t)(meta.y - 1) << 28), lev + 1u);
            sp += no;
        }
        // ---- reserve room in the pool and copy: far list, then the frontier by level, deepest
        // first
        unsigned off = 0;
        const int tot = fn + frn;
        if (!over && lane == 0) off = atomicAdd(a.span_next, (unsigned)tot);
        off = __shfl_sync(kFull, off, 0);
        if (!over && (int64_t)off + tot > a.span_pool_cap) over = true;
        if (over) {
            if (lane == 0) a.span_meta[si] = make_int4(-1, 0, 0, 0);
            continue;
        }
        uint32_t *dst = a.span_pool + off;
        for (int q = lane; q < fn; q += 32) dst[q] = tfar[q];
        if (lane < kLevels) S.cnt[lane] = 0u;
        __syncwarp();
        for (int base = 0; base < frn; base += 32) {
            const int q = base + lane;
            const uint32_t lv = q < frn ? tlev[q] : 0xffu;
            const unsigned peers = __match_any_sync(kFull, lv);
            if (q < frn && lane == __ffs(peers) - 1) S.cnt[lv] += __popc(peers);
            __syncwarp();
        }
        if (lane == 0) {
            uint32_t run = 0;
            for (int lv = kLevels - 1; lv >= 0; --lv) {
                const uint32_t cn = S.cnt[lv];
                S.cnt[lv] = run;
                run += cn;
            }
        }
        __syncwarp();
        for (int base = 0; base < frn; base += 32) {
            const int q = base + lane;
            const bool valid = q < frn;
            const uint32_t lv = valid ? tlev[q] : 0xffu;
            const unsigned peers = __match_any_sync(kFull, lv);
            if (valid) dst[fn + S.cnt[lv] + __popc(peers & lt)] = tfr[q];
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) S.cnt[lv] += __popc(peers);
            __syncwarp();
        }
        if (lane == 0) {
            a.span_off[si] = off;
            a.span_meta[si] = make_int4(fn, frn, (int)nfl, (int)nfc);
        }
    }
}

// FP64 walk, operation for operation the plain per-particle definition: the MAC is
// l^2 < theta^2 d^2 with l^2 of the cell's level and d the distance to its FP64 centre of mass.
// kFast (NBODY_FP64_FAST): the same walk and acceptance tests, pair terms by pair64_fast.
template <int kThreads, bool kFast>
__global__ void __launch_bounds__(kThreads) walk64_kernel(WalkArgs a)
{
    const int lane = threadIdx.x & 31;
    const int gi = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    int g0, gcount, root_lo;
    if (!group_of(a, gi, g0, gcount, root_lo)) return;  // uniform per warp
    const int i = g0 + lane;
    const bool live = lane < gcount;
    // pre-order nodes of the group's system: [first, end)
    int first = 0, n_nodes = (int)*a.d_nn;
    const LevelTables *tab = a.tab;  // the group's system's cell sizes
    if (a.groups) {
        const int k = a.groups[gi].z;
        first = (int)a.node_off[a.start[k]];
        n_nodes = min(n_nodes, (int)a.node_off[a.start[k + 1]]);
        tab += k;
    }
    const double G = a.G;
    const double eps2 = __dmul_rn(a.eps, a.eps);
    const double th2 = __dmul_rn(a.theta, a.theta);
    D4 me;
    me.x = me.y = me.z = me.w = 0.0;
    if (live) me = a.sbody64[i];
    double ax = 0.0, ay = 0.0, az = 0.0;
    uint32_t pp = 0, pc = 0;
    int next = (!live || n_nodes - first < 2 || __ldg(&a.wn[first].count) != 0) ? n_nodes
                                                                                : first + 1;
    // the warp visits each node at most once (next only grows), so this budget ends the loop
    // only when a test lowers it
    int64_t steps_left = a.step_limit;
    for (;;) {
        const int j = __reduce_min_sync(kFull, next);
        if (j >= n_nodes) break;
        if (--steps_left < 0) {
            if (lane == 0) atomicOr(a.err, kErrStack);
            break;
        }
        if (next != j) continue;
        const int4 meta = __ldg(reinterpret_cast<const int4 *>(&a.wn[j].skip));
        const int skip = meta.x, first = meta.y, count = meta.z;
        if (count >= 1) {
            const int end = min(first + count, a.n);
            for (int b = first; b < end; ++b) {
                if (b == i) continue;
                const D4 s = a.sbody64[b];
                pair64_any<kFast>(s.x, s.y, s.z, s.w, me.x, me.y, me.z, G, eps2, ax, ay, az);
                ++pp;
            }
            next = skip;
        } else {
            const D4 s = a.com64[j];
            const double dx = __dsub_rn(s.x, me.x), dy = __dsub_rn(s.y, me.y),
                         dz = __dsub_rn(s.z, me.z);
            const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                        __dmul_rn(dz, dz));
            const double l2 = tab->l2[a.level[j]];
            if (l2 < __dmul_rn(th2, d2)) {
                if (a.q64)
                    cell64q(s.x, s.y, s.z, s.w, a.q64 + 6 * (size_t)j, me.x, me.y, me.z, G, eps2,
                            ax, ay, az);
                else
                    pair64_any<kFast>(s.x, s.y, s.z, s.w, me.x, me.y, me.z, G, eps2, ax, ay, az);
                ++pc;
                next = skip;
            } else {
                next = j + 1;
            }
        }
        next = max(next, j + 1);
    }
    if (live) write_out(a, i, ax, ay, az, pp, pc);
}

// ------------------------------------------------------------------------------------------
// Direct sum (Algorithm 1): every target against all n sources in ascending index order,
// skipping itself.  Sources are staged through shared memory a tile at a time.
// ------------------------------------------------------------------------------------------

constexpr int kDirectThreads = 256;   // FP64 direct sum
constexpr int kD32Threads = 128;      // FP32 direct sum: threads per block
constexpr int kD32Per = 2;            // targets per thread
constexpr int kD32Tile = 256;         // sources per shared-memory tile
constexpr int kD32MinChunk = 4096;    // sources per block at least

// FP32 sources (x - c, y - c, z - c, G m) of all bodies, converted once per call.
__global__ void direct32_prep_kernel(const double *__restrict__ pos, const double *__restrict__ mass,
                                     int n, double G, const Box *__restrict__ box,
                                     float4 *__restrict__ src)
{
    const double cx = box->c[0], cy = box->c[1], cz = box->c[2];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        src[j] = make_float4((float)(pos[j] - cx), (float)(pos[(size_t)n + j] - cy),
                             (float)(pos[2 * (size_t)n + j] - cz), (float)(G * mass[j]));
}

// One block: kD32Threads * kD32Per targets against one chunk of the sources (blockIdx.y), two
// sources at a time with packed FP32 arithmetic; each thread keeps kD32Per targets, so a source
// pair read from shared memory serves all of them.  A target meets itself in its own chunk at
// zero separation, which adds exactly zero.  Partial sums go to part[chunk][3][nt].
template <bool kGuard>
__global__ void __launch_bounds__(kD32Threads) direct32_chunk_kernel(
    const float4 *__restrict__ src, int n, const int64_t *__restrict__ targets, int nt,
    float eps2s, int chunk, float *__restrict__ part)
{
    __shared__ float4 tile[kD32Tile];   // pair-interleaved (see put_entry)
    const float2 eps2 = make_float2(eps2s, eps2s);
    float2 nme[kD32Per][3], ax[kD32Per], ay[kD32Per], az[kD32Per];
#pragma unroll
    for (int k = 0; k < kD32Per; ++k) {
        const int t = (blockIdx.x * kD32Per + k) * kD32Threads + threadIdx.x;
        const int i = t < nt ? (targets ? (int)targets[t] : t) : 0;
        const float4 me = src[i];
        nme[k][0] = make_float2(-me.x, -me.x);
        nme[k][1] = make_float2(-me.y, -me.y);
        nme[k][2] = make_float2(-me.z, -me.z);
        ax[k] = ay[k] = az[k] = make_float2(0.f, 0.f);
    }
    const int lo = blockIdx.y * chunk, hi = min(n, lo + chunk);
    for (int base = lo; base < hi; base += kD32Tile) {
        __syncthreads();
        for (int k = threadIdx.x; k < kD32Tile; k += kD32Threads) {
            const int j = base + k;
            put_entry(tile, k, j < hi ? src[j] : make_float4(0.f, 0.f, 0.f, 0.f));
        }
        __syncthreads();
        const int pairs = (min(kD32Tile, hi - base) + 1) >> 1;
#pragma unroll 2
        for (int q = 0; q < pairs; ++q) {
            const float4 u = tile[2 * q], v = tile[2 * q + 1];
#pragma unroll
            for (int k = 0; k < kD32Per; ++k)
                pair32x2<kGuard>(u, v, nme[k][0], nme[k][1], nme[k][2], eps2, ax[k], ay[k], az[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < kD32Per; ++k) {
        const int t = (blockIdx.x * kD32Per + k) * kD32Threads + threadIdx.x;
        if (t >= nt) continue;
        float *o = part + (size_t)blockIdx.y * 3 * nt;
        o[t] = ax[k].x + ax[k].y;
        o[(size_t)nt + t] = ay[k].x + ay[k].y;
        o[2 * (size_t)nt + t] = az[k].x + az[k].y;
    }
}

// acc = sum over the chunks, in chunk order, in FP64.
__global__ void direct32_reduce_kernel(const float *__restrict__ part, int chunks, int nt,
                                       double *__restrict__ acc)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 3 * nt; k += gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int c = 0; c < chunks; ++c) sum += (double)part[(size_t)c * 3 * nt + k];
        acc[k] = sum;
    }
}

struct alignas(16) Src64 {
    double x, y, z, m;
};

template <bool kFast>
__global__ void __launch_bounds__(kDirectThreads) direct64_kernel(
    const double *__restrict__ pos, const double *__restrict__ mass, int n,
    const int64_t *__restrict__ targets, int nt, double G, double eps2, double *__restrict__ acc)
{
    __shared__ Src64 tile[kDirectThreads];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = t < nt;
    const int i = live ? (targets ? (int)targets[t] : t) : -1;
    double xi = 0.0, yi = 0.0, zi = 0.0;
    if (live) {
        xi = pos[i];
        yi = pos[(size_t)n + i];
        zi = pos[2 * (size_t)n + i];
    }
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int base = 0; base < n; base += kDirectThreads) {
        const int j = base + threadIdx.x;
        __syncthreads();
        if (j < n) {
            Src64 s;
            s.x = pos[j];
            s.y = pos[(size_t)n + j];
            s.z = pos[2 * (size_t)n + j];
            s.m = mass[j];
            tile[threadIdx.x] = s;
        }
        __syncthreads();
        const int m = min(kDirectThreads, n - base);
        for (int k = 0; k < m; ++k) {
            if (base + k == i) continue;
            const Src64 s = tile[k];
            pair64_any<kFast>(s.x, s.y, s.z, s.m, xi, yi, zi, G, eps2, ax, ay, az);
        }
    }
    if (live) {
        acc[t] = ax;
        acc[(size_t)nt + t] = ay;
        acc[2 * (size_t)nt + t] = az;
    }
}

}  // namespace

namespace {

// Launch shapes: FP32 group walk with 2 / 4 / 8 warps per block, FP64 walk with 64 / 128 / 256
// threads per block.
// Blocks of the persistent group walk: as many as fit on the GPU at once (never more than the
// groups need).
template <int kWarps, bool kKahan, bool kGuard, bool kGroup, bool kQuad>
int persistent_blocks(int64_t groups)
{
    static int resident = 0;  // per kernel instance, per process
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, group_walk32_kernel<kWarps, kKahan, kGuard, kGroup, kQuad>, kWarps * 32,
            group_smem_bytes<kQuad>() * kWarps);
        resident = std::max(1, sms) * std::max(1, per_sm);
    }
    return (int)std::min<int64_t>((groups + kWarps - 1) / kWarps, resident);
}

template <int kWarps, bool kKahan, bool kGuard, bool kGroup, bool kQuad>
void launch_group_variant(const WalkArgs &a, int64_t groups, cudaStream_t s)
{
    const int blocks = persistent_blocks<kWarps, kKahan, kGuard, kGroup, kQuad>(groups);
    group_walk32_kernel<kWarps, kKahan, kGuard, kGroup, kQuad>
        <<<blocks, kWarps * 32, group_smem_bytes<kQuad>() * kWarps, s>>>(a);
}

template <int kWarps, bool kKahan, bool kGuard, int kBuf, int kStackN>
int pb_persistent_blocks(int64_t groups)
{
    static int resident = 0;  // per kernel instance, per process
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, pb_walk32_kernel<kWarps, kKahan, kGuard, kBuf, kStackN>, kWarps * 32,
            sizeof(PbSmem<kBuf, kStackN>) * kWarps);
        resident = std::max(1, sms) * std::max(1, per_sm);
    }
    return (int)std::min<int64_t>((groups + kWarps - 1) / kWarps, resident);
}

constexpr int kFarWarps = 4;       // warps per block of the far walk
constexpr int kFarBlocksPerSm = 8;

// The walk with the fast stack, then the overflow walk of the groups it handed on (a launch that
// finds an empty list and returns at once, unless a group was that deep).
template <int kWarps, bool kKahan, bool kGuard, int kBuf>
void launch_pb(const WalkArgs &a, int64_t groups, cudaStream_t s)
{
    const int blocks = pb_persistent_blocks<kWarps, kKahan, kGuard, kBuf, kPbFast>(groups);
    pb_walk32_kernel<kWarps, kKahan, kGuard, kBuf, kPbFast>
        <<<blocks, kWarps * 32, sizeof(PbSmem<kBuf, kPbFast>) * kWarps, s>>>(a);
    WalkArgs o = a;
    o.groups = a.overflow;
    o.n_groups = (int)std::min<int64_t>(groups, INT32_MAX);
    o.d_ngroups = a.n_overflow;
    o.overflow = nullptr;
    o.work = a.work + 1;
    const int ob = pb_persistent_blocks<4, kKahan, kGuard, 64, kPbStack>(groups);
    pb_walk32_kernel<4, kKahan, kGuard, 64, kPbStack>
        <<<ob, 4 * 32, sizeof(PbSmem<64, kPbStack>) * 4, s>>>(o);
    count_launches(1);
}

template <int kWarps, bool kKahan, bool kGuard>
void launch_group(const WalkArgs &a, int64_t groups, int buf, cudaStream_t s)
{
    const bool quad = a.gq != nullptr;
    if (!a.group_mac && !quad) {
        if (a.span_meta && !a.groups) {
            cudaMemsetAsync(a.span_next, 0, 2 * sizeof(unsigned), s);
            far_walk32_kernel<kFarWarps>
                <<<span_far_warps(a.n, a.span_bodies) / kFarWarps, kFarWarps * 32, 0, s>>>(a);
            count_launches(1);
        }
        if (buf == 128) launch_pb<kWarps, kKahan, kGuard, 128>(a, groups, s);
        else launch_pb<kWarps, kKahan, kGuard, 64>(a, groups, s);
        return;
    }
    if (a.group_mac) {
        if (quad) launch_group_variant<kWarps, kKahan, kGuard, true, true>(a, groups, s);
        else launch_group_variant<kWarps, kKahan, kGuard, true, false>(a, groups, s);
    } else {
        launch_group_variant<kWarps, kKahan, kGuard, false, true>(a, groups, s);
    }
}

template <int kWarps>
void launch_group(const WalkArgs &a, int64_t groups, bool kahan, bool guard, int buf,
                  cudaStream_t s)
{
    if (kahan) {
        if (guard) launch_group<kWarps, true, true>(a, groups, buf, s);
        else launch_group<kWarps, true, false>(a, groups, buf, s);
    } else {
        if (guard) launch_group<kWarps, false, true>(a, groups, buf, s);
        else launch_group<kWarps, false, false>(a, groups, buf, s);
    }
}

template <int kWarps, bool kKahan, bool kGuard>
cudaError_t allow_group_smem_kg()
{
    // the per-body test with monopole cells runs pb_walk32_kernel
    const void *fns[3] = {(const void *)group_walk32_kernel<kWarps, kKahan, kGuard, true, false>,
                          (const void *)group_walk32_kernel<kWarps, kKahan, kGuard, false, true>,
                          (const void *)group_walk32_kernel<kWarps, kKahan, kGuard, true, true>};
    const int bytes[3] = {(int)(group_smem_bytes<false>() * kWarps),
                          (int)(group_smem_bytes<true>() * kWarps),
                          (int)(group_smem_bytes<true>() * kWarps)};
    for (int k = 0; k < 3; ++k) {
        const cudaError_t e =
            cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes[k]);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaFuncSetAttribute(
        (const void *)pb_walk32_kernel<kWarps, kKahan, kGuard, 64, kPbFast>,
        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(PbSmem<64, kPbFast>) * kWarps));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(
            (const void *)pb_walk32_kernel<kWarps, kKahan, kGuard, 128, kPbFast>,
            cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)(sizeof(PbSmem<128, kPbFast>) * kWarps));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)pb_walk32_kernel<4, kKahan, kGuard, 64, kPbStack>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(PbSmem<64, kPbStack>) * 4));
    return e;
}

template <int kWarps>
cudaError_t allow_group_smem()
{
    cudaError_t e = allow_group_smem_kg<kWarps, true, true>();
    if (e == cudaSuccess) e = allow_group_smem_kg<kWarps, true, false>();
    if (e == cudaSuccess) e = allow_group_smem_kg<kWarps, false, true>();
    if (e == cudaSuccess) e = allow_group_smem_kg<kWarps, false, false>();
    return e;
}

template <int kThreads>
void launch_w64(const WalkArgs &a, int64_t groups, bool fast, cudaStream_t s)
{
    const int per_block = kThreads / 32;
    const int blocks = (int)((groups + per_block - 1) / per_block);
    if (fast) walk64_kernel<kThreads, true><<<blocks, kThreads, 0, s>>>(a);
    else walk64_kernel<kThreads, false><<<blocks, kThreads, 0, s>>>(a);
}

}  // namespace

int span_far_warps(int n, int span_bodies)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        sms = std::max(1, sms);
    }
    const int spans = (n + span_bodies - 1) / std::max(32, span_bodies);
    const int blocks = std::max(1, std::min((spans + kFarWarps - 1) / kFarWarps, sms * kFarBlocksPerSm));
    return blocks * kFarWarps;
}

cudaError_t walk_prepare()
{
    cudaError_t e = allow_group_smem<2>();
    if (e == cudaSuccess) e = allow_group_smem<4>();
    if (e == cudaSuccess) e = allow_group_smem<8>();
    return e;
}

WalkShape walk_shape32(int shape)
{
    // warps per block, span of the shared far walk (0: none), interaction buffer entries,
    // groups that follow the tree's cells
    static const WalkShape table[kWalkShapes] = {
        {2, 256, 128, false}, {4, 256, 128, false}, {8, 256, 128, false}, {4, 0, 128, false},
        {4, 128, 128, false}, {4, 512, 128, false}, {4, 256, 64, false},  {4, 0, 128, true}};
    if (shape < 0 || shape >= kWalkShapes) shape = kDefaultWalkShape;
    return table[shape];
}

int walk_shape_threads(int precision, int shape)
{
    static const int w64_threads[3] = {64, 128, 256};
    if (shape < 0 || shape >= kWalkShapes) shape = kDefaultWalkShape;
    return is_fp64(precision) ? w64_threads[shape < 3 ? shape : 1] : 32 * walk_shape32(shape).warps;
}

void launch_walk(int precision, const WalkArgs &a, int shape, cudaStream_t s)
{
    if (a.n <= 0) return;
    // FP32 walks: zero separations (a body and its own bucket, or eps^2 that rounds to zero in
    // FP32) are guarded
    const bool guard = !((float)(a.eps * a.eps) > 0.f);
    const int64_t groups = a.groups ? (int64_t)a.n_groups : ((int64_t)a.n + 31) / 32;
    if (groups <= 0) return;
    if (shape < 0 || shape >= kWalkShapes) shape = kDefaultWalkShape;
    if (is_fp64(precision)) {
        const bool fast = precision == NBODY_FP64_FAST;
        if (shape == 0) launch_w64<64>(a, groups, fast, s);
        else if (shape == 2) launch_w64<256>(a, groups, fast, s);
        else launch_w64<128>(a, groups, fast, s);
    } else {
        const bool kahan = precision == NBODY_FP32_KAHAN;
        const WalkShape sh = walk_shape32(shape);
        cudaMemsetAsync(a.work, 0, 2 * sizeof(unsigned), s);
        if (a.n_overflow) cudaMemsetAsync(a.n_overflow, 0, sizeof(unsigned), s);
        if (sh.warps == 2) launch_group<2>(a, groups, kahan, guard, sh.buf, s);
        else if (sh.warps == 8) launch_group<8>(a, groups, kahan, guard, sh.buf, s);
        else launch_group<4>(a, groups, kahan, guard, sh.buf, s);
    }
    count_launches(1);
}

int direct32_chunks(int n, int nt)
{
    // about 64 blocks per SM (16,384 targets x 1M sources: 49 TFLOP/s with 8 per SM, 52.7 with
    // 32, 53.1 with 64), chunks of at least kD32MinChunk sources
    const int tblocks = (nt + kD32Threads * kD32Per - 1) / (kD32Threads * kD32Per);
    int chunks = (152 * 64 + tblocks - 1) / std::max(1, tblocks);
    chunks = std::min(chunks, std::max(1, n / kD32MinChunk));
    return std::max(1, chunks);
}

void launch_direct(int precision, const double *pos, const double *mass, int n,
                   const int64_t *targets, int nt, double G, double eps, const Box *box,
                   double *acc, const DirectScratch &sc, cudaStream_t s)
{
    if (nt <= 0) return;
    if (is_fp64(precision)) {
        const int blocks = (nt + kDirectThreads - 1) / kDirectThreads;
        if (precision == NBODY_FP64_FAST)
            direct64_kernel<true><<<blocks, kDirectThreads, 0, s>>>(pos, mass, n, targets, nt, G,
                                                                    eps * eps, acc);
        else
            direct64_kernel<false><<<blocks, kDirectThreads, 0, s>>>(pos, mass, n, targets, nt, G,
                                                                     eps * eps, acc);
        count_launches(1);
        return;
    }
    const int chunks = direct32_chunks(n, nt);
    const int chunk = (n + chunks - 1) / chunks;
    direct32_prep_kernel<<<std::min((n + 255) / 256, 152 * 16), 256, 0, s>>>(pos, mass, n, G, box,
                                                                            sc.src);
    const dim3 grid((nt + kD32Threads * kD32Per - 1) / (kD32Threads * kD32Per), chunks);
    const float eps2 = (float)(eps * eps);
    if (eps > 0.0)
        direct32_chunk_kernel<false><<<grid, kD32Threads, 0, s>>>(sc.src, n, targets, nt, eps2,
                                                                  chunk, sc.part);
    else
        direct32_chunk_kernel<true><<<grid, kD32Threads, 0, s>>>(sc.src, n, targets, nt, eps2,
                                                                 chunk, sc.part);
    direct32_reduce_kernel<<<std::min((3 * nt + 255) / 256, 152 * 16), 256, 0, s>>>(
        sc.part, chunks, nt, acc);
    count_launches(3);
}

}  // namespace nb

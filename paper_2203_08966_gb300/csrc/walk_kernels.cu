// Force kernels: the Barnes-Hut walk (Algorithm 2, "Compute Cell Force") and the direct sum
// (Algorithm 1), both with the softened pair kernel of eq. `motion` (§2.1).
//
// Walk.  The nodes are stored in pre-order, each with `skip` = the index of the first node after
// its subtree.  A body's recursive walk over the children of every opened cell then becomes a
// monotone scan over node indices: at node j the body either opens j (next node j + 1, its first
// child) or is done with j's subtree (next node skip[j]: a leaf, or a cell accepted by l/d <
// theta).  One warp owns 32 Morton-consecutive bodies; every lane keeps its own `next`, and the
// warp visits the minimum `next` over its lanes, so each lane sees exactly its own sequence of
// nodes in its own order.  The per-body result (interaction list and summation order) is that of
// the per-particle recursive walk; only lanes whose `next` equals the visited node do work there.
#include <math.h>

#include "nbody_internal.cuh"

namespace nb {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWalkThreads = 128;

__device__ __forceinline__ float4 ldg4(const float4 *p) { return __ldg(p); }

// FP32 softened pair term: a += w (s - x) / (|s - x|^2 + eps^2)^(3/2), w = G m (eq. `motion`).
// kGuard: a zero separation with zero softening contributes nothing (as in the oracle).
template <bool kGuard>
__device__ __forceinline__ void pair32(const float4 &s, float xi, float yi, float zi, float eps2,
                                       float &tx, float &ty, float &tz)
{
    const float dx = s.x - xi, dy = s.y - yi, dz = s.z - zi;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    float rinv = rsqrtf(r2);
    if (kGuard) rinv = r2 > 0.f ? rinv : 0.f;
    const float f = s.w * (rinv * rinv) * rinv;
    tx = f * dx;
    ty = f * dy;
    tz = f * dz;
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

// FP32 accumulator.  Plain: one running sum per component.  Compensated: the terms go into a
// plain FP32 partial sum, which is folded into a Kahan-compensated total (Kahan 1965) every
// kFold walk iterations and at the end, so the compensation costs a few operations per block of
// terms instead of four per term; the error of the total is that of partials of at most kFold
// terms plus a compensated sum over the partials.
template <bool kKahan>
struct Acc3 {
    static constexpr int kFold = 64;
    float x = 0.f, y = 0.f, z = 0.f;     // plain sum, or the current partial
    float sx = 0.f, sy = 0.f, sz = 0.f;  // compensated total
    float cx = 0.f, cy = 0.f, cz = 0.f;  // its compensation
    __device__ __forceinline__ void add(float tx, float ty, float tz)
    {
        x += tx;
        y += ty;
        z += tz;
    }
    __device__ __forceinline__ static void kahan(float &s, float &c, float t)
    {
        const float yv = t - c;
        const float u = s + yv;
        c = (u - s) - yv;
        s = u;
    }
    __device__ __forceinline__ void fold()
    {
        if (kKahan) {
            kahan(sx, cx, x);
            kahan(sy, cy, y);
            kahan(sz, cz, z);
            x = y = z = 0.f;
        }
    }
    __device__ __forceinline__ float3 result()
    {
        if (kKahan) {
            fold();
            return make_float3(sx, sy, sz);
        }
        return make_float3(x, y, z);
    }
};

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

// FP32 walk.  MAC: accept a cell when d^2 > l^2 / theta^2 (the node's `crit`), i.e. l/d < theta.
template <bool kKahan, bool kGuard>
__global__ void __launch_bounds__(kWalkThreads) walk32_kernel(WalkArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int i = warp * 32 + lane;
    if (warp * 32 >= a.n) return;  // whole warp out of range (uniform per warp)
    const bool live = i < a.n;
    const int n_nodes = a.n_nodes;
    const float eps2 = (float)(a.eps * a.eps);
    const float4 me = live ? ldg4(a.sbody32 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    Acc3<kKahan> acc;
    uint32_t pp = 0, pc = 0;
    // the root is never tested: a body starts at the root's first child (none when the root is a
    // leaf, i.e. a single body)
    int next = (!live || n_nodes < 2 || __ldg(&a.wn[0].count) != 0) ? n_nodes : 1;
    unsigned it = 0;
    for (;;) {
        const int j = __reduce_min_sync(kFull, next);
        if (j >= n_nodes) break;
        if (kKahan && (++it % Acc3<kKahan>::kFold) == 0) acc.fold();
        if (next != j) continue;
        const float4 c = ldg4(&a.wn[j].c);
        const int4 meta = __ldg(reinterpret_cast<const int4 *>(&a.wn[j].skip));
        const int skip = meta.x, first = meta.y, count = meta.z;
        const float crit = __int_as_float(meta.w);
        float tx, ty, tz;
        if (count == 1) {
            if (first != i) {
                pair32<kGuard>(c, me.x, me.y, me.z, eps2, tx, ty, tz);
                acc.add(tx, ty, tz);
                ++pp;
            }
            next = skip;
        } else if (count > 1) {
            const int end = min(first + count, a.n);
            for (int b = first; b < end; ++b) {
                if (b == i) continue;
                pair32<kGuard>(ldg4(a.sbody32 + b), me.x, me.y, me.z, eps2, tx, ty, tz);
                acc.add(tx, ty, tz);
                ++pp;
            }
            next = skip;
        } else {
            const float dx = c.x - me.x, dy = c.y - me.y, dz = c.z - me.z;
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (d2 > crit) {
                pair32<kGuard>(c, me.x, me.y, me.z, eps2, tx, ty, tz);
                acc.add(tx, ty, tz);
                ++pc;
                next = skip;
            } else {
                next = j + 1;
            }
        }
        next = max(next, j + 1);  // progress even on a malformed skip
    }
    const float3 r = acc.result();
    if (live) write_out(a, i, (double)r.x, (double)r.y, (double)r.z, pp, pc);
}

// FP64 walk, operation for operation the plain per-particle definition: the MAC is
// l^2 < theta^2 d^2 with l^2 of the cell's level and d the distance to its FP64 centre of mass.
__global__ void __launch_bounds__(kWalkThreads) walk64_kernel(WalkArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int i = warp * 32 + lane;
    if (warp * 32 >= a.n) return;
    const bool live = i < a.n;
    const int n_nodes = a.n_nodes;
    const double G = a.G;
    const double eps2 = __dmul_rn(a.eps, a.eps);
    const double th2 = __dmul_rn(a.theta, a.theta);
    D4 me;
    me.x = me.y = me.z = me.w = 0.0;
    if (live) me = a.sbody64[i];
    double ax = 0.0, ay = 0.0, az = 0.0;
    uint32_t pp = 0, pc = 0;
    int next = (!live || n_nodes < 2 || __ldg(&a.wn[0].count) != 0) ? n_nodes : 1;
    for (;;) {
        const int j = __reduce_min_sync(kFull, next);
        if (j >= n_nodes) break;
        if (next != j) continue;
        const int4 meta = __ldg(reinterpret_cast<const int4 *>(&a.wn[j].skip));
        const int skip = meta.x, first = meta.y, count = meta.z;
        if (count >= 1) {
            const int end = min(first + count, a.n);
            for (int b = first; b < end; ++b) {
                if (b == i) continue;
                const D4 s = a.sbody64[b];
                pair64(s.x, s.y, s.z, s.w, me.x, me.y, me.z, G, eps2, ax, ay, az);
                ++pp;
            }
            next = skip;
        } else {
            const D4 s = a.com64[j];
            const double dx = __dsub_rn(s.x, me.x), dy = __dsub_rn(s.y, me.y),
                         dz = __dsub_rn(s.z, me.z);
            const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                        __dmul_rn(dz, dz));
            const double l2 = a.tab->l2[a.level[j]];
            if (l2 < __dmul_rn(th2, d2)) {
                pair64(s.x, s.y, s.z, s.w, me.x, me.y, me.z, G, eps2, ax, ay, az);
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

constexpr int kDirectThreads = 256;

template <bool kGuard>
__global__ void __launch_bounds__(kDirectThreads) direct32_kernel(
    const double *__restrict__ pos, const double *__restrict__ mass, int n,
    const int64_t *__restrict__ targets, int nt, double G, float eps2, const Box *__restrict__ box,
    double *__restrict__ acc)
{
    __shared__ float4 tile[kDirectThreads];
    const double cx = box->c[0], cy = box->c[1], cz = box->c[2];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = t < nt;
    const int i = live ? (targets ? (int)targets[t] : t) : -1;
    float xi = 0.f, yi = 0.f, zi = 0.f;
    if (live) {
        xi = (float)(pos[i] - cx);
        yi = (float)(pos[(size_t)n + i] - cy);
        zi = (float)(pos[2 * (size_t)n + i] - cz);
    }
    float ax = 0.f, ay = 0.f, az = 0.f;
    for (int base = 0; base < n; base += kDirectThreads) {
        const int j = base + threadIdx.x;
        __syncthreads();
        if (j < n) {
            tile[threadIdx.x] = make_float4((float)(pos[j] - cx), (float)(pos[(size_t)n + j] - cy),
                                            (float)(pos[2 * (size_t)n + j] - cz),
                                            (float)(G * mass[j]));
        } else {
            tile[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const int m = min(kDirectThreads, n - base);
        const int self = i - base;  // in [0, m) when the target itself is in this tile
        if (self >= 0 && self < m) {
            for (int k = 0; k < m; ++k) {
                if (k == self) continue;
                float tx, ty, tz;
                pair32<kGuard>(tile[k], xi, yi, zi, eps2, tx, ty, tz);
                ax += tx; ay += ty; az += tz;
            }
        } else {
#pragma unroll 8
            for (int k = 0; k < m; ++k) {
                float tx, ty, tz;
                pair32<kGuard>(tile[k], xi, yi, zi, eps2, tx, ty, tz);
                ax += tx; ay += ty; az += tz;
            }
        }
    }
    if (live) {
        acc[t] = ax;
        acc[(size_t)nt + t] = ay;
        acc[2 * (size_t)nt + t] = az;
    }
}

struct alignas(16) Src64 {
    double x, y, z, m;
};

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
            pair64(s.x, s.y, s.z, s.m, xi, yi, zi, G, eps2, ax, ay, az);
        }
    }
    if (live) {
        acc[t] = ax;
        acc[(size_t)nt + t] = ay;
        acc[2 * (size_t)nt + t] = az;
    }
}

}  // namespace

void launch_walk(int precision, const WalkArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return;
    const int64_t threads = ((int64_t)a.n + 31) / 32 * 32;
    const int blocks = (int)((threads + kWalkThreads - 1) / kWalkThreads);
    const bool guard = !(a.eps > 0.0);
    if (precision == NBODY_FP64) {
        walk64_kernel<<<blocks, kWalkThreads, 0, s>>>(a);
    } else if (precision == NBODY_FP32_KAHAN) {
        if (guard) walk32_kernel<true, true><<<blocks, kWalkThreads, 0, s>>>(a);
        else walk32_kernel<true, false><<<blocks, kWalkThreads, 0, s>>>(a);
    } else {
        if (guard) walk32_kernel<false, true><<<blocks, kWalkThreads, 0, s>>>(a);
        else walk32_kernel<false, false><<<blocks, kWalkThreads, 0, s>>>(a);
    }
    count_launches(1);
}

void launch_direct(int precision, const double *pos, const double *mass, int n,
                   const int64_t *targets, int nt, double G, double eps, const Box *box,
                   double *acc, cudaStream_t s)
{
    if (nt <= 0) return;
    const int blocks = (nt + kDirectThreads - 1) / kDirectThreads;
    if (precision == NBODY_FP64) {
        direct64_kernel<<<blocks, kDirectThreads, 0, s>>>(pos, mass, n, targets, nt, G, eps * eps,
                                                          acc);
    } else {
        const float eps2 = (float)(eps * eps);
        if (eps > 0.0)
            direct32_kernel<false><<<blocks, kDirectThreads, 0, s>>>(pos, mass, n, targets, nt, G,
                                                                     eps2, box, acc);
        else
            direct32_kernel<true><<<blocks, kDirectThreads, 0, s>>>(pos, mass, n, targets, nt, G,
                                                                    eps2, box, acc);
    }
    count_launches(1);
}

}  // namespace nb

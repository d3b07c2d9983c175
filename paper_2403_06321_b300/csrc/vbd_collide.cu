// vbd_collide.cu -- vertex-triangle self-collision detection (Sec. 3.5) for
// sm_103a, run once at the start of each step on x^t.
//
// A boundary vertex a has penetrated when it lies in (or on) a tet it is not
// a vertex of.  It is then paired with the nearest boundary triangle within
// the detection distance r that shares no tet with it; triangles within
// 1e-5 r of the nearest distance count as tied and the lowest index wins.
//
// Broad phase: spatial hashes of triangle and tet centroids, with cells of
// c_tri = 1.05 (R_tri + r) and c_tet = 1.05 R_tet, R the largest
// centroid-to-corner distance of any triangle (tet) at this step.  A triangle
// within r of a vertex, or a tet holding it, has its centroid within R + r
// (R) of the vertex (the element lies in the ball of radius R about its
// centroid), hence in one of the 27 cells around the vertex's cell of that
// table; candidates whose ball is out of reach are skipped before the exact
// tests.  Each element is
// stored once (count, prefix sum, fill), so the tables never overflow.
//
// CCD (Sec. 3.5), before every n_col-th iteration: each boundary vertex
// without a step-start pair is swept along its straight path from x^t to
// the current iterate against the boundary triangles (their corners moving
// the same way) that share no tet with it.  Broad phase: bounding spheres of
// each triangle's six corner positions (both ends of its motion) hashed with
// cells of 1.05 (R_tri + R_v), R_v the largest half path of a vertex; a
// triangle that meets the vertex's path has its sphere centre within
// R_tri + R_v of the path's midpoint.  Narrow phase: the earliest root of the
// coplanarity cubic at which the vertex lies in the closed triangle; impacts
// within 1e-5 in time are tied and the lowest triangle index wins.  The pair
// keeps the impact point's barycentric weights (contact_w).
//
// The sweep needs, for each free vertex, the pairs in which it is a triangle
// corner: that reverse list is built the same way and then sorted per vertex
// so that forces are always summed in the same order.
//
// No kernel here waits on another thread; every loop is bounded by array
// sizes.
#include "vbd_kernels.h"

#include <algorithm>

#include "vbd_geom.cuh"

namespace vbd {

namespace {

using geom::cross;
using geom::dot;
using geom::f3;
using geom::operator-;
using geom::operator+;
using geom::operator*;
using geom::fminf3;
using geom::fmaxf3;

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// ---- broad phase ------------------------------------------------------------
// FP32 throughout.  Cell coordinates floor(x / c) of a point and of an
// element's centroid are exact enough while |x| / c < 2^16: the rounding of
// x = X + u, of the centroid and of the product stays below 0.02 cells,
// which the 5% margin of c covers, and below the 3% of c by which bounding
// spheres are inflated.  Positions beyond that range are counted in
// counters[4] (the host reports VBD_ERR_RANGE) and hashed after clamping.
constexpr float kRange = 65536.0f;
constexpr float kMargin = 1.05f;
constexpr float kSlack = 0.03f;

__device__ __forceinline__ float3 position(const Dev &d, int i) {
    const float4 X = __ldg(d.rest + i), u = __ldg(d.u + i);
    return make_float3(X.x + u.x, X.y + u.y, X.z + u.z);
}

// cell of the triangle table: a triangle within r of a vertex has its
// centroid within R_tri + r of it
__device__ __forceinline__ float tri_cell_width(const Dev &d, float r) {
    return kMargin * (__uint_as_float(d.cell_size[0]) + r) + 1e-30f;
}

// cell of the tet table: a tet holding a point has its centroid within R_tet
__device__ __forceinline__ float tet_cell_width(const Dev &d) {
    return kMargin * __uint_as_float(d.cell_size[1]) + 1e-30f;
}

// cell of the swept-triangle table (CCD): a triangle whose motion meets a
// vertex's path has its sphere centre within R_tri + R_v of the path's midpoint
__device__ __forceinline__ float swept_cell_width(const Dev &d) {
    return kMargin * (__uint_as_float(d.cell_size[0]) + __uint_as_float(d.cell_size[2])) + 1e-30f;
}

// cell of the edge table (edge-edge CCD): two edges whose motions meet have
// sphere centres within 2 R_edge of each other
__device__ __forceinline__ float edge_cell_width(const Dev &d) {
    return kMargin * 2.0f * __uint_as_float(d.cell_size[3]) + 1e-30f;
}

template <int K>
__device__ __forceinline__ float table_cell_width(const Dev &d, float r) {
    return K == 3 ? tri_cell_width(d, r)
                  : (K == 4 ? tet_cell_width(d) : (K == 5 ? swept_cell_width(d) : edge_cell_width(d)));
}

__device__ __forceinline__ int3 cell_of(const Dev &d, float3 p, float inv_c) {
    float q[3] = {floorf(p.x * inv_c), floorf(p.y * inv_c), floorf(p.z * inv_c)};
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        ok &= fabsf(q[k]) < kRange;  // false for NaN too
        q[k] = fminf(fmaxf(q[k], -kRange), kRange);
        if (q[k] != q[k]) q[k] = 0.0f;
    }
    if (!ok) atomicAdd(d.counters + 4, 1ull);
    return make_int3((int)q[0], (int)q[1], (int)q[2]);
}

__device__ __forceinline__ int bucket_of(int i, int j, int k, int nb) {
    unsigned h = (unsigned)i * 73856093u ^ (unsigned)j * 19349663u ^ (unsigned)k * 83492791u;
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    return (int)(h & (unsigned)(nb - 1));
}

// Bounding sphere of each element (K = 3 triangle, 4 tet): centroid and the
// largest centroid-to-corner distance; the largest radius goes to *rmax (as
// float bits: non-negative floats order like their unsigned bits).
template <int K>
__global__ void k_bounds(Dev d, const int4 *items, int n, float4 *sphere, unsigned *rmax) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int4 v = items[t];
    const int c[4] = {v.x, v.y, v.z, v.w};
    float3 p[K];
    float3 m = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        p[k] = position(d, c[k]);
        m = m + p[k];
    }
    m = (1.0f / K) * m;
    float R2 = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float3 e = p[k] - m;
        R2 = fmaxf(R2, dot(e, e));
    }
    float R = sqrtf(R2);
    if (!(R >= 0.f)) R = 0.f;  // a NaN position never widens the cells
    sphere[t] = make_float4(m.x, m.y, m.z, R);
    atomicMax(rmax, __float_as_uint(R));
}

// Bounding sphere of each triangle's corners at both ends of their motion
// (x^t = X + ut and the current X + u), for the CCD.
__global__ void k_bounds_swept(Dev d, int n, float4 *sphere, unsigned *rmax) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int4 v = d.tri[t];
    const int c[3] = {v.x, v.y, v.z};
    float3 p[6];
    float3 m = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float3 X = f3(__ldg(d.rest + c[k]));
        p[k] = X + f3(__ldg(d.ut + c[k]));
        p[k + 3] = X + f3(__ldg(d.u + c[k]));
        m = m + p[k] + p[k + 3];
    }
    m = (1.0f / 6.0f) * m;
    float R2 = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float3 e = p[k] - m;
        R2 = fmaxf(R2, dot(e, e));
    }
    float R = sqrtf(R2);
    if (!(R >= 0.f)) R = 0.f;
    sphere[t] = make_float4(m.x, m.y, m.z, R);
    atomicMax(rmax, __float_as_uint(R));
}

// the largest half path |u - ut| / 2 of a boundary vertex
__global__ void k_path_radius(Dev d, int n_surf, unsigned *rmax) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_surf) return;
    const int a = d.surf[k];
    const float3 e = f3(__ldg(d.u + a)) - f3(__ldg(d.ut + a));
    float R = 0.5f * sqrtf(dot(e, e));
    if (!(R >= 0.f)) R = 0.f;
    atomicMax(rmax, __float_as_uint(R));
}

__device__ __forceinline__ int sphere_bucket(const Dev &d, float4 s, float inv_c, int nb) {
    const int3 q = cell_of(d, make_float3(s.x, s.y, s.z), inv_c);
    return bucket_of(q.x, q.y, q.z, nb);
}

template <int K>
__global__ void k_count(Dev d, const float4 *sphere, int n, int nb, float r, int *count) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    atomicAdd(count + sphere_bucket(d, sphere[t], 1.0f / table_cell_width<K>(d, r), nb), 1);
}

// entries[] of bucket b: the ids whose sphere centre hashes to b; with
// `sorted`, each entry's sphere beside it (the query streams those)
template <int K>
__global__ void k_fill(Dev d, const float4 *sphere, int n, int nb, float r, const int *start, int *fill,
                       int *entries, float4 *sorted = nullptr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float4 sp = sphere[t];
    const int b = sphere_bucket(d, sp, 1.0f / table_cell_width<K>(d, r), nb);
    const int k = start[b] + atomicAdd(fill + b, 1);
    entries[k] = t;
    if (sorted) sorted[k] = sp;
}

// ---- narrow phase -------------------------------------------------------------
// Whether the origin lies in the closed tet with corners p0..p3 (positions
// relative to the vertex): its barycentric coordinates d_k / D, from the edge
// matrix [p1 - p0, p2 - p0, p3 - p0] by Cramer's rule, are all >= 0 and sum
// to at most 1 (compared without dividing).
__device__ __forceinline__ bool origin_in_tet(float3 p0, float3 p1, float3 p2, float3 p3) {
    const float3 e1 = p1 - p0, e2 = p2 - p0, e3 = p3 - p0;
    const float3 r = make_float3(-p0.x, -p0.y, -p0.z);
    float D = dot(e1, cross(e2, e3));
    if (D == 0.0f) return false;
    float d1 = dot(r, cross(e2, e3)), d2 = dot(e1, cross(r, e3)), d3 = dot(e1, cross(e2, r));
    if (D < 0.0f) {
        D = -D; d1 = -d1; d2 = -d2; d3 = -d3;
    }
    return d1 >= 0.0f && d2 >= 0.0f && d3 >= 0.0f && d1 + d2 + d3 <= D;
}

// bucket of the n-th of the 27 cells around c (n = 0..26)
__device__ __forceinline__ int neighbour_bucket(int3 c, int n, int nb) {
    return bucket_of(c.x + n % 3 - 1, c.y + (n / 3) % 3 - 1, c.z + n / 9 - 1, nb);
}

__device__ __forceinline__ float3 rel(const Dev &d, int k, float3 Xa, float3 ua) {
    return (f3(__ldg(d.rest + k)) - Xa) + (f3(__ldg(d.u + k)) - ua);
}

__device__ __forceinline__ bool sphere_far(float4 s, float3 x, float reach) {
    const float3 e = make_float3(s.x - x.x, s.y - x.y, s.z - x.z);
    const float lim = s.w + reach;
    return dot(e, e) > lim * lim;
}

// Nearest admissible triangle of vertex a (boundary index k) among the
// The hits of one lane within `tol` of its best value so far (the tie
// window): up to two, else `full` and the query scans again.
struct TieWindow {
    float ta, tb;
    int fa, fb, n;
    bool full;
    __device__ void add(float t, int f, float best, float tol) {
        if (!(t <= best + tol)) return;
        if (n == 0) {
            ta = t;
            fa = f;
            n = 1;
        } else if (n == 1) {
            tb = t;
            fb = f;
            n = 2;
        } else {
            full = true;
        }
    }
    // the best value has moved down to `best`: drop what left the window
    __device__ void shrink(float best, float tol) {
        const float w = best + tol;
        if (n == 2 && !(tb <= w)) n = 1;
        if (n >= 1 && !(ta <= w)) {
            ta = tb;
            fa = fb;
            n -= 1;
        }
    }
    // lowest index among the hits by `lim`, -1 if none
    __device__ int lowest(float lim) const {
        int f = -1;
        if (n >= 1 && ta <= lim) f = fa;
        if (n >= 2 && tb <= lim && (f < 0 || fb < f)) f = fb;
        return f;
    }
};

// triangles of this lane's neighbour cells (n = lane, lane + Q, ... < 27):
// pass 0 returns the nearest distance within r (or -1) and keeps the hits
// of its tie window (1e-5 r) in `win`; pass 1 (only when a window was full)
// the lowest triangle index within `lim` (or -1).  Triangles whose bounding
// sphere is farther than r (plus the rounding slack) are skipped before the
// exact test.
template <int Q>
__device__ __forceinline__ float nearest_tri(const Dev &d, int k, float3 xa, float3 Xa, float3 ua, int3 cell,
                                            int nb, int lane, float r, float slack, int pass, float lim,
                                            int &pair, TieWindow &win) {
    const int g0 = d.ring_off[k], g1 = d.ring_off[k + 1];
    float best = -1.f;
    for (int n = lane; n < 27; n += Q) {
        const int b = neighbour_bucket(cell, n, nb);
        const int e1 = d.cell_start[b + 1];
        for (int e = d.cell_start[b]; e < e1; ++e) {
            if (sphere_far(d.cell_tri_sph[e], xa, r + slack)) continue;
            const int t = d.cell_tri[e];
            if (pass == 1 && pair >= 0 && t >= pair) continue;
            const int4 v = d.tri[t];
            bool adjacent = false;
            for (int g = g0; g < g1 && !adjacent; ++g) {
                const int w = d.ring[g];
                adjacent = (w == v.x) | (w == v.y) | (w == v.z);
            }
            if (adjacent) continue;
            const float3 pa = rel(d, v.x, Xa, ua), pb = rel(d, v.y, Xa, ua), pc = rel(d, v.z, Xa, ua);
            const float3 w = geom::nearest_weights(pa, pb, pc);
            const float3 qp = make_float3(w.x * pa.x + w.y * pb.x + w.z * pc.x, w.x * pa.y + w.y * pb.y + w.z * pc.y,
                                          w.x * pa.z + w.y * pb.z + w.z * pc.z);
            const float dist = sqrtf(dot(qp, qp));
            if (dist > r) continue;
            if (pass == 0) {
                if (best < 0.f || dist < best) {
                    best = dist;
                    win.shrink(best, 1e-5f * r);
                }
                win.add(dist, t, best, 1e-5f * r);
            }
            if (pass == 1 && dist <= lim) pair = t;
        }
    }
    return best;
}

// Q lanes per boundary vertex (or edge), each taking every Q-th of the 27
// neighbour cells; their results are combined with shuffles (a minimum
// distance, an "any" and a minimum index), so the outcome does not depend
// on the split.  Measured on the 900k-vertex slab scene (ms per step, Q = 8 /
// 4 / 2 / 1): proximity query 6.07 / 5.99 / 5.96 / 5.99, vertex-triangle
// CCD 8.15 / 7.84 / 7.72 / 7.77, edge-edge CCD 22.4 / 19.9 / 18.6 / 18.4.
// The pair exists when a triangle lies within r and the vertex has
// penetrated; the triangle search runs first, so that the tet test runs
// only for the (few) vertices near another surface.
constexpr int kProximityLanes = 2;
constexpr int kCcdLanes = 2;
constexpr int kEdgeLanes = 1;

template <int Q>
__device__ __forceinline__ float group_min_dist(float v) {  // -1 = none
#pragma unroll
    for (int off = Q / 2; off > 0; off >>= 1) {
        const float o = __shfl_xor_sync(0xffffffffu, v, off);
        if (o >= 0.f && (v < 0.f || o < v)) v = o;
    }
    return v;
}

template <int Q>
__device__ __forceinline__ int group_min_index(int v) {  // -1 = none
#pragma unroll
    for (int off = Q / 2; off > 0; off >>= 1) {
        const int o = __shfl_xor_sync(0xffffffffu, v, off);
        if (o >= 0 && (v < 0 || o < v)) v = o;
    }
    return v;
}

__global__ void __launch_bounds__(128) k_query(Dev d, int n_surf, int nb_tri, int nb_tet, float r) {
    constexpr int Q = kProximityLanes;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = (int)(g / Q), lane = (int)(g % Q);
    const bool active = k < n_surf;  // inactive lanes still join the shuffles
    const int a = active ? d.surf[k] : 0;
    const float c = tri_cell_width(d, r);
    const float slack = kSlack * c;
    const float3 Xa = f3(__ldg(d.rest + a)), ua = f3(__ldg(d.u + a));
    const float3 xa = Xa + ua;
    const int3 cell = active ? cell_of(d, xa, 1.0f / c) : make_int3(0, 0, 0);
    int pair = -1;
    TieWindow win = {0.f, 0.f, -1, -1, 0, false};
    float best = active ? nearest_tri<Q>(d, k, xa, Xa, ua, cell, nb_tri, lane, r, slack, 0, 0.f, pair, win) : -1.f;
    best = group_min_dist<Q>(best);
    bool inside = false;
    if (best >= 0.f) {  // uniform over the group
        // penetration: inside a tet that does not hold the vertex
        const float ct = tet_cell_width(d);
        const float tslack = kSlack * ct;
        const int3 tcell = cell_of(d, xa, 1.0f / ct);
        for (int n = lane; n < 27 && !inside; n += Q) {
            const int b = neighbour_bucket(tcell, n, nb_tet);
            const int e1 = d.tet_start[b + 1];
            for (int e = d.tet_start[b]; e < e1 && !inside; ++e) {
                if (sphere_far(d.cell_tet_sph[e], xa, tslack)) continue;
                const int4 v = d.tet_v[d.cell_tet[e]];
                if (v.x == a || v.y == a || v.z == a || v.w == a) continue;
                inside = origin_in_tet(rel(d, v.x, Xa, ua), rel(d, v.y, Xa, ua), rel(d, v.z, Xa, ua),
                                       rel(d, v.w, Xa, ua));
            }
        }
    }
    const unsigned group_mask = ((1u << Q) - 1u) << (threadIdx.x & 31 & ~(Q - 1));
    inside = (__ballot_sync(0xffffffffu, inside) & group_mask) != 0;
    const bool rescan = group_min_index<Q>(win.full ? 0 : -1) == 0;  // on every lane of the warp
    if (inside) {
        if (rescan)
            nearest_tri<Q>(d, k, xa, Xa, ua, cell, nb_tri, lane, r, slack, 1, best + 1e-5f * r, pair, win);
        else
            pair = win.lowest(best + 1e-5f * r);
    }
    pair = group_min_index<Q>(pair);
    if (active && lane == 0) {
        d.contact[a] = pair;
        if (d.contact_w) d.contact_w[a] = make_float4(0.f, 0.f, 0.f, 0.f);  // a DCD pair (or none)
        if (pair >= 0) atomicAdd(d.counters + 3, 1ull);
    }
}

// ---- CCD narrow phase ------------------------------------------------------------
// Earliest root in [t0, 1] of c0 + c1 t + c2 t^2 + c3 t^3: the interval is cut
// at the roots of the derivative into monotone pieces; the first piece that
// starts at a zero or changes sign is narrowed by false position (Illinois
// variant; plain halving after 16 steps) to a bracket of 1e-7.  -1 if none;
// a cubic that vanishes identically (coplanar motion) has no root.
__device__ __forceinline__ float cubic_first_root(float c0, float c1, float c2, float c3, float t0) {
    if (!(fabsf(c0) + fabsf(c1) + fabsf(c2) + fabsf(c3) > 0.f)) return -1.f;
    float cut[4];
    int nc = 0;
    cut[nc++] = t0;
    const float qa = 3.f * c3, qb = 2.f * c2, qc = c1;
    float r0 = 2.f, r1 = 2.f;
    if (qa != 0.f) {
        const float disc = qb * qb - 4.f * qa * qc;
        if (disc >= 0.f) {
            const float sq = sqrtf(disc);
            r0 = (-qb - sq) / (2.f * qa);
            r1 = (-qb + sq) / (2.f * qa);
            if (r0 > r1) { const float t = r0; r0 = r1; r1 = t; }
        }
    } else if (qb != 0.f) {
        r0 = -qc / qb;
    }
    if (r0 > t0 && r0 < 1.f) cut[nc++] = r0;
    if (r1 > t0 && r1 < 1.f) cut[nc++] = r1;
    cut[nc++] = 1.f;
    for (int k = 0; k + 1 < nc; ++k) {
        float lo = cut[k], hi = cut[k + 1];
        float flo = ((c3 * lo + c2) * lo + c1) * lo + c0;
        const float fhi = ((c3 * hi + c2) * hi + c1) * hi + c0;
        float fh = fhi;
        if (flo == 0.f) return lo;
        if ((flo < 0.f) == (fh < 0.f) && fh != 0.f) continue;
        if (fh == 0.f) return hi;
        // Illinois false position: the secant point of the bracket, and the
        // value kept at an end that stays twice in a row halved, so that both
        // ends close in; the midpoint where rounding puts the secant point
        // outside the open bracket, and from step 16 on.  The sign at lo is
        // that of the first flo throughout (halving only scales the kept values)
        const bool neg_lo = flo < 0.f;
        int side = 0;
        for (int it = 0; it < 64 && hi - lo > 1e-7f; ++it) {
            float m = it < 16 ? (lo * fh - hi * flo) / (fh - flo) : 0.5f * (lo + hi);
            if (!(m > lo && m < hi)) m = 0.5f * (lo + hi);
            const float fm = ((c3 * m + c2) * m + c1) * m + c0;
            if (fm == 0.f) return m;
            if ((fm < 0.f) == neg_lo) {
                lo = m;
                flo = fm;
                if (side == -1) fh *= 0.5f;
                side = -1;
            } else {
                hi = m;
                fh = fm;
                if (side == 1) flo *= 0.5f;
                side = 1;
            }
        }
        return hi;
    }
    return -1.f;
}

// Time of impact of a vertex with a triangle whose corners, relative to the
// vertex, move as A_k + t B_k (t in [0, 1]); -1 if none.  The coplanarity
// cubic r_1 . (r_2 x r_3) comes from the trilinear expansion; its roots are
// taken in order and the first with the vertex in the closed triangle (all
// barycentric weights >= 0) is the impact, its weights in w.
__device__ __forceinline__ float vt_impact(float3 A0, float3 A1, float3 A2, float3 B0, float3 B1, float3 B2,
                                           float3 &w) {
    const float3 a12 = cross(A1, A2);
    const float c0 = dot(A0, a12);
    const float c1 = dot(B0, a12) + dot(A0, cross(B1, A2)) + dot(A0, cross(A1, B2));
    const float3 b12 = cross(B1, B2);
    const float c2 = dot(B0, cross(B1, A2)) + dot(B0, cross(A1, B2)) + dot(A0, b12);
    const float c3 = dot(B0, b12);
    float t0 = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
        const float t = cubic_first_root(c0, c1, c2, c3, t0);
        if (t < 0.f) return -1.f;
        const float3 r1 = A0 + t * B0, r2 = A1 + t * B1, r3 = A2 + t * B2;
        const float3 n = cross(r2 - r1, r3 - r1);
        const float nn = dot(n, n);
        if (nn > 0.f) {
            w = make_float3(dot(cross(r2, r3), n) / nn, dot(cross(r3, r1), n) / nn, dot(cross(r1, r2), n) / nn);
            if (w.x >= 0.f && w.y >= 0.f && w.z >= 0.f) return t;
        }
        t0 = t + 1e-6f;
        if (t0 >= 1.f) return -1.f;
    }
    return -1.f;
}

// whether the axis-aligned box of six points leaves out the origin
__device__ __forceinline__ bool box_misses_origin(float3 p0, float3 p1, float3 p2, float3 p3, float3 p4, float3 p5) {
    const float lox = fminf(fminf(fminf(p0.x, p1.x), fminf(p2.x, p3.x)), fminf(p4.x, p5.x));
    const float hix = fmaxf(fmaxf(fmaxf(p0.x, p1.x), fmaxf(p2.x, p3.x)), fmaxf(p4.x, p5.x));
    const float loy = fminf(fminf(fminf(p0.y, p1.y), fminf(p2.y, p3.y)), fminf(p4.y, p5.y));
    const float hiy = fmaxf(fmaxf(fmaxf(p0.y, p1.y), fmaxf(p2.y, p3.y)), fmaxf(p4.y, p5.y));
    const float loz = fminf(fminf(fminf(p0.z, p1.z), fminf(p2.z, p3.z)), fminf(p4.z, p5.z));
    const float hiz = fmaxf(fmaxf(fmaxf(p0.z, p1.z), fmaxf(p2.z, p3.z)), fmaxf(p4.z, p5.z));
    return lox > 0.f || hix < 0.f || loy > 0.f || hiy < 0.f || loz > 0.f || hiz < 0.f;
}

// relative start position and motion of corner k seen from vertex a
__device__ __forceinline__ void rel_path(const Dev &d, int k, float3 Xa, float3 uta, float3 ua, float3 &A, float3 &B) {
    const float3 utk = f3(__ldg(d.ut + k));
    A = (f3(__ldg(d.rest + k)) - Xa) + (utk - uta);
    B = (f3(__ldg(d.u + k)) - ua) - (utk - uta);
}

// earliest admissible impact of vertex a (boundary index k) among the
// triangles of this lane's cells: pass 0 returns the earliest time (or -1)
// and keeps the hits of its tie window in `win`; pass 1 (only when a window
// was full) the lowest triangle index hit by time `lim` (or -1)
template <int Q>
__device__ __forceinline__ float earliest_impact(const Dev &d, int k, float3 Xa, float3 uta, float3 ua, float3 mid,
                                                float Ra, int3 cell, int nb, int lane, float slack, int pass,
                                                float lim, int &pair, TieWindow &win) {
    const int g0 = d.ring_off[k], g1 = d.ring_off[k + 1];
    float best = -1.f;
    for (int n = lane; n < 27; n += Q) {
        const int b = neighbour_bucket(cell, n, nb);
        const int e1 = d.cell_start[b + 1];
        for (int e = d.cell_start[b]; e < e1; ++e) {
            if (sphere_far(d.cell_tri_sph[e], mid, Ra + slack)) continue;
            const int t = d.cell_tri[e];
            if (pass == 1 && pair >= 0 && t >= pair) continue;
            const int4 v = d.tri[t];
            bool adjacent = false;
            for (int g = g0; g < g1 && !adjacent; ++g) {
                const int q = d.ring[g];
                adjacent = (q == v.x) | (q == v.y) | (q == v.z);
            }
            if (adjacent) continue;
            float3 A0, A1, A2, B0, B1, B2, w;
            rel_path(d, v.x, Xa, uta, ua, A0, B0);
            rel_path(d, v.y, Xa, uta, ua, A1, B1);
            rel_path(d, v.z, Xa, uta, ua, A2, B2);
            // seen from the vertex the triangle moves inside the box of its six
            // corner positions; if that box misses the origin there is no impact
            if (box_misses_origin(A0, A1, A2, A0 + B0, A1 + B1, A2 + B2)) continue;
            const float ti = vt_impact(A0, A1, A2, B0, B1, B2, w);
            if (ti < 0.f) continue;
            if (pass == 0) {
                if (best < 0.f || ti < best) {
                    best = ti;
                    win.shrink(best, 1e-5f);
                }
                win.add(ti, t, best, 1e-5f);
            }
            if (pass == 1 && ti <= lim) pair = t;
        }
    }
    return best;
}

__global__ void __launch_bounds__(128) k_ccd(Dev d, int n_surf, int nb) {
    constexpr int Q = kCcdLanes;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = (int)(g / Q), lane = (int)(g % Q);
    const bool active = k < n_surf;  // inactive lanes still join the shuffles
    const int a = active ? d.surf[k] : 0;
    // a vertex paired at the step start keeps that pair (uniform over the group)
    const bool keep = active && d.contact[a] >= 0 && !(d.contact_w[a].w > 0.5f);
    const float3 Xa = f3(__ldg(d.rest + a)), uta = f3(__ldg(d.ut + a)), ua = f3(__ldg(d.u + a));
    const float3 path = ua - uta;
    const float3 mid = Xa + uta + 0.5f * path;
    const float Ra = 0.5f * sqrtf(dot(path, path));
    const float c = swept_cell_width(d);
    const float slack = kSlack * c;
    const int3 cell = (active && !keep) ? cell_of(d, mid, 1.0f / c) : make_int3(0, 0, 0);
    int pair = -1;
    TieWindow win = {0.f, 0.f, -1, -1, 0, false};
    float best = (active && !keep)
                     ? earliest_impact<Q>(d, k, Xa, uta, ua, mid, Ra, cell, nb, lane, slack, 0, 0.f, pair, win)
                     : -1.f;
    best = group_min_dist<Q>(best);
    const bool rescan = group_min_index<Q>(win.full ? 0 : -1) == 0;  // on every lane of the warp
    if (best >= 0.f) {  // uniform over the group
        if (rescan)
            earliest_impact<Q>(d, k, Xa, uta, ua, mid, Ra, cell, nb, lane, slack, 1, best + 1e-5f, pair, win);
        else
            pair = win.lowest(best + 1e-5f);
    }
    pair = group_min_index<Q>(pair);
    if (!active || lane != 0 || keep) return;
    if (pair >= 0) {
        const int4 v = d.tri[pair];
        float3 A0, A1, A2, B0, B1, B2, w = make_float3(0.f, 0.f, 0.f);
        rel_path(d, v.x, Xa, uta, ua, A0, B0);
        rel_path(d, v.y, Xa, uta, ua, A1, B1);
        rel_path(d, v.z, Xa, uta, ua, A2, B2);
        vt_impact(A0, A1, A2, B0, B1, B2, w);
        d.contact[a] = pair;
        d.contact_w[a] = make_float4(w.x, w.y, w.z, 1.f);
        atomicAdd(d.counters + 3, 1ull);
    } else {
        d.contact[a] = -1;
        d.contact_w[a] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void k_rev_count(Dev d, int n_surf, int n_free, int *count) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_surf) return;
    const int T = d.contact[d.surf[k]];
    if (T < 0) return;
    const int4 v = d.tri[T];
    if (v.x < n_free) atomicAdd(count + v.x, 1);
    if (v.y < n_free) atomicAdd(count + v.y, 1);
    if (v.z < n_free) atomicAdd(count + v.z, 1);
}

__global__ void k_rev_fill(Dev d, int n_surf, int n_free) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_surf) return;
    const int a = d.surf[k];
    const int T = d.contact[a];
    if (T < 0) return;
    const int4 v = d.tri[T];
    const int c[3] = {v.x, v.y, v.z};
    for (int j = 0; j < 3; ++j)
        if (c[j] < n_free) d.rev[d.rev_off[c[j]] + atomicAdd(d.rev_fill + c[j], 1)] = a;
}

// insertion sort of each corner's (short) list; only boundary vertices have one
__global__ void k_rev_sort(Dev d, int n_surf, int n_free) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_surf) return;
    const int i = d.surf[k];
    if (i >= n_free) return;
    const int r0 = d.rev_off[i], r1 = d.rev_off[i + 1];
    for (int p = r0 + 1; p < r1; ++p) {
        const int key = d.rev[p];
        int q = p - 1;
        while (q >= r0 && d.rev[q] > key) {
            d.rev[q + 1] = d.rev[q];
            --q;
        }
        d.rev[q + 1] = key;
    }
}

// ---- exclusive prefix sum of n ints into out[0..n] (out[n] = total) -------
__device__ __forceinline__ int block_exclusive_scan(int v, int *total) {
    __shared__ int warp_sum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int s = lane < kScanThreads / 32 ? warp_sum[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        if (lane < kScanThreads / 32) warp_sum[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const int before = wid > 0 ? warp_sum[wid - 1] : 0;
    *total = warp_sum[kScanThreads / 32 - 1];
    __syncthreads();  // warp_sum is reused by the next call
    return before + incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int *in, int *out, int n, int *tile_sums) {
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < n ? in[base + j] : 0;
        s += v[j];
    }
    int total;
    int run = block_exclusive_scan(s, &total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// one block: exclusive scan of the tile sums in place; tile_sums[n_tiles] = total
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int *tile_sums, int n_tiles) {
    int carry = 0;
    for (int b0 = 0; b0 < n_tiles; b0 += kScanThreads) {
        const int i = b0 + threadIdx.x;
        const int v = i < n_tiles ? tile_sums[i] : 0;
        int total;
        const int ex = block_exclusive_scan(v, &total);
        if (i < n_tiles) tile_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) tile_sums[n_tiles] = carry;
}

__global__ void k_scan_add(int *out, int n, const int *tile_sums, int n_tiles) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_sums[i / kScanTile];
    if (i == 0) out[n] = tile_sums[n_tiles];
}

void exclusive_scan(const int *in, int *out, int n, int *tmp, cudaStream_t s) {
    const int tiles = std::max(1, (int)blocks_for(n, kScanTile));
    k_scan_tiles<<<tiles, kScanThreads, 0, s>>>(in, out, n, tmp);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp, tiles);
    k_scan_add<<<std::max(1u, blocks_for(n, 256)), 256, 0, s>>>(out, n, tmp, tiles);
}


// ---- edge-edge CCD ------------------------------------------------------------
// Bounding sphere of each boundary edge's motion (both endpoints at x^t and
// at the current iterate).
__global__ void k_edge_bounds(Dev d, int n, unsigned *rmax) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int4 v = d.edge_v[e];
    const float3 X0 = f3(__ldg(d.rest + v.x)), X1 = f3(__ldg(d.rest + v.y));
    const float3 p[4] = {X0 + f3(__ldg(d.ut + v.x)), X1 + f3(__ldg(d.ut + v.y)), X0 + f3(__ldg(d.u + v.x)),
                         X1 + f3(__ldg(d.u + v.y))};
    const float3 m = 0.25f * (p[0] + p[1] + p[2] + p[3]);
    float R2 = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float3 q = p[k] - m;
        R2 = fmaxf(R2, dot(q, q));
    }
    float R = sqrtf(R2);
    if (!(R >= 0.f)) R = 0.f;
    d.edge_sphere[e] = make_float4(m.x, m.y, m.z, R);
    atomicMax(rmax, __float_as_uint(R));
}

// Time of impact of edges (p0, p1) and (q0, q1): with A_k + t B_k the paths
// of p1, q0, q1 relative to p0, the four points are coplanar where the
// cubic (p1 - p0) . ((q0 - p0) x (q1 - p0)) vanishes; its roots are taken in
// order and the first at which the segments cross (p0 + s (p1 - p0) =
// q0 + u (q1 - q0), s and u in [0, 1], in their common plane) is the impact.
// Segments within about 6 degrees of parallel (|e x g| < 0.1 |e| |g|) do not
// count: their crossing point is ill-conditioned.  -1 if none; s, u out.
__device__ __forceinline__ float ee_impact(float3 A0, float3 A1, float3 A2, float3 B0, float3 B1, float3 B2,
                                           float &s, float &u) {
    const float3 a12 = cross(A1, A2);
    const float c0 = dot(A0, a12);
    const float c1 = dot(B0, a12) + dot(A0, cross(B1, A2)) + dot(A0, cross(A1, B2));
    const float3 b12 = cross(B1, B2);
    const float c2 = dot(B0, cross(B1, A2)) + dot(B0, cross(A1, B2)) + dot(A0, b12);
    const float c3 = dot(B0, b12);
    float t0 = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
        const float t = cubic_first_root(c0, c1, c2, c3, t0);
        if (t < 0.f) return -1.f;
        const float3 e = A0 + t * B0, w = A1 + t * B1;
        const float3 g = (A2 + t * B2) - w;
        const float3 n = cross(e, g);
        const float nn = dot(n, n);
        if (nn > 0.01f * dot(e, e) * dot(g, g)) {  // not within ~6 degrees of parallel
            s = dot(cross(w, g), n) / nn;
            u = dot(cross(w, e), n) / nn;
            if (s >= 0.f && s <= 1.f && u >= 0.f && u <= 1.f) return t;
        }
        t0 = t + 1e-6f;
        if (t0 >= 1.f) return -1.f;
    }
    return -1.f;
}

// path of vertex k relative to vertex o: A (at x^t) + t B
__device__ __forceinline__ void rel_path2(const Dev &d, int k, int o, float3 &A, float3 &B) {
    const float3 uto = f3(__ldg(d.ut + o)), uo = f3(__ldg(d.u + o)), utk = f3(__ldg(d.ut + k));
    A = (f3(__ldg(d.rest + k)) - f3(__ldg(d.rest + o))) + (utk - uto);
    B = (f3(__ldg(d.u + k)) - uo) - (utk - uto);
}

// path of vertex k relative to vertex o, with o's rest position, x^t and
// current displacements given (the same arithmetic as rel_path2)
__device__ __forceinline__ void rel_path_from(const Dev &d, int k, float3 Ro, float3 uto, float3 uo, float3 &A,
                                              float3 &B) {
    const float3 utk = f3(__ldg(d.ut + k));
    A = (f3(__ldg(d.rest + k)) - Ro) + (utk - uto);
    B = (f3(__ldg(d.u + k)) - uo) - (utk - uto);
}

// earliest impact of edge e (vertices p0, p1, rings k0, k1) among the edges
// of this lane's cells; pass 0: earliest time, with the hits in its tie
// window kept in `win`; pass 1 (only when a window was full): lowest index
// hit by `lim`.  Candidates: no vertex in the 1-ring of p0 or p1.  The
// filters run cheapest first (bounding spheres, a shared vertex, the motion
// boxes seen from p0, then the rings); the candidate set does not depend on
// their order.
template <int Q>
__device__ __forceinline__ float earliest_edge(const Dev &d, int e, int4 ev, float4 sph, int3 cell, int nb, int lane,
                                              float slack, int pass, float lim, int &pair, TieWindow &win) {
    const int g0 = d.ring_off[ev.z], g1 = d.ring_off[ev.z + 1];
    const int h0 = d.ring_off[ev.w], h1 = d.ring_off[ev.w + 1];
    const float3 Ro = f3(__ldg(d.rest + ev.x)), uto = f3(__ldg(d.ut + ev.x)), uo = f3(__ldg(d.u + ev.x));
    float3 A0, B0;
    rel_path_from(d, ev.y, Ro, uto, uo, A0, B0);
    // seen from p0, both segments move inside the box of their end
    // positions; boxes that do not overlap cannot meet
    const float3 z = make_float3(0.f, 0.f, 0.f);
    const float3 lo_e = fminf3(fminf3(z, A0), A0 + B0), hi_e = fmaxf3(fmaxf3(z, A0), A0 + B0);
    float best = -1.f;
    for (int n = lane; n < 27; n += Q) {
        const int b = neighbour_bucket(cell, n, nb);
        const int e1 = d.edge_start[b + 1];
        for (int k = d.edge_start[b]; k < e1; ++k) {
            if (sphere_far(d.cell_edge_sph[k], make_float3(sph.x, sph.y, sph.z), sph.w + slack)) continue;
            const int f = d.cell_edge[k];
            if (f == e || (pass == 1 && pair >= 0 && f >= pair)) continue;
            const int4 fv = d.edge_v[f];
            if (fv.x == ev.x || fv.x == ev.y || fv.y == ev.x || fv.y == ev.y) continue;  // in both rings
            float3 A1, A2, B1, B2;
            rel_path_from(d, fv.x, Ro, uto, uo, A1, B1);
            rel_path_from(d, fv.y, Ro, uto, uo, A2, B2);
            const float3 lo_f = fminf3(fminf3(A1, A2), fminf3(A1 + B1, A2 + B2));
            const float3 hi_f = fmaxf3(fmaxf3(A1, A2), fmaxf3(A1 + B1, A2 + B2));
            if (lo_f.x > hi_e.x || hi_f.x < lo_e.x || lo_f.y > hi_e.y || hi_f.y < lo_e.y || lo_f.z > hi_e.z ||
                hi_f.z < lo_e.z)
                continue;
            bool adjacent = false;
            for (int g = g0; g < g1 && !adjacent; ++g) {
                const int q = d.ring[g];
                adjacent = (q == fv.x) | (q == fv.y);
            }
            for (int g = h0; g < h1 && !adjacent; ++g) {
                const int q = d.ring[g];
                adjacent = (q == fv.x) | (q == fv.y);
            }
            if (adjacent) continue;
            float ss, uu;
            const float t = ee_impact(A0, A1, A2, B0, B1, B2, ss, uu);
            if (t < 0.f) continue;
            if (pass == 0) {
                if (best < 0.f || t < best) {
                    best = t;
                    win.shrink(best, 1e-5f);
                }
                win.add(t, f, best, 1e-5f);
            }
            if (pass == 1 && t <= lim) pair = f;
        }
    }
    return best;
}

__global__ void __launch_bounds__(128) k_ee_query(Dev d, int n_edges, int nb) {
    constexpr int Q = kEdgeLanes;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int e = (int)(g / Q), lane = (int)(g % Q);
    const bool active = e < n_edges;
    const bool carried = active && d.ee_partner[e] >= 0 && d.ee_prm[e].z > 0.5f;
    const int4 ev = active ? d.edge_v[e] : make_int4(0, 0, 0, 0);
    const float4 sph = active ? d.edge_sphere[e] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float c = edge_cell_width(d);
    const float slack = kSlack * c;
    const bool search = active && !carried;
    const int3 cell = search ? cell_of(d, make_float3(sph.x, sph.y, sph.z), 1.0f / c) : make_int3(0, 0, 0);
    int pair = -1;
    TieWindow win = {0.f, 0.f, -1, -1, 0, false};
    float best = search ? earliest_edge<Q>(d, e, ev, sph, cell, nb, lane, slack, 0, 0.f, pair, win) : -1.f;
    best = group_min_dist<Q>(best);
    // every lane's hits by best + 1e-5 are in its window unless it was full
    // (a lane's window only drops hits later than its own earliest + 1e-5);
    // the shuffles run on every lane of the warp
    const bool rescan = group_min_index<Q>(win.full ? 0 : -1) == 0;
    if (best >= 0.f) {
        if (rescan)
            earliest_edge<Q>(d, e, ev, sph, cell, nb, lane, slack, 1, best + 1e-5f, pair, win);
        else
            pair = win.lowest(best + 1e-5f);
    }
    pair = group_min_index<Q>(pair);
    if (!active || lane != 0) return;
    d.ee_found[e] = pair;
    if (pair >= 0) {
        const int4 fv = d.edge_v[pair];
        float3 A0, A1, A2, B0, B1, B2;
        rel_path2(d, ev.y, ev.x, A0, B0);
        rel_path2(d, fv.x, ev.x, A1, B1);
        rel_path2(d, fv.y, ev.x, A2, B2);
        float ss = 0.f, uu = 0.f;
        const float t = ee_impact(A0, A1, A2, B0, B1, B2, ss, uu);
        d.ee_hit[e] = make_float4(ss, uu, t, 0.f);
    }
}

// The pair each edge holds after a CCD: the edge it hit first, unless that
// edge hit this one too and has the lower index (it holds the pair), or
// already carries this pair; the normal is the edges' unit common
// perpendicular at the current iterate, oriented along x_b - x_a there and
// frozen (a pair with x_b - x_a perpendicular to it is dropped).  Carried
// pairs stay.
__global__ void k_ee_assign(Dev d, int n_edges) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edges) return;
    if (d.ee_partner[e] >= 0 && d.ee_prm[e].z > 0.5f) return;  // carried
    const int f = d.ee_found[e];
    int partner = -1;
    if (f >= 0 && !(d.ee_found[f] == e && f < e) && !(d.ee_partner[f] == e && d.ee_prm[f].z > 0.5f)) {
        const float4 h = d.ee_hit[e];
        const int4 ev = d.edge_v[e], fv = d.edge_v[f];
        float3 A0, B0, A1, B1, A2, B2;  // current positions relative to p0: A + B
        rel_path2(d, ev.y, ev.x, A0, B0);
        rel_path2(d, fv.x, ev.x, A1, B1);
        rel_path2(d, fv.y, ev.x, A2, B2);
        const float3 p1 = A0 + B0, q0 = A1 + B1, q1 = A2 + B2;
        const float3 dl = ((1.f - h.y) * q0 + h.y * q1) - h.x * p1;
        // the edges' common perpendicular, pointing along x_b - x_a
        const float3 nv = cross(p1, q1 - q0);
        const float side = dot(nv, dl);
        float len = sqrtf(dot(nv, nv));
        if (len > 0.f && side != 0.f) {
            if (side < 0.f) len = -len;
            partner = f;
            d.ee_prm[e] = make_float4(h.x, h.y, 0.f, 0.f);
            d.ee_nrm[e] = make_float4(nv.x / len, nv.y / len, nv.z / len, 0.f);
            atomicAdd(d.counters + 3, 1ull);
        }
    }
    d.ee_partner[e] = partner;
}

// At the step start: a pair whose depth is still positive (at x^t) is
// carried into the step; the others end.
__global__ void k_ee_carry(Dev d, int n_edges) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edges) return;
    const int f = d.ee_partner[e];
    if (f < 0) return;
    const float4 prm = d.ee_prm[e], n = d.ee_nrm[e];
    const int4 ev = d.edge_v[e], fv = d.edge_v[f];
    float3 A0, B0, A1, B1, A2, B2;
    rel_path2(d, ev.y, ev.x, A0, B0);
    rel_path2(d, fv.x, ev.x, A1, B1);
    rel_path2(d, fv.y, ev.x, A2, B2);
    const float3 p1 = A0 + B0, q0 = A1 + B1, q1 = A2 + B2;
    const float3 dl = ((1.f - prm.y) * q0 + prm.y * q1) - prm.x * p1;
    if (dot(dl, make_float3(n.x, n.y, n.z)) > 0.f) {
        d.ee_prm[e] = make_float4(prm.x, prm.y, 1.f, 0.f);
    } else {
        d.ee_partner[e] = -1;
        d.ee_prm[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// per free vertex, its edge-edge items (4 (holding edge) + role), sorted
__global__ void k_ee_count(Dev d, int n_edges, int n_free, int *count) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edges) return;
    const int f = d.ee_partner[e];
    if (f < 0) return;
    const int4 ev = d.edge_v[e], fv = d.edge_v[f];
    const int v[4] = {ev.x, ev.y, fv.x, fv.y};
    for (int j = 0; j < 4; ++j)
        if (v[j] < n_free) atomicAdd(count + v[j], 1);
}

__global__ void k_ee_fill(Dev d, int n_edges, int n_free) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edges) return;
    const int f = d.ee_partner[e];
    if (f < 0) return;
    const int4 ev = d.edge_v[e], fv = d.edge_v[f];
    const int v[4] = {ev.x, ev.y, fv.x, fv.y};
    for (int j = 0; j < 4; ++j)
        if (v[j] < n_free) d.ee_item[d.ee_off[v[j]] + atomicAdd(d.ee_vfill + v[j], 1)] = 4 * e + j;
}

__global__ void k_ee_sort(Dev d, int n_free) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_free) return;
    const int r0 = d.ee_off[i], r1 = d.ee_off[i + 1];
    for (int p = r0 + 1; p < r1; ++p) {
        const int key = d.ee_item[p];
        int q = p - 1;
        while (q >= r0 && d.ee_item[q] > key) {
            d.ee_item[q + 1] = d.ee_item[q];
            --q;
        }
        d.ee_item[q + 1] = key;
    }
}

void build_ee_lists(const Dev &d, const CollideDims &c, int n_free, cudaStream_t s) {
    if (n_free <= 0) return;
    cudaMemsetAsync(d.ee_vfill, 0, sizeof(int) * (size_t)n_free, s);
    k_ee_count<<<blocks_for(c.n_edges, 256), 256, 0, s>>>(d, c.n_edges, n_free, d.ee_vfill);
    exclusive_scan(d.ee_vfill, d.ee_off, n_free, d.scan_tmp, s);
    cudaMemsetAsync(d.ee_vfill, 0, sizeof(int) * (size_t)n_free, s);
    k_ee_fill<<<blocks_for(c.n_edges, 256), 256, 0, s>>>(d, c.n_edges, n_free);
    k_ee_sort<<<blocks_for(n_free, 256), 256, 0, s>>>(d, n_free);
}

// reverse corner lists of the current pairs, for the sweep
void build_reverse_lists(const Dev &d, const CollideDims &c, int n_free, cudaStream_t s) {
    if (n_free <= 0) return;
    cudaMemsetAsync(d.rev_fill, 0, sizeof(int) * (size_t)n_free, s);
    k_rev_count<<<blocks_for(c.n_surf, 256), 256, 0, s>>>(d, c.n_surf, n_free, d.rev_fill);
    exclusive_scan(d.rev_fill, d.rev_off, n_free, d.scan_tmp, s);
    cudaMemsetAsync(d.rev_fill, 0, sizeof(int) * (size_t)n_free, s);
    k_rev_fill<<<blocks_for(c.n_surf, 256), 256, 0, s>>>(d, c.n_surf, n_free);
    k_rev_sort<<<blocks_for(c.n_surf, 256), 256, 0, s>>>(d, c.n_surf, n_free);
}

}  // namespace

int scan_tmp_needed(int n) { return (int)blocks_for(std::max(n, 1), kScanTile) + 1; }

void launch_detect(const Dev &d, const CollideDims &c, int n_free, cudaStream_t s) {
    if (c.n_surf <= 0 || c.n_tris <= 0) return;
    // broad phase: bounding spheres and the cell size, then triangles and
    // tets bucketed by the cell of their centre
    cudaMemsetAsync(d.cell_size, 0, 2 * sizeof(unsigned), s);
    k_bounds<3><<<blocks_for(c.n_tris, 256), 256, 0, s>>>(d, d.tri, c.n_tris, d.tri_sphere, d.cell_size);
    k_bounds<4><<<blocks_for(c.n_tets, 256), 256, 0, s>>>(d, d.tet_v, c.n_tets, d.tet_sphere, d.cell_size + 1);
    cudaMemsetAsync(d.cell_fill, 0, sizeof(int) * (size_t)c.n_buckets, s);
    k_count<3><<<blocks_for(c.n_tris, 256), 256, 0, s>>>(d, d.tri_sphere, c.n_tris, c.n_buckets, c.radius,
                                                         d.cell_fill);
    exclusive_scan(d.cell_fill, d.cell_start, c.n_buckets, d.scan_tmp, s);
    cudaMemsetAsync(d.cell_fill, 0, sizeof(int) * (size_t)c.n_buckets, s);
    k_fill<3><<<blocks_for(c.n_tris, 256), 256, 0, s>>>(d, d.tri_sphere, c.n_tris, c.n_buckets, c.radius,
                                                        d.cell_start, d.cell_fill, d.cell_tri, d.cell_tri_sph);
    cudaMemsetAsync(d.tet_fill, 0, sizeof(int) * (size_t)c.n_tet_buckets, s);
    k_count<4><<<blocks_for(c.n_tets, 256), 256, 0, s>>>(d, d.tet_sphere, c.n_tets, c.n_tet_buckets, c.radius,
                                                         d.tet_fill);
    exclusive_scan(d.tet_fill, d.tet_start, c.n_tet_buckets, d.scan_tmp, s);
    cudaMemsetAsync(d.tet_fill, 0, sizeof(int) * (size_t)c.n_tet_buckets, s);
    k_fill<4><<<blocks_for(c.n_tets, 256), 256, 0, s>>>(d, d.tet_sphere, c.n_tets, c.n_tet_buckets, c.radius,
                                                        d.tet_start, d.tet_fill, d.cell_tet, d.cell_tet_sph);
    // narrow phase
    k_query<<<blocks_for((long long)c.n_surf * kProximityLanes, 128), 128, 0, s>>>(d, c.n_surf, c.n_buckets,
                                                                              c.n_tet_buckets, c.radius);
    build_reverse_lists(d, c, n_free, s);
    if (c.ee_on && c.n_edges > 0) {  // edge-edge pairs still penetrated at x^t are carried
        k_ee_carry<<<blocks_for(c.n_edges, 256), 256, 0, s>>>(d, c.n_edges);
        build_ee_lists(d, c, n_free, s);
    }
}

void launch_ccd(const Dev &d, const CollideDims &c, int n_free, cudaStream_t s) {
    if (c.n_surf <= 0 || c.n_tris <= 0 || !d.contact_w) return;
    // broad phase: spheres of the triangles' motions and the vertices' half paths
    cudaMemsetAsync(d.cell_size, 0, 3 * sizeof(unsigned), s);
    k_bounds_swept<<<blocks_for(c.n_tris, 256), 256, 0, s>>>(d, c.n_tris, d.tri_sphere, d.cell_size);
    k_path_radius<<<blocks_for(c.n_surf, 256), 256, 0, s>>>(d, c.n_surf, d.cell_size + 2);
    cudaMemsetAsync(d.cell_fill, 0, sizeof(int) * (size_t)c.n_buckets, s);
    k_count<5><<<blocks_for(c.n_tris, 256), 256, 0, s>>>(d, d.tri_sphere, c.n_tris, c.n_buckets, 0.f, d.cell_fill);
    exclusive_scan(d.cell_fill, d.cell_start, c.n_buckets, d.scan_tmp, s);
    cudaMemsetAsync(d.cell_fill, 0, sizeof(int) * (size_t)c.n_buckets, s);
    k_fill<5><<<blocks_for(c.n_tris, 256), 256, 0, s>>>(d, d.tri_sphere, c.n_tris, c.n_buckets, 0.f, d.cell_start,
                                                        d.cell_fill, d.cell_tri, d.cell_tri_sph);
    k_ccd<<<blocks_for((long long)c.n_surf * kCcdLanes, 128), 128, 0, s>>>(d, c.n_surf, c.n_buckets);
    build_reverse_lists(d, c, n_free, s);
    if (!c.ee_on || c.n_edges <= 0) return;
    // edge-edge: spheres of the edges' motions, their hash, the query, the pairs
    cudaMemsetAsync(d.cell_size + 3, 0, sizeof(unsigned), s);
    k_edge_bounds<<<blocks_for(c.n_edges, 256), 256, 0, s>>>(d, c.n_edges, d.cell_size + 3);
    cudaMemsetAsync(d.edge_fill, 0, sizeof(int) * (size_t)c.n_edge_buckets, s);
    k_count<6><<<blocks_for(c.n_edges, 256), 256, 0, s>>>(d, d.edge_sphere, c.n_edges, c.n_edge_buckets, 0.f,
                                                          d.edge_fill);
    exclusive_scan(d.edge_fill, d.edge_start, c.n_edge_buckets, d.scan_tmp, s);
    cudaMemsetAsync(d.edge_fill, 0, sizeof(int) * (size_t)c.n_edge_buckets, s);
    k_fill<6><<<blocks_for(c.n_edges, 256), 256, 0, s>>>(d, d.edge_sphere, c.n_edges, c.n_edge_buckets, 0.f,
                                                         d.edge_start, d.edge_fill, d.cell_edge, d.cell_edge_sph);
    k_ee_query<<<blocks_for((long long)c.n_edges * kEdgeLanes, 128), 128, 0, s>>>(d, c.n_edges, c.n_edge_buckets);
    k_ee_assign<<<blocks_for(c.n_edges, 256), 256, 0, s>>>(d, c.n_edges);
    build_ee_lists(d, c, n_free, s);
}

}  // namespace vbd

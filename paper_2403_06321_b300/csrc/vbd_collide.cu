// vbd_collide.cu -- vertex-triangle self-collision detection (Sec. 3.5) for
// sm_103a, run once at the start of each step on x^t.
//
// A boundary vertex a has penetrated when it lies in (or on) a tet it is not
// a vertex of.  It is then paired with the nearest boundary triangle within
// the detection distance r that shares no tet with it; triangles within
// 1e-5 r of the nearest distance count as tied and the lowest index wins.
//
// Broad phase: spatial hashes of triangle and tet centroids with one cell
// size c = 1.01 max(R_tri + r, R_tet), R the largest centroid-to-corner
// distance of any triangle (tet) at this step.  A triangle within r of a
// vertex, or a tet holding it, has its centroid within c of the vertex (the
// element lies in the ball of radius R about its centroid), hence in one of
// the 27 cells around the vertex's cell.  Each element is stored once
// (count, prefix sum, fill), so the tables never overflow.
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

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// The broad phase works in FP64 on x = X + u (both FP32, so the sum is exact):
// cell indices then stay exact far from the origin.
__device__ __forceinline__ double3 position(const Dev &d, int i) {
    const float4 X = __ldg(d.rest + i), u = __ldg(d.u + i);
    return make_double3((double)X.x + u.x, (double)X.y + u.y, (double)X.z + u.z);
}

// centroid of the first K corners of an element (K = 3 triangle, 4 tet)
template <int K>
__device__ __forceinline__ double3 centroid(const Dev &d, int4 v) {
    const int c[4] = {v.x, v.y, v.z, v.w};
    double3 m = make_double3(0.0, 0.0, 0.0);
    for (int k = 0; k < K; ++k) {
        const double3 p = position(d, c[k]);
        m.x += p.x; m.y += p.y; m.z += p.z;
    }
    return make_double3(m.x / K, m.y / K, m.z / K);
}

__device__ __forceinline__ double inv_cell_width(const Dev &d, float r) {
    const double c = fmax((double)__uint_as_float(d.cell_size[0]) + r, (double)__uint_as_float(d.cell_size[1]));
    return 1.0 / (1.01 * c + 1e-300);
}

__device__ __forceinline__ long long cell_coord(double x, double inv_c) {
    // clamp so that the conversion is defined for any finite or infinite input
    const double q = fmin(fmax(floor(x * inv_c), -1.0e15), 1.0e15);
    return (long long)q;
}

__device__ __forceinline__ int bucket_of(long long i, long long j, long long k, int nb) {
    unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ull;
    h ^= (unsigned long long)j * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
    h ^= (unsigned long long)k * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
    h ^= h >> 31;
    return (int)(h & (unsigned long long)(nb - 1));
}

// largest centroid-to-corner distance of the elements, as float bits (the
// values are non-negative, so unsigned order is float order)
template <int K>
__global__ void k_radius(Dev d, const int4 *items, int n, unsigned *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int4 v = items[t];
    const double3 m = centroid<K>(d, v);
    const int c[4] = {v.x, v.y, v.z, v.w};
    double R2 = 0.0;
    for (int k = 0; k < K; ++k) {
        const double3 p = position(d, c[k]);
        const double dx = p.x - m.x, dy = p.y - m.y, dz = p.z - m.z;
        R2 = fmax(R2, dx * dx + dy * dy + dz * dz);
    }
    float R = (float)sqrt(R2);
    if (!(R >= 0.f)) R = 0.f;  // a NaN position never widens the cells
    atomicMax(out, __float_as_uint(R));
}

template <int K>
__device__ __forceinline__ int item_bucket(const Dev &d, int4 v, double inv_c, int nb) {
    const double3 m = centroid<K>(d, v);
    return bucket_of(cell_coord(m.x, inv_c), cell_coord(m.y, inv_c), cell_coord(m.z, inv_c), nb);
}

template <int K>
__global__ void k_count(Dev d, const int4 *items, int n, int nb, float r, int *count) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    atomicAdd(count + item_bucket<K>(d, items[t], inv_cell_width(d, r), nb), 1);
}

template <int K>
__global__ void k_fill(Dev d, const int4 *items, int n, int nb, float r, const int *start, int *fill,
                       int *entries) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int b = item_bucket<K>(d, items[t], inv_cell_width(d, r), nb);
    entries[start[b] + atomicAdd(fill + b, 1)] = t;
}

// Whether the origin lies in the closed tet with corners p0..p3 (positions
// relative to the vertex): its barycentric coordinates, from the edge matrix
// E = [p1 - p0, p2 - p0, p3 - p0] by Cramer's rule, are all >= 0.
__device__ __forceinline__ bool origin_in_tet(float3 p0, float3 p1, float3 p2, float3 p3) {
    const float3 e1 = p1 - p0, e2 = p2 - p0, e3 = p3 - p0;
    const float3 r = make_float3(-p0.x, -p0.y, -p0.z);
    const float D = dot(e1, cross(e2, e3));
    if (D == 0.0f) return false;
    const float l1 = dot(r, cross(e2, e3)) / D;
    const float l2 = dot(e1, cross(r, e3)) / D;
    const float l3 = dot(e1, cross(e2, r)) / D;
    return l1 >= 0.0f && l2 >= 0.0f && l3 >= 0.0f && 1.0f - (l1 + l2 + l3) >= 0.0f;
}

// the 27 buckets around a cell, each once (two neighbour cells may share one)
__device__ __forceinline__ int neighbour_buckets(long long ci, long long cj, long long ck, int nb, int out[27]) {
    int n = 0;
    for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj)
            for (int dk = -1; dk <= 1; ++dk) {
                const int b = bucket_of(ci + di, cj + dj, ck + dk, nb);
                bool dup = false;
                for (int q = 0; q < n; ++q) dup |= (out[q] == b);
                if (!dup) out[n++] = b;
            }
    return n;
}

__device__ __forceinline__ float3 rel(const Dev &d, int k, float3 Xa, float3 ua) {
    return (f3(__ldg(d.rest + k)) - Xa) + (f3(__ldg(d.u + k)) - ua);
}

// one thread per boundary vertex: penetration test, then the nearest
// admissible triangle within r
__global__ void k_query(Dev d, int n_surf, int nb_tri, int nb_tet, float r) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_surf) return;
    const int a = d.surf[k];
    const double inv_c = inv_cell_width(d, r);
    const double3 xa = position(d, a);
    const long long ci = cell_coord(xa.x, inv_c), cj = cell_coord(xa.y, inv_c), ck = cell_coord(xa.z, inv_c);
    const float3 Xa = f3(__ldg(d.rest + a)), ua = f3(__ldg(d.u + a));
    int bk[27];
    // penetration: inside a tet that does not hold the vertex
    int nbk = neighbour_buckets(ci, cj, ck, nb_tet, bk);
    bool inside = false;
    for (int q = 0; q < nbk && !inside; ++q) {
        const int e1 = d.tet_start[bk[q] + 1];
        for (int e = d.tet_start[bk[q]]; e < e1 && !inside; ++e) {
            const int4 v = d.tet_v[d.cell_tet[e]];
            if (v.x == a || v.y == a || v.z == a || v.w == a) continue;
            inside = origin_in_tet(rel(d, v.x, Xa, ua), rel(d, v.y, Xa, ua), rel(d, v.z, Xa, ua),
                                   rel(d, v.w, Xa, ua));
        }
    }
    int pair = -1;
    if (inside) {
        // pass 0: the nearest distance; pass 1: the lowest index within
        // 1e-5 r of it (a nearest point on a shared edge or corner is equally
        // near several triangles; rounding must not choose)
        const int g0 = d.ring_off[k], g1 = d.ring_off[k + 1];
        float best = -1.f;
        nbk = neighbour_buckets(ci, cj, ck, nb_tri, bk);
        for (int pass = 0; pass < 2 && !(pass == 1 && best < 0.f); ++pass) {
            const float lim = best + 1e-5f * r;
            for (int q = 0; q < nbk; ++q) {
                const int e1 = d.cell_start[bk[q] + 1];
                for (int e = d.cell_start[bk[q]]; e < e1; ++e) {
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
                    const float3 qp = make_float3(w.x * pa.x + w.y * pb.x + w.z * pc.x,
                                                  w.x * pa.y + w.y * pb.y + w.z * pc.y,
                                                  w.x * pa.z + w.y * pb.z + w.z * pc.z);
                    const float dist = sqrtf(dot(qp, qp));
                    if (dist > r) continue;
                    if (pass == 0 && (best < 0.f || dist < best)) best = dist;
                    if (pass == 1 && dist <= lim) pair = t;
                }
            }
        }
    }
    d.contact[a] = pair;
    if (pair >= 0) atomicAdd(d.counters + 3, 1ull);
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

}  // namespace

int scan_tmp_needed(int n) { return (int)blocks_for(std::max(n, 1), kScanTile) + 1; }

void launch_detect(const Dev &d, const CollideDims &c, int n_free, cudaStream_t s) {
    if (c.n_surf <= 0 || c.n_tris <= 0) return;
    // broad phase: cell size, then triangles and tets bucketed by centroid cell
    cudaMemsetAsync(d.cell_size, 0, 2 * sizeof(unsigned), s);
    k_radius<3><<<blocks_for(c.n_tris, 256), 256, 0, s>>>(d, d.tri, c.n_tris, d.cell_size);
    k_radius<4><<<blocks_for(c.n_tets, 256), 256, 0, s>>>(d, d.tet_v, c.n_tets, d.cell_size + 1);
    cudaMemsetAsync(d.cell_fill, 0, sizeof(int) * (size_t)c.n_buckets, s);
    k_count<3><<<blocks_for(c.n_tris, 256), 256, 0, s>>>(d, d.tri, c.n_tris, c.n_buckets, c.radius, d.cell_fill);
    exclusive_scan(d.cell_fill, d.cell_start, c.n_buckets, d.scan_tmp, s);
    cudaMemsetAsync(d.cell_fill, 0, sizeof(int) * (size_t)c.n_buckets, s);
    k_fill<3><<<blocks_for(c.n_tris, 256), 256, 0, s>>>(d, d.tri, c.n_tris, c.n_buckets, c.radius, d.cell_start,
                                                         d.cell_fill, d.cell_tri);
    cudaMemsetAsync(d.tet_fill, 0, sizeof(int) * (size_t)c.n_tet_buckets, s);
    k_count<4><<<blocks_for(c.n_tets, 256), 256, 0, s>>>(d, d.tet_v, c.n_tets, c.n_tet_buckets, c.radius,
                                                          d.tet_fill);
    exclusive_scan(d.tet_fill, d.tet_start, c.n_tet_buckets, d.scan_tmp, s);
    cudaMemsetAsync(d.tet_fill, 0, sizeof(int) * (size_t)c.n_tet_buckets, s);
    k_fill<4><<<blocks_for(c.n_tets, 256), 256, 0, s>>>(d, d.tet_v, c.n_tets, c.n_tet_buckets, c.radius,
                                                         d.tet_start, d.tet_fill, d.cell_tet);
    // narrow phase
    k_query<<<blocks_for(c.n_surf, 128), 128, 0, s>>>(d, c.n_surf, c.n_buckets, c.n_tet_buckets, c.radius);
    // reverse lists for the sweep
    if (n_free <= 0) return;
    cudaMemsetAsync(d.rev_fill, 0, sizeof(int) * (size_t)n_free, s);
    k_rev_count<<<blocks_for(c.n_surf, 256), 256, 0, s>>>(d, c.n_surf, n_free, d.rev_fill);
    exclusive_scan(d.rev_fill, d.rev_off, n_free, d.scan_tmp, s);
    cudaMemsetAsync(d.rev_fill, 0, sizeof(int) * (size_t)n_free, s);
    k_rev_fill<<<blocks_for(c.n_surf, 256), 256, 0, s>>>(d, c.n_surf, n_free);
    k_rev_sort<<<blocks_for(c.n_surf, 256), 256, 0, s>>>(d, c.n_surf, n_free);
}

}  // namespace vbd

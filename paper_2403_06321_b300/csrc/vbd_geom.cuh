// vbd_geom.cuh -- small float3 helpers and the vertex-triangle geometry shared
// by the sweep (contact forces) and the collision kernels (detection).
#pragma once
#include <cuda_runtime.h>

#include "vbd_kernels.h"

namespace vbd {
namespace geom {

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) {
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 operator+(float3 a, float3 b) {
    return make_float3(a.x + b.x, a.y + b.y, a.z + b.z);
}
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 fminf3(float3 a, float3 b) {
    return make_float3(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z));
}
__device__ __forceinline__ float3 fmaxf3(float3 a, float3 b) {
    return make_float3(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z));
}
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Barycentric weights of the point of triangle (a, b, c) nearest to the
// origin.  The triangle is convex, so that point is unique: the orthogonal
// projection onto the plane when it falls inside, else the nearest of the
// three edges' clamped projections (the first edge wins an exact tie).
__device__ __forceinline__ float3 nearest_weights(float3 a, float3 b, float3 c) {
    const float3 e0 = b - a, e1 = c - a;
    const float3 r = make_float3(-a.x, -a.y, -a.z);
    const float g00 = dot(e0, e0), g01 = dot(e0, e1), g11 = dot(e1, e1);
    const float r0 = dot(r, e0), r1 = dot(r, e1);
    const float den = g00 * g11 - g01 * g01;
    const float wb = (g11 * r0 - g01 * r1) / den;
    const float wc = (g00 * r1 - g01 * r0) / den;
    const float wa = 1.0f - wb - wc;
    if (wa >= 0.0f && wb >= 0.0f && wc >= 0.0f) return make_float3(wa, wb, wc);
    const float3 P[3] = {a, b, c};
    float best = -1.0f;
    float w[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const float3 p0 = P[e], p1 = P[(e + 1) % 3];
        const float3 dd = p1 - p0;
        float t = -dot(p0, dd) / dot(dd, dd);
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        const float3 q = p0 + t * dd;
        const float d2 = dot(q, q);
        if (best < 0.0f || d2 < best) {
            best = d2;
            w[0] = w[1] = w[2] = 0.0f;
            w[e] = 1.0f - t;
            w[(e + 1) % 3] = t;
        }
    }
    return make_float3(w[0], w[1], w[2]);
}

// Depth, normal and weights of the pair (vertex a, triangle t) at x = X + u:
// d = (q - x_a).n of Eq. 12 with q the contact point and n the triangle's
// unit normal (positive when the vertex is behind the triangle).
// Differences are formed separately for the rest positions and the
// displacements, so that FP32 keeps the small gaps exact to rounding.  A
// pair found by CCD (contact_w[a].w = 1) acts through its impact point,
// whose barycentric weights stay fixed (Sec. 3.5); a DCD pair through the
// nearest point.
__device__ __forceinline__ float pair_depth(const Dev &d, int a, int4 t, float3 &n, float3 &w) {
    const float3 Xa = f3(__ldg(d.rest + a)), ua = f3(__ldg(d.u + a));
    const float3 pa = (f3(__ldg(d.rest + t.x)) - Xa) + (f3(__ldg(d.u + t.x)) - ua);
    const float3 pb = (f3(__ldg(d.rest + t.y)) - Xa) + (f3(__ldg(d.u + t.y)) - ua);
    const float3 pc = (f3(__ldg(d.rest + t.z)) - Xa) + (f3(__ldg(d.u + t.z)) - ua);
    const float4 cw = d.contact_w ? d.contact_w[a] : make_float4(0.f, 0.f, 0.f, 0.f);
    w = cw.w > 0.5f ? make_float3(cw.x, cw.y, cw.z) : nearest_weights(pa, pb, pc);
    const float3 q = make_float3(w.x * pa.x + w.y * pb.x + w.z * pc.x, w.x * pa.y + w.y * pb.y + w.z * pc.y,
                                 w.x * pa.z + w.y * pb.z + w.z * pc.z);
    const float3 nn = cross(pb - pa, pc - pa);
    n = rsqrtf(dot(nn, nn)) * nn;
    return dot(q, n);
}

}  // namespace geom
}  // namespace vbd

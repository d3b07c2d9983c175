// vbd_kernels.cu -- forward kernels of Vertex Block Descent for sm_103a.
//
// One time step (Algorithm 1) is
//   k_predict            y (Eq. 3) and the initial guess (Sec. 3.7), once per step
//   k_sweep<L>           one Gauss-Seidel pass over one colour (Sec. 3.1-3.9),
//                        iters * n_colors launches per step -- the hot path
//                        (k_sweep_persist: the same on a persistent grid;
//                        k_sweep_rest: gradients recomputed from rest positions)
//   k_cheby              Chebyshev update (Eqs. 18-19), once per iteration if enabled
//   k_finish             v = (x - x^t)/h (Eq. 6), once per step
//
// The sweep is memory bound: per (vertex, incident tet) pair ("slot") it
// streams 48 bytes of precomputed rest data (three vertex ids and the three
// shape gradients) once per iteration and gathers three neighbour positions;
// the tet's volume follows from the gradients, its material from the vertex
// (or, for per-tet materials, from the tet's arrays).  Slots of one colour are contiguous, so the
// stream is fully sequential; L lanes of a warp cooperate on one vertex
// (lanes stride over its slots), reduce f_i and H_i with xor shuffles in a
// fixed order (deterministic), and one lane solves the 3x3 system.
#include "vbd_kernels.h"

#include <algorithm>
#include <cstdio>
#include <mutex>

#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "vbd_geom.cuh"

namespace cg = cooperative_groups;

namespace vbd {

namespace {

using geom::cross;
using geom::dot;
using geom::f3;
using geom::operator-;
using geom::operator+;

constexpr unsigned FULL = 0xffffffffu;

// f_i and the symmetric H_i (upper triangle) accumulated over incident tets
struct Acc {
    float f0, f1, f2, h00, h01, h02, h11, h12, h22;
};

// Contribution of one tet to the vertex that owns the slot (Eqs. 8-9 with the
// stable neo-Hookean element), written in terms of displacements so that no
// step subtracts nearly equal numbers.  With d_k = u_k - u_i for the three
// other vertices and their shape gradients g_k (g_i = -(g_a + g_b + g_c)):
//   F = I + D,  D = sum_k d_k g_k^T
//   J - 1      = tr D + (sum of principal 2x2 minors of D) + det D
//   c' = cof(F) g_i - g_i = (tr D) g_i - D^T g_i + cof(D) g_i,   c = g_i + c'
//   V P g_i    = V mu (D g_i - c') + V lam (J - 1) c     (alpha lam = lam + mu)
//   f_i -= V P g_i,   H_i += V mu |g_i|^2 I + V lam c c^T.
// Material of a slot: the tet's volume is 1 / (6 |det[g_a; g_b; g_c]|) (any
// three of a tet's four shape gradients are the rows of the inverse rest edge
// matrix up to a sign), mu and lambda are the vertex's, or the tet's.
__device__ __forceinline__ float2 slot_material(const Dev &d, const SweepParams &p, int s, float2 vm,
                                                float3 ga, float3 gb, float3 gc) {
    const float detg = dot(ga, cross(gb, gc));
    const float V = __frcp_rn(6.0f * fabsf(detg));
    if (p.per_tet_mat) {
        const int j = __ldcs(d.slot_tet + s);
        vm = make_float2(__ldg(d.tet_mu + j), __ldg(d.tet_lam + j));
    }
    return make_float2(V * vm.x, V * vm.y);
}

// Neighbour positions: through the read-only path when no other CTA writes d.u
// during the launch (one launch per colour), else from L2 (COH: the fused
// iteration kernel, where other CTAs of the cluster wrote the previous colour).
template <bool COH>
__device__ __forceinline__ float4 load_u(const float4 *u, int i) {
    return COH ? __ldcg(u + i) : __ldg(u + i);
}

// The element part shared by both slot forms: d_k = u_k - u_i, g_k the shape
// gradients of the three other vertices, Vmu = V mu, Vlam = V lambda.
__device__ __forceinline__ void tet_contrib(float3 da, float3 db, float3 dc, float3 ga, float3 gb, float3 gc,
                                            float Vmu, float Vlam, Acc &acc) {
    const float3 gi = make_float3(-(ga.x + gb.x + gc.x), -(ga.y + gb.y + gc.y), -(ga.z + gb.z + gc.z));
    // columns of D: D_s = da * ga[s] + db * gb[s] + dc * gc[s]
    const float3 D0 = make_float3(da.x * ga.x + db.x * gb.x + dc.x * gc.x,
                                  da.y * ga.x + db.y * gb.x + dc.y * gc.x,
                                  da.z * ga.x + db.z * gb.x + dc.z * gc.x);
    const float3 D1 = make_float3(da.x * ga.y + db.x * gb.y + dc.x * gc.y,
                                  da.y * ga.y + db.y * gb.y + dc.y * gc.y,
                                  da.z * ga.y + db.z * gb.y + dc.z * gc.y);
    const float3 D2 = make_float3(da.x * ga.z + db.x * gb.z + dc.x * gc.z,
                                  da.y * ga.z + db.y * gb.z + dc.y * gc.z,
                                  da.z * ga.z + db.z * gb.z + dc.z * gc.z);
    const float tr = D0.x + D1.y + D2.z;
    const float3 q0 = cross(D1, D2), q1 = cross(D2, D0), q2 = cross(D0, D1);  // columns of cof(D)
    // the sum of the principal 2x2 minors of D is the trace of cof(D)
    const float jm1 = tr + (q0.x + q1.y + q2.z) + dot(D0, q0);
    const float3 cp = make_float3(tr * gi.x - dot(D0, gi) + gi.x * q0.x + gi.y * q1.x + gi.z * q2.x,
                                  tr * gi.y - dot(D1, gi) + gi.x * q0.y + gi.y * q1.y + gi.z * q2.y,
                                  tr * gi.z - dot(D2, gi) + gi.x * q0.z + gi.y * q1.z + gi.z * q2.z);
    const float3 c = make_float3(gi.x + cp.x, gi.y + cp.y, gi.z + cp.z);
    const float3 Dg = make_float3(gi.x * D0.x + gi.y * D1.x + gi.z * D2.x,
                                  gi.x * D0.y + gi.y * D1.y + gi.z * D2.y,
                                  gi.x * D0.z + gi.y * D1.z + gi.z * D2.z);
    const float k = Vlam * jm1;
    acc.f0 -= Vmu * (Dg.x - cp.x) + k * c.x;
    acc.f1 -= Vmu * (Dg.y - cp.y) + k * c.y;
    acc.f2 -= Vmu * (Dg.z - cp.z) + k * c.z;
    const float dg = Vmu * dot(gi, gi);
    acc.h00 += dg + Vlam * c.x * c.x;
    acc.h11 += dg + Vlam * c.y * c.y;
    acc.h22 += dg + Vlam * c.z * c.z;
    acc.h01 += Vlam * c.x * c.y;
    acc.h02 += Vlam * c.x * c.z;
    acc.h12 += Vlam * c.y * c.z;
}

template <bool COH = false>
__device__ __forceinline__ void accumulate_slot(const Dev &d, const SweepParams &p, int s, float2 vm,
                                                int4 r0, float4 r1, float4 r2, float3 ui, Acc &acc) {
    const float4 *__restrict__ u = d.u;
    const float3 da = f3(load_u<COH>(u, r0.x)) - ui;
    const float3 db = f3(load_u<COH>(u, r0.y)) - ui;
    const float3 dc = f3(load_u<COH>(u, r0.z)) - ui;
    const float3 ga = make_float3(__int_as_float(r0.w), r1.x, r1.y);
    const float3 gb = make_float3(r1.z, r1.w, r2.x);
    const float3 gc = make_float3(r2.y, r2.z, r2.w);
    const float2 mat = slot_material(d, p, s, vm, ga, gb, gc);
    tet_contrib(da, db, dc, ga, gb, gc, mat.x, mat.y, acc);
}

// Compact form of a slot (variant 5): only the three neighbour ids of the
// 48-byte record are read (16 bytes with the unused fourth word); the shape
// gradients and the volume are recomputed from the rest positions:
// with rest edges e_k = X_k - X_i, the rows of the inverse rest edge matrix
// are g_a = (e_b x e_c)/det, g_b = (e_c x e_a)/det, g_c = (e_a x e_b)/det,
// det = e_a . (e_b x e_c), V = |det| / 6.  It trades 32 streamed bytes per
// slot for three gathered rest positions and about 40 flops.
template <bool COH = false>
__device__ __forceinline__ void accumulate_slot_rest(const Dev &d, const SweepParams &p, int s, float2 vm,
                                                     int4 r0, float3 ui, float3 Xi, Acc &acc) {
    const float4 *__restrict__ u = d.u;
    const float3 da = f3(load_u<COH>(u, r0.x)) - ui;
    const float3 db = f3(load_u<COH>(u, r0.y)) - ui;
    const float3 dc = f3(load_u<COH>(u, r0.z)) - ui;
    const float3 ea = f3(__ldg(d.rest + r0.x)) - Xi;
    const float3 eb = f3(__ldg(d.rest + r0.y)) - Xi;
    const float3 ec = f3(__ldg(d.rest + r0.z)) - Xi;
    float3 ga = cross(eb, ec), gb = cross(ec, ea), gc = cross(ea, eb);
    const float det = dot(ea, ga);
    const float inv = __frcp_rn(det);
    ga = make_float3(ga.x * inv, ga.y * inv, ga.z * inv);
    gb = make_float3(gb.x * inv, gb.y * inv, gb.z * inv);
    gc = make_float3(gc.x * inv, gc.y * inv, gc.z * inv);
    const float V = fabsf(det) * (1.0f / 6.0f);
    if (p.per_tet_mat) {
        const int j = __ldcs(d.slot_tet + s);
        vm = make_float2(__ldg(d.tet_mu + j), __ldg(d.tet_lam + j));
    }
    tet_contrib(da, db, dc, ga, gb, gc, V * vm.x, V * vm.y, acc);
}

// ---- two slots per lane in packed FP32 (variant 6) -------------------------
// sm_100+ issues FP32 add, multiply and fused multiply-add on register pairs
// (one instruction, two IEEE single-precision results, each rounded as the
// scalar operation would be).  The element arithmetic is the same for every
// slot, so a lane evaluates two of its slots at once: the x half of each pair
// belongs to slot s, the y half to slot s + L.  This halves the FP32
// instructions of the compact-slot pass (about three quarters of its
// instructions) and keeps the two slots' gathers in flight together.
__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a b - c
__device__ __forceinline__ float2 fms2(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, make_float2(-c.x, -c.y));
}

struct V2 {
    float2 x, y, z;
};
__device__ __forceinline__ V2 cross2(const V2 &a, const V2 &b) {
    return {fms2(a.y, b.z, mul2(a.z, b.y)), fms2(a.z, b.x, mul2(a.x, b.z)), fms2(a.x, b.y, mul2(a.y, b.x))};
}
__device__ __forceinline__ float2 dot2(const V2 &a, const V2 &b) {
    return fma2(a.x, b.x, fma2(a.y, b.y, mul2(a.z, b.z)));
}
// (positions of slot a) - (a position common to both), per component
__device__ __forceinline__ V2 diff2(float4 a, float4 b, float3 o) {
    return {sub2(p2(a.x, b.x), bc2(o.x)), sub2(p2(a.y, b.y), bc2(o.y)), sub2(p2(a.z, b.z), bc2(o.z))};
}

struct Acc2 {
    float2 f0, f1, f2, h00, h01, h02, h11, h12, h22;
};

// tet_contrib for two slots, with sg = g_a + g_b + g_c = -g_i so that no
// result needs a separate negation:
//   D = sum_k d_k g_k^T,  J - 1 = tr D + tr cof(D) + det D,
//   cq = (tr D) sg - D^T sg + cof(D) sg = -(cof(F) g_i - g_i),
//   cn = sg + cq = -cof(F) g_i,  Dsg = D sg = -D g_i,
//   f_i += V mu (Dsg - cq) + V lam (J - 1) cn,
//   H_i += V mu |sg|^2 I + V lam cn cn^T.
__device__ __forceinline__ void tet_contrib2(const V2 &da, const V2 &db, const V2 &dc, const V2 &ga,
                                             const V2 &gb, const V2 &gc, float2 Vmu, float2 Vlam, Acc2 &acc) {
    const V2 sg = {add2(add2(ga.x, gb.x), gc.x), add2(add2(ga.y, gb.y), gc.y), add2(add2(ga.z, gb.z), gc.z)};
    const V2 D0 = {fma2(da.x, ga.x, fma2(db.x, gb.x, mul2(dc.x, gc.x))),
                   fma2(da.y, ga.x, fma2(db.y, gb.x, mul2(dc.y, gc.x))),
                   fma2(da.z, ga.x, fma2(db.z, gb.x, mul2(dc.z, gc.x)))};
    const V2 D1 = {fma2(da.x, ga.y, fma2(db.x, gb.y, mul2(dc.x, gc.y))),
                   fma2(da.y, ga.y, fma2(db.y, gb.y, mul2(dc.y, gc.y))),
                   fma2(da.z, ga.y, fma2(db.z, gb.y, mul2(dc.z, gc.y)))};
    const V2 D2 = {fma2(da.x, ga.z, fma2(db.x, gb.z, mul2(dc.x, gc.z))),
                   fma2(da.y, ga.z, fma2(db.y, gb.z, mul2(dc.y, gc.z))),
                   fma2(da.z, ga.z, fma2(db.z, gb.z, mul2(dc.z, gc.z)))};
    const float2 tr = add2(add2(D0.x, D1.y), D2.z);
    const V2 q0 = cross2(D1, D2), q1 = cross2(D2, D0), q2 = cross2(D0, D1);  // columns of cof(D)
    const float2 jm1 = add2(add2(tr, add2(add2(q0.x, q1.y), q2.z)), dot2(D0, q0));
    const V2 cq = {fma2(tr, sg.x, fma2(sg.x, q0.x, fma2(sg.y, q1.x, fms2(sg.z, q2.x, dot2(D0, sg))))),
                   fma2(tr, sg.y, fma2(sg.x, q0.y, fma2(sg.y, q1.y, fms2(sg.z, q2.y, dot2(D1, sg))))),
                   fma2(tr, sg.z, fma2(sg.x, q0.z, fma2(sg.y, q1.z, fms2(sg.z, q2.z, dot2(D2, sg)))))};
    const V2 cn = {add2(sg.x, cq.x), add2(sg.y, cq.y), add2(sg.z, cq.z)};
    const V2 Dsg = {fma2(sg.x, D0.x, fma2(sg.y, D1.x, mul2(sg.z, D2.x))),
                    fma2(sg.x, D0.y, fma2(sg.y, D1.y, mul2(sg.z, D2.y))),
                    fma2(sg.x, D0.z, fma2(sg.y, D1.z, mul2(sg.z, D2.z)))};
    const float2 k = mul2(Vlam, jm1);
    acc.f0 = fma2(Vmu, sub2(Dsg.x, cq.x), fma2(k, cn.x, acc.f0));
    acc.f1 = fma2(Vmu, sub2(Dsg.y, cq.y), fma2(k, cn.y, acc.f1));
    acc.f2 = fma2(Vmu, sub2(Dsg.z, cq.z), fma2(k, cn.z, acc.f2));
    const float2 dg = mul2(Vmu, dot2(sg, sg));
    const V2 vc = {mul2(Vlam, cn.x), mul2(Vlam, cn.y), mul2(Vlam, cn.z)};
    acc.h00 = add2(acc.h00, fma2(vc.x, cn.x, dg));
    acc.h11 = add2(acc.h11, fma2(vc.y, cn.y, dg));
    acc.h22 = add2(acc.h22, fma2(vc.z, cn.z, dg));
    acc.h01 = fma2(vc.x, cn.y, acc.h01);
    acc.h02 = fma2(vc.x, cn.z, acc.h02);
    acc.h12 = fma2(vc.y, cn.z, acc.h12);
}

// Compact slots s (x half) and s + L (y half, or a repeat of s with zero
// weight when the lane has an odd number of slots): shape gradients and
// volume from the FP32 rest positions, as in accumulate_slot_rest.
__device__ __forceinline__ void accumulate_pair_rest(const Dev &d, const SweepParams &p, int sa, int sb, bool hasb,
                                                     float2 vm, int4 ra, int4 rb, float3 ui, float3 Xi,
                                                     Acc2 &acc) {
    const float4 *__restrict__ u = d.u;
    const float4 *__restrict__ X = d.rest;
    const float4 ua0 = __ldg(u + ra.x), ua1 = __ldg(u + ra.y), ua2 = __ldg(u + ra.z);
    const float4 ub0 = __ldg(u + rb.x), ub1 = __ldg(u + rb.y), ub2 = __ldg(u + rb.z);
    const float4 Xa0 = __ldg(X + ra.x), Xa1 = __ldg(X + ra.y), Xa2 = __ldg(X + ra.z);
    const float4 Xb0 = __ldg(X + rb.x), Xb1 = __ldg(X + rb.y), Xb2 = __ldg(X + rb.z);
    float2 mu2 = bc2(vm.x), lam2 = bc2(vm.y);
    if (p.per_tet_mat) {
        const int ja = __ldcs(d.slot_tet + sa), jb = hasb ? __ldcs(d.slot_tet + sb) : ja;
        mu2 = p2(__ldg(d.tet_mu + ja), __ldg(d.tet_mu + jb));
        lam2 = p2(__ldg(d.tet_lam + ja), __ldg(d.tet_lam + jb));
    }
    const V2 da = diff2(ua0, ub0, ui), db = diff2(ua1, ub1, ui), dc = diff2(ua2, ub2, ui);
    const V2 ea = diff2(Xa0, Xb0, Xi), eb = diff2(Xa1, Xb1, Xi), ec = diff2(Xa2, Xb2, Xi);
    V2 ga = cross2(eb, ec), gb = cross2(ec, ea), gc = cross2(ea, eb);
    const float2 det = dot2(ea, ga);
    const float2 inv = p2(__frcp_rn(det.x), __frcp_rn(det.y));
    ga = {mul2(ga.x, inv), mul2(ga.y, inv), mul2(ga.z, inv)};
    gb = {mul2(gb.x, inv), mul2(gb.y, inv), mul2(gb.z, inv)};
    gc = {mul2(gc.x, inv), mul2(gc.y, inv), mul2(gc.z, inv)};
    // V = |det| / 6; the repeated slot of an odd count weighs nothing
    const float2 V = mul2(p2(fabsf(det.x), hasb ? fabsf(det.y) : 0.f), bc2(1.0f / 6.0f));
    tet_contrib2(da, db, dc, ga, gb, gc, mul2(V, mu2), mul2(V, lam2), acc);
}

// Edge-edge pair item j = 4 (holding edge) + role (Sec. 3.5): with the
// contact points x_a = (1 - s) p0 + s p1, x_b = (1 - u) q0 + u q1 and the
// frozen normal n, d = (x_b - x_a).n = sum_v c_v x_v . n with
// c = (-(1 - s), -s, 1 - u, u); for d > 0 the vertex of role r gets
// -k_c d c_r n and k_c c_r^2 n n^T (Eq. 12, n held constant).
__device__ __forceinline__ bool ee_item(const Dev &d, const SweepParams &p, int vi, int j, Acc &c) {
    const int e = j >> 2, r = j & 3;
    const int f = d.ee_partner[e];
    if (f < 0) return false;
    const int4 ev = d.edge_v[e], fv = d.edge_v[f];
    const float4 prm = d.ee_prm[e], nv = d.ee_nrm[e];
    const float cw[4] = {-(1.f - prm.x), -prm.x, 1.f - prm.y, prm.y};
    const int vid[4] = {ev.x, ev.y, fv.x, fv.y};
    // the weights sum to zero, so positions are taken relative to vertex vi
    const float3 Xi = f3(__ldg(d.rest + vi)), ui = f3(__ldg(d.u + vi));
    float dep = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float3 q = (f3(__ldg(d.rest + vid[k])) - Xi) + (f3(__ldg(d.u + vid[k])) - ui);
        dep += cw[k] * (q.x * nv.x + q.y * nv.y + q.z * nv.z);
    }
    if (!(dep > 0.f)) return false;
    const float cr = r == 0 ? cw[0] : (r == 1 ? cw[1] : (r == 2 ? cw[2] : cw[3]));
    const float fs = -p.kc * dep * cr, hs = p.kc * cr * cr;
    c.f0 += fs * nv.x; c.f1 += fs * nv.y; c.f2 += fs * nv.z;
    c.h00 += hs * nv.x * nv.x; c.h01 += hs * nv.x * nv.y; c.h02 += hs * nv.x * nv.z;
    c.h11 += hs * nv.y * nv.y; c.h12 += hs * nv.y * nv.z; c.h22 += hs * nv.z * nv.z;
    return true;
}

template <int L>
__device__ __forceinline__ float sub_reduce(float v) {
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// Vertex-triangle contact forces on vertex vi (Sec. 3.5, penalty of Eq. 12).
// Its items are its own pair (if any) and the pairs in which it is a
// triangle corner (d.rev, ascending).  As the vertex of its own pair it gets
// k_c d n and k_c n n^T; as corner k of another vertex's triangle, -k_c d
// w_k n and k_c w_k^2 n n^T; only pairs with d > 0 act.  The L lanes of the
// vertex take the items in turn and their sums are reduced like the slots.
// Positions come from d.u: a vertex in any pair ("involved") writes its
// update to d.unew, copied back after the pass, so that d.u keeps the
// pass-start positions its partners read (x^new of Algorithm 1); partners
// of an involved vertex are involved too, and other vertices of the colour
// touch only other colours, so they update in place.
// With ground friction on (mu_c > 0) the pairs get friction too (Sec. 3.6):
// the contact points moved by delta = (x_a - x_a^t) - sum_k w_k (x_k - x_k^t)
// since the step start (displacements: the rest positions cancel), u is its
// part tangent to n, and with the pair's normal force k_c d a vertex whose
// delta derivative is s I (1 for the pair's vertex, -w_k for corner k) gets
// -s c u and s^2 c (I - n n^T), c = mu_c k_c d f1(|u|)/|u| (Eq. 15).
__device__ __forceinline__ bool contact_item(const Dev &d, const SweepParams &p, int vi, int own, int item, int r0,
                                             Acc &c) {
    const float kc = p.kc;
    int a, k = -1;
    int4 t;
    if (item == 0 && own >= 0) {
        a = vi;
        t = d.tri[own];
    } else {
        a = d.rev[r0 + item - (own >= 0 ? 1 : 0)];
        t = d.tri[d.contact[a]];
        k = (t.x == vi) ? 0 : ((t.y == vi) ? 1 : 2);
    }
    float3 n, w;
    const float dep = geom::pair_depth(d, a, t, n, w);
    if (!(dep > 0.0f)) return false;
    // s = 1 for the pair's vertex, -w_k for corner k: the penalty force is
    // k_c d s n and its Hessian s^2 k_c n n^T (d decreases along n at the vertex)
    const float sgn = k < 0 ? 1.0f : -(k == 0 ? w.x : (k == 1 ? w.y : w.z));
    const float fs = sgn * kc * dep, hs = sgn * sgn * kc;
    c.f0 += fs * n.x; c.f1 += fs * n.y; c.f2 += fs * n.z;
    c.h00 += hs * n.x * n.x; c.h01 += hs * n.x * n.y; c.h02 += hs * n.x * n.z;
    c.h11 += hs * n.y * n.y; c.h12 += hs * n.y * n.z; c.h22 += hs * n.z * n.z;
    if (p.mu_c > 0.0f) {
        const float3 da = f3(__ldg(d.u + a)) - f3(__ldg(d.ut + a));
        const float3 d0 = f3(__ldg(d.u + t.x)) - f3(__ldg(d.ut + t.x));
        const float3 d1 = f3(__ldg(d.u + t.y)) - f3(__ldg(d.ut + t.y));
        const float3 d2 = f3(__ldg(d.u + t.z)) - f3(__ldg(d.ut + t.z));
        float3 dl = make_float3(da.x - (w.x * d0.x + w.y * d1.x + w.z * d2.x),
                                da.y - (w.x * d0.y + w.y * d1.y + w.z * d2.y),
                                da.z - (w.x * d0.z + w.y * d1.z + w.z * d2.z));
        const float dn = dot(dl, n);
        dl = make_float3(dl.x - dn * n.x, dl.y - dn * n.y, dl.z - dn * n.z);
        const float um = sqrtf(dot(dl, dl));
        const float f1u = um < p.eps_h ? (2.0f / p.eps_h - um / (p.eps_h * p.eps_h)) : 1.0f / um;
        const float cf = p.mu_c * kc * dep * f1u;
        const float ff = -sgn * cf, hf = sgn * sgn * cf;
        c.f0 += ff * dl.x; c.f1 += ff * dl.y; c.f2 += ff * dl.z;
        c.h00 += hf * (1.f - n.x * n.x); c.h11 += hf * (1.f - n.y * n.y); c.h22 += hf * (1.f - n.z * n.z);
        c.h01 -= hf * n.x * n.y; c.h02 -= hf * n.x * n.z; c.h12 -= hf * n.y * n.z;
    }
    return true;
}

// Local solve of Sec. 3.2 for one vertex: Eq. 7 with the inertia terms of
// Eqs. 8-9, damping (Eqs. 10-11), ground and wall penalties (Eq. 12,
// Sec. 3.4), self-contact, singular skip, analytic inverse.
// sc: self-contact sums (f, H) and bit 0 = some pair acted, bit 1 = involved.
// EXT = false compiles the optional parts out (the register-capped sweeps
// keep their operands live otherwise): the line search and the subspace
// step; EXT = true runs them when p.line_search / p.n_sub ask for them.
template <bool SC, bool EXT = true>
__device__ __forceinline__ void solve_and_store(const Dev &d, const SweepParams &p, int vi, float4 xi,
                                                const Acc &a, const Acc &ca, int sc) {
    // xi holds the displacement u_i; ym the displacement of the inertia target
    const float4 yv = d.ym[vi];
    const float mh2 = yv.w;
    const float kdh = p.kd_over_h;
    // variational part (inertia + elasticity), kept for the line search
    const float fv0 = mh2 * (yv.x - xi.x) + a.f0;
    const float fv1 = mh2 * (yv.y - xi.y) + a.f1;
    const float fv2 = mh2 * (yv.z - xi.z) + a.f2;
    float f0 = fv0, f1 = fv1, f2 = fv2;
    const float s = 1.0f + kdh;
    float h00 = s * a.h00 + mh2, h11 = s * a.h11 + mh2, h22 = s * a.h22 + mh2;
    float h01 = s * a.h01, h02 = s * a.h02, h12 = s * a.h12;
    if (kdh != 0.0f) {
        const float4 xt = d.ut[vi];
        const float dx = xi.x - xt.x, dy = xi.y - xt.y, dz = xi.z - xt.z;
        f0 -= kdh * (a.h00 * dx + a.h01 * dy + a.h02 * dz);
        f1 -= kdh * (a.h01 * dx + a.h11 * dy + a.h12 * dz);
        f2 -= kdh * (a.h02 * dx + a.h12 * dy + a.h22 * dz);
    }
    float flag = xi.w;
    // self-contact sums first, so that they are dead before the plane loop
    bool stage = p.to_unew != 0;  // write to d.unew (copied back after the pass)
    if (SC && (sc & 2)) {
        f0 += ca.f0; f1 += ca.f1; f2 += ca.f2;
        h00 += ca.h00; h01 += ca.h01; h02 += ca.h02; h11 += ca.h11; h12 += ca.h12; h22 += ca.h22;
        if (sc & 1) flag = 1.0f;
        stage = true;
    }
    // ground and walls (Sec. 3.4): penalty of Eq. 12 per static half-space,
    // at the position P = X + u
    float3 P = make_float3(0.f, 0.f, 0.f);
    if (p.n_planes > 0) {
        const float4 X = d.rest[vi];
        P = make_float3(X.x + xi.x, X.y + xi.y, X.z + xi.z);
    }
    // unrolled: constant plane indices keep the plane data in the constant bank
#pragma unroll
    for (int k = 0; k < kMaxPlanes; ++k) {
        if (k >= p.n_planes) break;
        const float4 pl = p.planes[k];
        const float pen = pl.w - (pl.x * P.x + pl.y * P.y + pl.z * P.z);
        if (pen > 0.0f) {
            const float kd = p.kc * pen;
            f0 += kd * pl.x; f1 += kd * pl.y; f2 += kd * pl.z;
            h00 += p.kc * pl.x * pl.x; h11 += p.kc * pl.y * pl.y; h22 += p.kc * pl.z * pl.z;
            h01 += p.kc * pl.x * pl.y; h02 += p.kc * pl.x * pl.z; h12 += p.kc * pl.y * pl.z;
            flag = 1.0f;
            if (p.mu_c > 0.0f) {
                // friction (Eqs. 13-16) on a static plane: sliding displacement
                // u = tangential part of x_i - x_i^t, normal-force magnitude kd
                const float4 ut = d.ut[vi];
                float dx = xi.x - ut.x, dy = xi.y - ut.y, dz = xi.z - ut.z;
                const float dn = dx * pl.x + dy * pl.y + dz * pl.z;
                dx -= dn * pl.x; dy -= dn * pl.y; dz -= dn * pl.z;
                const float um = sqrtf(dx * dx + dy * dy + dz * dz);
                const float f1u = um < p.eps_h ? (2.0f / p.eps_h - um / (p.eps_h * p.eps_h)) : 1.0f / um;
                const float c = p.mu_c * kd * f1u;
                f0 -= c * dx; f1 -= c * dy; f2 -= c * dz;
                h00 += c * (1.f - pl.x * pl.x); h11 += c * (1.f - pl.y * pl.y); h22 += c * (1.f - pl.z * pl.z);
                h01 -= c * pl.x * pl.y; h02 -= c * pl.x * pl.z; h12 -= c * pl.y * pl.z;
            }
        }
    }
    float4 *out = stage ? d.unew : d.u;
    float dx, dy, dz;
    const int sub = (EXT && p.n_sub > 0) ? d.sub_id[vi] : -1;
    if (sub >= 0) {
        // subspace constraint (Sec. 3.4): Q^T H Q dz = Q^T f in the basis q_1
        // (.w = L) and q_2 of the line or plane, dx = Q dz, with the singular
        // test of Sec. 3.2 on the L x L matrix
        const float4 qa = d.sub_q[2 * sub], qb = d.sub_q[2 * sub + 1];
        const float ha0 = h00 * qa.x + h01 * qa.y + h02 * qa.z;
        const float ha1 = h01 * qa.x + h11 * qa.y + h12 * qa.z;
        const float ha2 = h02 * qa.x + h12 * qa.y + h22 * qa.z;
        const float A00 = qa.x * ha0 + qa.y * ha1 + qa.z * ha2;
        const float b0 = qa.x * f0 + qa.y * f1 + qa.z * f2;
        bool singular;
        float z0, z1 = 0.f;
        if (qa.w < 1.5f) {
            singular = !(fabsf(A00) > p.det_eps * fabsf(A00));
            z0 = b0 / A00;
        } else {
            const float A01 = qb.x * ha0 + qb.y * ha1 + qb.z * ha2;
            const float A11 = qb.x * (h00 * qb.x + h01 * qb.y + h02 * qb.z) +
                              qb.y * (h01 * qb.x + h11 * qb.y + h12 * qb.z) +
                              qb.z * (h02 * qb.x + h12 * qb.y + h22 * qb.z);
            const float b1 = qb.x * f0 + qb.y * f1 + qb.z * f2;
            const float det2 = A00 * A11 - A01 * A01;
            const float tr2 = 0.5f * (A00 + A11);
            singular = !(fabsf(det2) > p.det_eps * tr2 * tr2);
            const float inv2 = 1.0f / det2;
            z0 = (A11 * b0 - A01 * b1) * inv2;
            z1 = (A00 * b1 - A01 * b0) * inv2;
        }
        if (singular) {
            atomicAdd(d.counters + 1, 1ull);
            if (stage || flag != xi.w) out[vi] = make_float4(xi.x, xi.y, xi.z, flag);
            return;
        }
        dx = qa.x * z0 + qb.x * z1;
        dy = qa.y * z0 + qb.y * z1;
        dz = qa.z * z0 + qb.z * z1;
    } else {
        // adjugate of the symmetric H
        const float a00 = h11 * h22 - h12 * h12;
        const float a01 = h02 * h12 - h01 * h22;
        const float a02 = h01 * h12 - h02 * h11;
        const float a11 = h00 * h22 - h02 * h02;
        const float a12 = h01 * h02 - h00 * h12;
        const float a22 = h00 * h11 - h01 * h01;
        const float det = h00 * a00 + h01 * a01 + h02 * a02;
        const float tr3 = (h00 + h11 + h22) * (1.0f / 3.0f);
        if (!(fabsf(det) > p.det_eps * fabsf(tr3 * tr3 * tr3))) {
            atomicAdd(d.counters + 1, 1ull);
            if (stage || flag != xi.w) out[vi] = make_float4(xi.x, xi.y, xi.z, flag);
            return;
        }
        const float inv = 1.0f / det;
        dx = (a00 * f0 + a01 * f1 + a02 * f2) * inv;
        dy = (a01 * f0 + a11 * f1 + a12 * f2) * inv;
        dz = (a02 * f0 + a12 * f1 + a22 * f2) * inv;
    }
    if (!(isfinite(dx) && isfinite(dy) && isfinite(dz))) {
        atomicAdd(d.counters + 0, 1ull);
        if (stage) out[vi] = xi;
        return;
    }
    if (EXT && p.line_search) {
        // G_i along dx: inertia + elasticity are exactly quadratic in x_i, so
        // G_i(x + alpha dx) - G_i(x) = -alpha fv.dx + alpha^2/2 dx.Hv.dx + the
        // change of the plane penalties, with fv, Hv the variational force and
        // Hessian.
        const float q1 = fv0 * dx + fv1 * dy + fv2 * dz;
        const float hx = (a.h00 + mh2) * dx + a.h01 * dy + a.h02 * dz;
        const float hy = a.h01 * dx + (a.h11 + mh2) * dy + a.h12 * dz;
        const float hz = a.h02 * dx + a.h12 * dy + (a.h22 + mh2) * dz;
        const float q2 = dx * hx + dy * hy + dz * hz;
        float alpha = 1.0f;
        bool ok = false;
        for (int k = 0; k < 8; ++k) {
            float dG = alpha * (0.5f * alpha * q2 - q1);
#pragma unroll
            for (int j = 0; j < kMaxPlanes; ++j) {
                if (j >= p.n_planes) break;
                const float4 pl = p.planes[j];
                const float pen = pl.w - (pl.x * P.x + pl.y * P.y + pl.z * P.z);
                const float p0 = fmaxf(pen, 0.0f);
                const float pa = fmaxf(pen - alpha * (pl.x * dx + pl.y * dy + pl.z * dz), 0.0f);
                dG += 0.5f * p.kc * (pa - p0) * (pa + p0);
            }
            if (dG <= 0.0f) {
                ok = true;
                break;
            }
            alpha *= 0.5f;
        }
        if (!ok) alpha = 0.0f;
        dx *= alpha;
        dy *= alpha;
        dz *= alpha;
    }
    out[vi] = make_float4(xi.x + dx, xi.y + dy, xi.z + dz, flag);
}

// One colour pass for the vertex of global thread gt (L lanes per vertex).
// RS: compact slots, shape gradients recomputed from the rest positions.
template <int L, bool SC, bool COH = false, bool EXT = true, bool RS = false>
__device__ __forceinline__ void sweep_body(const Dev &d, const SweepParams &p, long long gt,
                                           int vbegin, int vend) {
    const int lane = threadIdx.x & (L - 1);
    const int vi = vbegin + (int)(gt / L);
    const bool active = vi < vend;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    int s0 = 0, s1 = 0;
    if (active) {
        xi = COH ? __ldcg(d.u + vi) : d.u[vi];
        s0 = d.slot_off[vi];
        s1 = d.slot_off[vi + 1];
    }
    const float3 x3 = f3(xi);
    const float2 vm = (active && !p.per_tet_mat) ? __ldg(d.vmat + vi) : make_float2(0.f, 0.f);
    Acc acc = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (RS) {
        const float3 X3 = active ? f3(__ldg(d.rest + vi)) : make_float3(0.f, 0.f, 0.f);
        for (int s = s0 + lane; s < s1; s += L)
            accumulate_slot_rest<COH>(d, p, s, vm, __ldcs(d.s0 + s), x3, X3, acc);
    } else {
        for (int s = s0 + lane; s < s1; s += L)
            accumulate_slot<COH>(d, p, s, vm, __ldcs(d.s0 + s), __ldcs(d.s1 + s), __ldcs(d.s2 + s), x3, acc);
    }
    acc.f0 = sub_reduce<L>(acc.f0);
    acc.f1 = sub_reduce<L>(acc.f1);
    acc.f2 = sub_reduce<L>(acc.f2);
    acc.h00 = sub_reduce<L>(acc.h00);
    acc.h01 = sub_reduce<L>(acc.h01);
    acc.h02 = sub_reduce<L>(acc.h02);
    acc.h11 = sub_reduce<L>(acc.h11);
    acc.h12 = sub_reduce<L>(acc.h12);
    acc.h22 = sub_reduce<L>(acc.h22);
    Acc ca = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int sc = 0;
    if (SC) {
        int own = -1, r0 = 0, n_vt = 0, e0 = 0, n_items = 0;
        if (active) {
            own = d.contact[vi];
            r0 = d.rev_off[vi];
            n_vt = (own >= 0 ? 1 : 0) + (d.rev_off[vi + 1] - r0);
            n_items = n_vt;
            if (p.ee_on) {
                e0 = d.ee_off[vi];
                n_items += d.ee_off[vi + 1] - e0;
            }
        }
        int hit = 0;
        for (int it = lane; it < n_items; it += L)
            hit |= (it < n_vt ? contact_item(d, p, vi, own, it, r0, ca)
                              : ee_item(d, p, vi, d.ee_item[e0 + it - n_vt], ca)) ? 1 : 0;
        if (__any_sync(FULL, n_items > 0)) {
            ca.f0 = sub_reduce<L>(ca.f0);
            ca.f1 = sub_reduce<L>(ca.f1);
            ca.f2 = sub_reduce<L>(ca.f2);
            ca.h00 = sub_reduce<L>(ca.h00);
            ca.h01 = sub_reduce<L>(ca.h01);
            ca.h02 = sub_reduce<L>(ca.h02);
            ca.h11 = sub_reduce<L>(ca.h11);
            ca.h12 = sub_reduce<L>(ca.h12);
            ca.h22 = sub_reduce<L>(ca.h22);
#pragma unroll
            for (int off = L / 2; off > 0; off >>= 1) hit |= __shfl_xor_sync(FULL, hit, off);
        }
        sc = (n_items > 0 ? 2 : 0) | hit;
    }
    if (active && lane == 0) solve_and_store<SC, EXT>(d, p, vi, xi, acc, ca, sc);
}

// Variant 6: the compact-slot pass with two slots per lane in packed FP32
// (accumulate_pair_rest); the solve is the one of sweep_body.
template <int L, bool EXT>
__device__ __forceinline__ void sweep_body_pair(const Dev &d, const SweepParams &p, long long gt, int vbegin,
                                                int vend) {
    const int lane = threadIdx.x & (L - 1);
    const int vi = vbegin + (int)(gt / L);
    const bool active = vi < vend;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    int s0 = 0, s1 = 0;
    if (active) {
        xi = d.u[vi];
        s0 = d.slot_off[vi];
        s1 = d.slot_off[vi + 1];
    }
    const float3 x3 = f3(xi);
    const float3 X3 = active ? f3(__ldg(d.rest + vi)) : make_float3(0.f, 0.f, 0.f);
    const float2 vm = (active && !p.per_tet_mat) ? __ldg(d.vmat + vi) : make_float2(0.f, 0.f);
    Acc2 a2;
    a2.f0 = a2.f1 = a2.f2 = a2.h00 = a2.h01 = a2.h02 = a2.h11 = a2.h12 = a2.h22 = make_float2(0.f, 0.f);
    for (int s = s0 + lane; s < s1; s += 2 * L) {
        const int sb = s + L;
        const bool hasb = sb < s1;
        const int4 ra = __ldcs(d.s0 + s);
        const int4 rb = hasb ? __ldcs(d.s0 + sb) : ra;
        accumulate_pair_rest(d, p, s, sb, hasb, vm, ra, rb, x3, X3, a2);
    }
    Acc acc = {a2.f0.x + a2.f0.y, a2.f1.x + a2.f1.y, a2.f2.x + a2.f2.y, a2.h00.x + a2.h00.y,
               a2.h01.x + a2.h01.y, a2.h02.x + a2.h02.y, a2.h11.x + a2.h11.y, a2.h12.x + a2.h12.y,
               a2.h22.x + a2.h22.y};
    acc.f0 = sub_reduce<L>(acc.f0);
    acc.f1 = sub_reduce<L>(acc.f1);
    acc.f2 = sub_reduce<L>(acc.f2);
    acc.h00 = sub_reduce<L>(acc.h00);
    acc.h01 = sub_reduce<L>(acc.h01);
    acc.h02 = sub_reduce<L>(acc.h02);
    acc.h11 = sub_reduce<L>(acc.h11);
    acc.h12 = sub_reduce<L>(acc.h12);
    acc.h22 = sub_reduce<L>(acc.h22);
    if (active && lane == 0) solve_and_store<false, EXT>(d, p, vi, xi, acc, acc, 0);
}

// Both gather kernels are held to 48 registers (5 CTAs of 256 threads per
// SM, no spills without the line search): 40 resident warps hide the gather
// latency better than 32 at 56 registers (measured 62.1 vs 64.0 us per
// 1M-vertex pass).  EXT: instance with the line search (Sec. 3.2) and the
// subspace step (Sec. 3.4) compiled in.
template <int L, bool EXT>
__global__ void __launch_bounds__(256, 5) k_sweep(Dev d, SweepParams p) {
    sweep_body<L, false, false, EXT>(d, p, (long long)blockIdx.x * blockDim.x + threadIdx.x, p.vbegin, p.vend);
}

// persistent form: a grid of (SMs x resident CTAs) walks the colour's
// vertices in grid-sized strides (the stride is uniform over a warp, so
// every lane joins the shuffles of each round)
template <int L, bool EXT>
__global__ void __launch_bounds__(256, 5) k_sweep_persist(Dev d, SweepParams p, long long threads) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < threads; base += stride)
        sweep_body<L, false, false, EXT>(d, p, base + threadIdx.x, p.vbegin, p.vend);
}

// persistent form over compact slots (gradients from the rest positions)
template <int L, bool EXT>
__global__ void __launch_bounds__(256, 4) k_sweep_rest(Dev d, SweepParams p, long long threads) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < threads; base += stride)
        sweep_body<L, false, false, EXT, true>(d, p, base + threadIdx.x, p.vbegin, p.vend);
}

// persistent form of the packed two-slot compact pass (variant 6)
#ifndef VBD_PAIR_MIN_BLOCKS
#define VBD_PAIR_MIN_BLOCKS 3
#endif
template <int L, bool EXT>
__global__ void __launch_bounds__(256, VBD_PAIR_MIN_BLOCKS) k_sweep_pair(Dev d, SweepParams p, long long threads) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < threads; base += stride)
        sweep_body_pair<L, EXT>(d, p, base + threadIdx.x, p.vbegin, p.vend);
}

// with self-contact forces; capped at 64 registers so that enough warps stay
// resident to hide the gather latency (EXT: with the subspace step)
template <int L, bool EXT>
__global__ void __launch_bounds__(256, 4) k_sweep_sc(Dev d, SweepParams p) {
    sweep_body<L, true, false, EXT>(d, p, (long long)blockIdx.x * blockDim.x + threadIdx.x, p.vbegin, p.vend);
}

// ---- two-phase tet-scatter-into-slots sweep ----------------------------------
// Phase 1: one thread per incidence slot of the colour computes that tet's
// force and Hessian block on the slot's vertex (the same arithmetic as
// accumulate_slot) and writes the 9 sums to the slot's place in a scratch
// buffer.  Phase 2: L lanes per vertex add up the vertex's scratch entries
// (in slot order, xor-reduced like k_sweep) and solve.  It moves 36 bytes
// more per slot twice (write and read back) than the gather, which is why the
// gather is the default; it exists to measure that choice.
__global__ void __launch_bounds__(256) k_scatter_slots(Dev d, SweepParams p, int sbegin, int nslots) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nslots) return;
    const int s = sbegin + t;
    const int vi = __ldcs(d.slot_vtx + s);
    const float3 x3 = f3(__ldg(d.u + vi));
    const float2 vm = p.per_tet_mat ? make_float2(0.f, 0.f) : __ldg(d.vmat + vi);
    Acc acc = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    accumulate_slot(d, p, s, vm, __ldcs(d.s0 + s), __ldcs(d.s1 + s), __ldcs(d.s2 + s), x3, acc);
    __stcs(d.scr0 + t, make_float4(acc.f0, acc.f1, acc.f2, acc.h00));
    __stcs(d.scr1 + t, make_float4(acc.h01, acc.h02, acc.h11, acc.h12));
    __stcs(d.scr2 + t, acc.h22);
}

template <int L>
__global__ void __launch_bounds__(256) k_scatter_reduce(Dev d, SweepParams p, int sbegin) {
    const int lane = threadIdx.x & (L - 1);
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int vi = p.vbegin + (int)(gt / L);
    const bool active = vi < p.vend;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    int s0 = 0, s1 = 0;
    if (active) {
        xi = d.u[vi];
        s0 = d.slot_off[vi] - sbegin;
        s1 = d.slot_off[vi + 1] - sbegin;
    }
    Acc acc = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = s0 + lane; k < s1; k += L) {
        const float4 a = __ldcs(d.scr0 + k), b = __ldcs(d.scr1 + k);
        acc.f0 += a.x; acc.f1 += a.y; acc.f2 += a.z; acc.h00 += a.w;
        acc.h01 += b.x; acc.h02 += b.y; acc.h11 += b.z; acc.h12 += b.w;
        acc.h22 += __ldcs(d.scr2 + k);
    }
    acc.f0 = sub_reduce<L>(acc.f0);
    acc.f1 = sub_reduce<L>(acc.f1);
    acc.f2 = sub_reduce<L>(acc.f2);
    acc.h00 = sub_reduce<L>(acc.h00);
    acc.h01 = sub_reduce<L>(acc.h01);
    acc.h02 = sub_reduce<L>(acc.h02);
    acc.h11 = sub_reduce<L>(acc.h11);
    acc.h12 = sub_reduce<L>(acc.h12);
    acc.h22 = sub_reduce<L>(acc.h22);
    if (active && lane == 0) solve_and_store<false>(d, p, vi, xi, acc, acc, 0);
}

// ---- pipelined sweep: slot records staged in shared memory by TMA ----------
// Persistent CTAs of TT threads walk the colour range in chunks of TT / 8
// consecutive vertices (8 lanes per vertex as in k_sweep).  A chunk's slot
// records are contiguous, so one thread copies them global -> shared with
// three bulk copies (cp.async.bulk, completion counted in bytes on an
// mbarrier), two chunks ahead of the consumers.  The stream is then in flight
// without occupying registers, which is what limits k_sweep.  Every wait is
// bounded: on time-out the CTA records an error (counters[2]), waits (again
// bounded) on the barriers of every chunk it has issued and returns; the host
// reports it.  Each stage barrier expects exactly the bytes of the copies
// issued to it, so that drain returns as soon as those copies have landed.
// Only if a copy itself never completes (a fault of the copy engine, which
// nothing here provokes) does the drain give up too, and the CTA then exits
// with that copy outstanding.  The time-out test hook therefore does not
// touch the stage barriers: it makes the first chunk also wait on a spare
// barrier that nothing ever arrives at.
constexpr int kPipeLanes = 8;
constexpr int kPipeStages = 2;
constexpr long long kWaitSpins = 1ll << 22;        // try_wait calls before giving up
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s of SM clock

struct StageMeta {
    int a;       // first slot of the chunk
    int n;       // slot count
    int pad;
    int direct;  // 1: consumers read global memory (chunk larger than a stage, or empty)
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    const unsigned a = smem_addr(bar);
    const long long t0 = clock64();
    for (long long i = 0; i < kWaitSpins; ++i) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok) : "r"(a), "r"(parity) : "memory");
        if (ok) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// shared-memory image of one stage (maxs slots)
struct StageView {
    int4 *s0;
    float4 *s1, *s2;
};

__device__ __forceinline__ StageView stage_view(char *base, int maxs) {
    StageView v;
    v.s0 = (int4 *)base;
    v.s1 = (float4 *)(base + 16 * (size_t)maxs);
    v.s2 = (float4 *)(base + 32 * (size_t)maxs);
    return v;
}

// Bytes of one stage: three 16-byte arrays, rounded to 128.
__host__ __device__ inline size_t pipe_stage_bytes(int maxs) {
    return ((size_t)48 * maxs + 127) & ~(size_t)127;
}
__host__ __device__ inline size_t pipe_smem_bytes(int maxs) {
    return 128 + kPipeStages * pipe_stage_bytes(maxs);
}

// issued by one thread: chunk q of the colour range into stage st
__device__ __forceinline__ void pipe_issue(const Dev &d, const SweepParams &p, int q, int cv, int maxs,
                                           char *stages, StageMeta *meta, unsigned long long *bar, int st) {
    const int v0 = p.vbegin + q * cv;
    const int v1 = min(p.vend, v0 + cv);
    const int a = d.slot_off[v0], b = d.slot_off[v1];
    const int n = b - a;
    StageMeta m;
    m.a = a;
    m.n = n;
    m.pad = 0;
    m.direct = (n <= 0 || n > maxs) ? 1 : 0;
    meta[st] = m;
    const unsigned ab = smem_addr(bar + st);
    if (m.direct) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(ab) : "memory");
        return;
    }
    const unsigned tx = 48u * (unsigned)n;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(ab), "r"(tx) : "memory");
    StageView v = stage_view(stages + st * pipe_stage_bytes(maxs), maxs);
    bulk_g2s(v.s0, d.s0 + a, 16u * n, bar + st);
    bulk_g2s(v.s1, d.s1 + a, 16u * n, bar + st);
    bulk_g2s(v.s2, d.s2 + a, 16u * n, bar + st);
}

template <int TT>
__global__ void __launch_bounds__(TT) k_sweep_pipe(Dev d, SweepParams p, int maxs) {
    constexpr int L = kPipeLanes;
    constexpr int CV = TT / L;  // vertices per chunk
    extern __shared__ __align__(128) char smem[];
    unsigned long long *bar = (unsigned long long *)smem;     // kPipeStages barriers + the spare
    StageMeta *meta = (StageMeta *)(smem + 64);               // kPipeStages records
    unsigned long long *never = bar + kPipeStages;            // spare: no arrival (time-out test)
    char *stages = smem + 128;
    const int n = p.vend - p.vbegin;
    const int nchunks = (n + CV - 1) / CV;
    const int first = blockIdx.x, stride = gridDim.x;
    if (threadIdx.x == 0) {
        for (int st = 0; st <= kPipeStages; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(bar + st)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int st = 0; st < kPipeStages; ++st)
            if (first + st * stride < nchunks)
                pipe_issue(d, p, first + st * stride, CV, maxs, stages, meta, bar, st);
    const int lane = threadIdx.x & (L - 1);
    for (int k = 0;; ++k) {
        const int q = first + k * stride;
        if (q >= nchunks) break;
        const int st = k % kPipeStages;
        bool ok = mbar_wait(bar + st, (unsigned)((k / kPipeStages) & 1));
        if (ok && k == 0 && p.stall_test) ok = mbar_wait(never, 0u);  // runs out after ~2 s
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicAdd(d.counters + 2, 1ull);
                // drain this CTA's outstanding copies before leaving (bounded):
                // chunks k .. k+kPipeStages-2 are issued (k .. kPipeStages-1 when k == 0)
                const int last = (k == 0) ? kPipeStages - 1 : k + kPipeStages - 2;
                for (int kk = k; kk <= last; ++kk)
                    if (first + kk * stride < nchunks)
                        mbar_wait(bar + kk % kPipeStages, (unsigned)((kk / kPipeStages) & 1));
            }
            return;
        }
        // all threads are past chunk k-1: its stage takes chunk k-1+kPipeStages
        // (the block barrier orders every thread's reads of the stage before
        // thread 0's next accesses; the proxy fence extends that order to the
        // bulk copies' async-proxy writes)
        if (k >= 1 && threadIdx.x == 0) {
            const int kk = k - 1 + kPipeStages;
            if (first + kk * stride < nchunks) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                pipe_issue(d, p, first + kk * stride, CV, maxs, stages, meta, bar, kk % kPipeStages);
            }
        }
        const StageMeta m = meta[st];
        const StageView v = stage_view(stages + st * pipe_stage_bytes(maxs), maxs);
        const int vi = p.vbegin + q * CV + (int)(threadIdx.x / L);
        const bool active = vi < p.vend;
        float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
        int s0 = 0, s1 = 0;
        if (active) {
            xi = d.u[vi];
            s0 = d.slot_off[vi] - m.a;
            s1 = d.slot_off[vi + 1] - m.a;
        }
        const float3 x3 = f3(xi);
        const float2 vm = (active && !p.per_tet_mat) ? __ldg(d.vmat + vi) : make_float2(0.f, 0.f);
        Acc acc = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (!m.direct) {
            for (int s = s0 + lane; s < s1; s += L)
                accumulate_slot(d, p, s + m.a, vm, v.s0[s], v.s1[s], v.s2[s], x3, acc);
        } else {
            for (int s = s0 + lane + m.a; s < s1 + m.a; s += L)
                accumulate_slot(d, p, s, vm, __ldcs(d.s0 + s), __ldcs(d.s1 + s), __ldcs(d.s2 + s), x3, acc);
        }
        acc.f0 = sub_reduce<L>(acc.f0);
        acc.f1 = sub_reduce<L>(acc.f1);
        acc.f2 = sub_reduce<L>(acc.f2);
        acc.h00 = sub_reduce<L>(acc.h00);
        acc.h01 = sub_reduce<L>(acc.h01);
        acc.h02 = sub_reduce<L>(acc.h02);
        acc.h11 = sub_reduce<L>(acc.h11);
        acc.h12 = sub_reduce<L>(acc.h12);
        acc.h22 = sub_reduce<L>(acc.h22);
        if (active && lane == 0) solve_and_store<false>(d, p, vi, xi, acc, acc, 0);
    }
}

// ---- warp rows: per-warp TMA ring over the slot stream (variant 7) ---------
// With vbd_params.warp_rows the slot records are also laid out in "warp
// rows" (Dev::wrow, built at bind by k_build_rows): the free vertices of a
// colour form groups of 8 consecutive vertices, one group per warp-turn; a
// group needs K = max over its vertices of ceil(slots / 4) iterations of 4
// lanes, and takes ceil(K / 2) rows.  Row m of a group holds iterations 2m
// and 2m + 1: entry 32 h + 4 j + l is slot 4 (2m + h) + l of the group's
// vertex j (the slot that lane l of the vertex's four lanes takes at
// iteration 2m + h of k_sweep<4>), or padding (id -1).  A row is one
// 3,072-byte record (the 64 entries' id words, then the two gradient words
// of each), so one bulk copy moves a warp's next 64 slots into its own
// shared-memory ring.  Each warp keeps kRowStages rows in flight, issued by
// its lane 0 as soon as a stage has been read: the slot stream is in flight
// without holding registers, and the lanes wait only on the L2 gathers of the
// neighbour positions.  Per lane the slots and the arithmetic are those of
// k_sweep<4> in the same order, so the positions equal variant 2's with 4
// lanes bit for bit.  Every wait is bounded as in k_sweep_pipe; on a time-out
// the warp records it (counters[2]), waits (bounded) for the rows it has
// issued and leaves.  Each stage barrier expects exactly the bytes copied to it.
constexpr int kRowStages = 2;
constexpr int kRowIters = 2;                     // iterations of 4 lanes per row
constexpr int kRowEntries = 32 * kRowIters;
constexpr int kRowBytes = 3 * kRowEntries * 16;  // one row: ids, then the gradient words
constexpr int kRowWarps = 8;                     // 256-thread CTAs
constexpr size_t kRowSmem = 256 + (size_t)kRowWarps * kRowStages * kRowBytes;

__device__ __forceinline__ void row_issue(const Dev &d, int row, char *stage, unsigned long long *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(kRowBytes)
                 : "memory");
    bulk_g2s(stage, d.wrow + (size_t)row * (3 * kRowEntries), (unsigned)kRowBytes, bar);
}

// one poll of a stage barrier, then the bounded wait only if the row is late
__device__ __forceinline__ bool row_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok ? true : mbar_wait(bar, parity);
}

#ifndef VBD_ROWS_MIN_BLOCKS
#define VBD_ROWS_MIN_BLOCKS 4
#endif
template <bool EXT>
__global__ void __launch_bounds__(256, VBD_ROWS_MIN_BLOCKS) k_sweep_rows(Dev d, SweepParams p) {
    constexpr int L = 4;
    extern __shared__ __align__(128) char smem[];
    const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
    // per warp: kRowStages stage barriers and a spare (time-out test), then its ring
    unsigned long long *bar = (unsigned long long *)smem + warp * (kRowStages + 1);
    char *ring = smem + 256 + (size_t)warp * kRowStages * kRowBytes;
    const int nwarps = gridDim.x * kRowWarps;
    const int w = blockIdx.x * kRowWarps + warp;
    const int ng = p.gend - p.gbegin;
    const int *__restrict__ grow = d.group_row + p.gbegin;
    if (wl == 0) {
        for (int st = 0; st <= kRowStages; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar + st)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // the issue cursor (lane 0 only): group ig, its row ik of iK, rows issued so far;
    // groups without rows (vertices in no tet) are stepped over, as the consumer does
    int ig = w, ik = 0, iK = 0, issued = 0;
    auto next_group = [&]() {
        ik = 0;
        iK = ig < ng ? grow[ig + 1] - grow[ig] : 0;
        while (ig < ng && iK == 0) {
            ig += nwarps;
            iK = ig < ng ? grow[ig + 1] - grow[ig] : 0;
        }
    };
    if (wl == 0) {
        next_group();
        for (int st = 0; st < kRowStages && ig < ng; ++st) {
            row_issue(d, grow[ig] + ik, ring + st * kRowBytes, bar + st);
            ++issued;
            if (++ik == iK) {
                ig += nwarps;
                next_group();
            }
        }
    }
    const int lane = wl & (L - 1);
    int r = 0, st = 0;
    unsigned phase = 0;
    for (int g = w; g < ng; g += nwarps) {
        const int K = grow[g + 1] - grow[g];
        const int vi = p.vbegin + 8 * g + (wl >> 2);
        const bool active = vi < p.vend;
        const float4 xi = active ? d.u[vi] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float3 x3 = f3(xi);
        const float2 vm = active ? __ldg(d.vmat + vi) : make_float2(0.f, 0.f);
        Acc acc = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < K; ++k, ++r) {
            bool ok = row_wait(bar + st, phase);
            if (ok && r == 0 && p.stall_test) ok = mbar_wait(bar + kRowStages, 0u);  // runs out after ~2 s
            if (!__all_sync(FULL, ok)) {
                if (wl == 0) {
                    atomicAdd(d.counters + 2, 1ull);
                    for (int q = r; q < issued; ++q)  // rows issued and not yet consumed
                        mbar_wait(bar + q % kRowStages, (unsigned)((q / kRowStages) & 1));
                }
                __syncwarp();
                return;
            }
            const float4 *row = (const float4 *)(ring + st * kRowBytes);
            float4 e[3 * kRowIters];
#pragma unroll
            for (int h = 0; h < kRowIters; ++h)
#pragma unroll
                for (int a = 0; a < 3; ++a) e[3 * h + a] = row[a * kRowEntries + 32 * h + wl];
            // every lane's reads of this stage are ordered before lane 0 refills it:
            // the warp barrier orders them before lane 0's next accesses, and the
            // proxy fence extends that order to the bulk copy's async-proxy writes
            __syncwarp();
            if (wl == 0 && ig < ng) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                row_issue(d, grow[ig] + ik, ring + st * kRowBytes, bar + st);
                ++issued;
                if (++ik == iK) {
                    ig += nwarps;
                    next_group();
                }
            }
            if (++st == kRowStages) {
                st = 0;
                phase ^= 1u;
            }
#pragma unroll
            for (int h = 0; h < kRowIters; ++h) {
                const int4 r0 = make_int4(__float_as_int(e[3 * h].x), __float_as_int(e[3 * h].y),
                                          __float_as_int(e[3 * h].z), __float_as_int(e[3 * h].w));
                if (r0.x >= 0) accumulate_slot(d, p, 0, vm, r0, e[3 * h + 1], e[3 * h + 2], x3, acc);
            }
        }
        acc.f0 = sub_reduce<L>(acc.f0);
        acc.f1 = sub_reduce<L>(acc.f1);
        acc.f2 = sub_reduce<L>(acc.f2);
        acc.h00 = sub_reduce<L>(acc.h00);
        acc.h01 = sub_reduce<L>(acc.h01);
        acc.h02 = sub_reduce<L>(acc.h02);
        acc.h11 = sub_reduce<L>(acc.h11);
        acc.h12 = sub_reduce<L>(acc.h12);
        acc.h22 = sub_reduce<L>(acc.h22);
        if (active && lane == 0) solve_and_store<false, EXT>(d, p, vi, xi, acc, acc, 0);
    }
}

// Builds the warp rows of one colour from the slot records (one warp per group).
__global__ void k_build_rows(Dev d, int vbegin, int vend, int gbegin, int gend) {
    const int wl = threadIdx.x & 31;
    const int j = wl >> 2, l = wl & 3;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < gend - gbegin; g += nwarps) {
        const int R0 = d.group_row[gbegin + g], R = d.group_row[gbegin + g + 1] - R0;
        const int v = vbegin + 8 * (int)g + j;
        const int s0 = v < vend ? d.slot_off[v] : 0, nv = v < vend ? d.slot_off[v + 1] - s0 : 0;
        for (int m = 0; m < R; ++m)
            for (int h = 0; h < kRowIters; ++h) {
                const int q = 4 * (kRowIters * m + h) + l;
                float4 *rw = d.wrow + (size_t)(R0 + m) * (3 * kRowEntries) + 32 * h + wl;
                if (q < nv) {
                    const int4 a = d.s0[s0 + q];
                    rw[0] = make_float4(__int_as_float(a.x), __int_as_float(a.y), __int_as_float(a.z),
                                        __int_as_float(a.w));
                    rw[kRowEntries] = d.s1[s0 + q];
                    rw[2 * kRowEntries] = d.s2[s0 + q];
                } else {
                    rw[0] = make_float4(__int_as_float(-1), __int_as_float(-1), __int_as_float(-1), 0.f);
                    rw[kRowEntries] = make_float4(0.f, 0.f, 0.f, 0.f);
                    rw[2 * kRowEntries] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
    }
}

// Eq. 3 and Sec. 3.7 options (a)-(d), Eq. 17.  Pinned vertices (ids >= n_free) keep x^t.
__global__ void k_predict(Dev d, int n, int n_free, float h, float3 g, float gnorm, int mode,
                          int cheby, int has_sub) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 xi = d.u[i];
    d.ut[i] = make_float4(xi.x, xi.y, xi.z, 0.f);
    if (i >= n_free) {
        d.u[i] = make_float4(xi.x, xi.y, xi.z, 0.f);
        return;
    }
    const float4 vi = d.v[i];
    const float h2 = h * h;
    d.ym[i] = make_float4(xi.x + h * vi.x + h2 * g.x, xi.y + h * vi.y + h2 * g.y,
                          xi.z + h * vi.z + h2 * g.z, d.mass[i] / h2);
    float4 xn;
    if (mode == 0) {
        xn = make_float4(xi.x, xi.y, xi.z, 0.f);
    } else {
        float at = (mode == 2) ? 1.f : 0.f;
        if (mode == 3 && gnorm > 0.f) {
            const float4 wi = d.vprev[i];
            const float comp = ((vi.x - wi.x) / h * g.x + (vi.y - wi.y) / h * g.y +
                                (vi.z - wi.z) / h * g.z) / gnorm;
            at = comp > gnorm ? 1.f : (comp < 0.f ? 0.f : comp / gnorm);
        }
        const float ah2 = h2 * at;
        xn = make_float4(xi.x + h * vi.x + ah2 * g.x, xi.y + h * vi.y + ah2 * g.y,
                         xi.z + h * vi.z + ah2 * g.z, 0.f);
        const int sub = has_sub ? d.sub_id[i] : -1;
        if (sub >= 0) {  // a subspace-constrained vertex starts on x^t + span(Q) (Sec. 3.4)
            const float4 qa = d.sub_q[2 * sub], qb = d.sub_q[2 * sub + 1];
            const float ex = xn.x - xi.x, ey = xn.y - xi.y, ez = xn.z - xi.z;
            const float ca = qa.x * ex + qa.y * ey + qa.z * ez;
            const float cb = qa.w < 1.5f ? 0.f : qb.x * ex + qb.y * ey + qb.z * ez;
            xn = make_float4(xi.x + ca * qa.x + cb * qb.x, xi.y + ca * qa.y + cb * qb.y,
                             xi.z + ca * qa.z + cb * qb.z, 0.f);
        }
    }
    d.u[i] = xn;
    if (cheby) d.cheb[0][i] = xn;
}

// Eq. 18 after iteration n: history buffer cheb[n & 1] holds x^(n-2) on entry
// and x^(n) on exit; the other buffer holds x^(n-1).  Vertices flagged in
// contact (x.w != 0: ground, wall or self-contact) keep the Gauss-Seidel
// result.
template <bool COH>
__device__ __forceinline__ void cheby_vertex(const Dev &d, int i, int n, float omega) {
    float4 *hist = d.cheb[n & 1];
    const float4 xb = COH ? __ldcg(d.u + i) : d.u[i];
    float4 xn = xb;
    // The history moves through L2 as a stream (evict-first), so that it does
    // not displace the positions the colour passes gather from L2.
    if (n >= 2 && xb.w == 0.f) {
        const float4 q = COH ? __ldcg(hist + i) : __ldcs(hist + i);
        xn = make_float4(omega * (xb.x - q.x) + q.x, omega * (xb.y - q.y) + q.y,
                         omega * (xb.z - q.z) + q.z, xb.w);
        d.u[i] = xn;
    }
    if (COH)
        hist[i] = xn;
    else
        __stcs(hist + i, xn);
}

__global__ void k_cheby(Dev d, int n_free, int n, float omega) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_free) cheby_vertex<false>(d, i, n, omega);
}

// ---- fused iteration loop for small meshes ------------------------------------
// All iterations of vbd_iterate in one launch of one thread-block cluster: the
// CTAs split each colour pass (and the Chebyshev update) and meet at the
// hardware cluster barrier between passes, whose release/acquire ordering
// makes one pass's writes visible to the next; positions are then read from
// L2 (__ldcg), never through the non-coherent path.  Same arithmetic as the
// per-colour launches, so the results are identical bit for bit.
template <int L>
__global__ void __launch_bounds__(kFusedThreads, 1) k_iterate_fused(Dev d, FusedParams f) {
    cg::cluster_group cluster = cg::this_cluster();
    const long long rank = cluster.block_rank();
    const long long stride = (long long)cluster.num_blocks() * blockDim.x;
    for (int n = f.first_n + 1; n <= f.first_n + f.iters; ++n) {
        for (int c = 0; c < f.n_colors; ++c) {
            const int vbegin = d.color_begin[c], vend = d.color_begin[c + 1];
            const long long threads = (long long)(vend - vbegin) * L;
            for (long long base = rank * blockDim.x; base < threads; base += stride)
                sweep_body<L, false, true>(d, f.p, base + threadIdx.x, vbegin, vend);
            cluster.sync();
        }
        if (f.cheby) {
            // omega_n of Eq. 19, the same FP64 recurrence as the host's
            const double r2 = f.rho * f.rho;
            double w = 1.0;
            for (int k = 2; k <= n; ++k) w = (k == 2) ? 2.0 / (2.0 - r2) : 4.0 / (4.0 - r2 * w);
            for (long long i = rank * blockDim.x + threadIdx.x; i < f.n_free; i += stride)
                cheby_vertex<true>(d, (int)i, n, (float)w);
            cluster.sync();
        }
    }
}

// Eq. 6; v^{t-1} <- v^t; optional tape row.
__global__ void k_finish(Dev d, int n, float h, float4 *tape_row) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 x = d.u[i], xt = d.ut[i];
    d.vprev[i] = d.v[i];
    d.v[i] = make_float4((x.x - xt.x) / h, (x.y - xt.y) / h, (x.z - xt.z) / h, 0.f);
    if (tape_row) tape_row[i] = make_float4(x.x, x.y, x.z, 0.f);
    if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z))) atomicAdd(d.counters + 0, 1ull);
}

__global__ void k_scatter(const float *src, float4 *dst, const int *new_of_orig, const float4 *rest, int n) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int i = new_of_orig[o];
    float4 a = make_float4(src[3 * o], src[3 * o + 1], src[3 * o + 2], 0.f);
    if (rest) {
        const float4 X = rest[i];
        a.x -= X.x; a.y -= X.y; a.z -= X.z;
    }
    dst[i] = a;
}

__global__ void k_gather(const float4 *src, float *dst, const int *new_of_orig, const float4 *rest, int n) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int i = new_of_orig[o];
    float4 a = src[i];
    if (rest) {
        const float4 X = rest[i];
        a.x += X.x; a.y += X.y; a.z += X.z;
    }
    dst[3 * o] = a.x;
    dst[3 * o + 1] = a.y;
    dst[3 * o + 2] = a.z;
}

// the pass wrote vertices [vbegin, vend) to unew (x^new of Algorithm 1); copy
// them back -- with involved_only, just the vertices in a self-contact pair
// a vertex is involved when it has a vertex-triangle pair, is a corner of
// one, or (ee_on) belongs to an edge-edge pair
__global__ void k_copy_back(Dev d, int vbegin, int vend, int involved_only, int ee_on) {
    const int i = vbegin + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vend) return;
    if (involved_only && d.contact[i] < 0 && d.rev_off[i + 1] == d.rev_off[i] &&
        !(ee_on && d.ee_off[i + 1] != d.ee_off[i]))
        return;
    d.u[i] = d.unew[i];
}

// Convergence report: max over free vertices of |dG/dx_i| (Eq. 2 with the
// plane penalties of Eq. 12), i.e. of the local force f_i of Eq. 8 at the
// current x and the current step's y, without moving anything.  Per vertex in
// FP32 like the sweep, reduced in FP64 by an atomic max on the bits of the
// non-negative doubles.  All free vertices in one launch (nothing is written
// but the maximum).
template <int L>
__global__ void __launch_bounds__(256) k_grad_norm(Dev d, SweepParams p, int n_free, double *out) {
    const int lane = threadIdx.x & (L - 1);
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int vi = (int)(gt / L);
    const bool active = vi < n_free;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    int s0 = 0, s1 = 0;
    if (active) {
        xi = d.u[vi];
        s0 = d.slot_off[vi];
        s1 = d.slot_off[vi + 1];
    }
    const float3 x3 = f3(xi);
    const float2 vm = (active && !p.per_tet_mat) ? __ldg(d.vmat + vi) : make_float2(0.f, 0.f);
    Acc acc = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int s = s0 + lane; s < s1; s += L)
        accumulate_slot(d, p, s, vm, __ldcs(d.s0 + s), __ldcs(d.s1 + s), __ldcs(d.s2 + s), x3, acc);
    acc.f0 = sub_reduce<L>(acc.f0);
    acc.f1 = sub_reduce<L>(acc.f1);
    acc.f2 = sub_reduce<L>(acc.f2);
    float g = 0.f;
    if (active && lane == 0) {
        const float4 yv = d.ym[vi];
        float f0 = yv.w * (yv.x - xi.x) + acc.f0, f1 = yv.w * (yv.y - xi.y) + acc.f1,
              f2 = yv.w * (yv.z - xi.z) + acc.f2;
        if (p.n_planes > 0) {
            const float4 X = d.rest[vi];
            const float3 P = make_float3(X.x + xi.x, X.y + xi.y, X.z + xi.z);
            for (int k = 0; k < p.n_planes; ++k) {
                const float4 pl = p.planes[k];
                const float pen = pl.w - (pl.x * P.x + pl.y * P.y + pl.z * P.z);
                if (pen > 0.f) {
                    f0 += p.kc * pen * pl.x;
                    f1 += p.kc * pen * pl.y;
                    f2 += p.kc * pen * pl.z;
                }
            }
        }
        // a non-finite component reports as +inf (fmaxf alone would drop a NaN)
        g = (isfinite(f0) && isfinite(f1) && isfinite(f2)) ? fmaxf(fabsf(f0), fmaxf(fabsf(f1), fabsf(f2)))
                                                             : INFINITY;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) g = fmaxf(g, __shfl_xor_sync(FULL, g, off));
    if ((threadIdx.x & 31) == 0 && g > 0.f)
        atomicMax((unsigned long long *)out, (unsigned long long)__double_as_longlong((double)g));
}

__global__ void k_restore_x(Dev d, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d.u[i] = d.ut[i];
}

// ---- FP64 energy of Eq. 2 (diagnostics) -----------------------------------
// Psi = mu/2 (tr F^T F - 3) + lam/2 (J - alpha)^2 evaluated from F = I + D.
constexpr int EB = 256;

__device__ __forceinline__ void block_sum_store(double v, double *out) {
    __shared__ double sh[EB / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < EB / 32; ++w) t += sh[w];
        *out = t;
    }
}

__global__ void __launch_bounds__(EB) k_energy_verts(Dev d, int n_free, double inv_2h2, SweepParams p,
                                                     double *partials) {
    double e = 0.0;
    for (int i = blockIdx.x * EB + threadIdx.x; i < n_free; i += gridDim.x * EB) {
        const float4 x = d.u[i], y = d.ym[i], X = d.rest[i];
        const double dx = (double)x.x - y.x, dy = (double)x.y - y.y, dz = (double)x.z - y.z;
        e += (double)d.mass[i] * inv_2h2 * (dx * dx + dy * dy + dz * dz);
        for (int k = 0; k < p.n_planes; ++k) {
            const float4 pl = p.planes[k];
            const double pen = (double)pl.w - ((double)pl.x * ((double)X.x + x.x) + (double)pl.y * ((double)X.y + x.y) +
                                               (double)pl.z * ((double)X.z + x.z));
            if (pen > 0.0) e += 0.5 * (double)p.kc * pen * pen;
        }
    }
    block_sum_store(e, partials + blockIdx.x);
}

__global__ void __launch_bounds__(EB) k_energy_tets(Dev d, int n_tets, double *partials) {
    double e = 0.0;
    for (int j = blockIdx.x * EB + threadIdx.x; j < n_tets; j += gridDim.x * EB) {
        // F = I + D with D from the displacements (rest edges times B give I)
        const int4 t = d.tet_v[j];
        const float4 p0 = d.u[t.x], p1 = d.u[t.y], p2 = d.u[t.z], p3 = d.u[t.w];
        const double E[3][3] = {{(double)p1.x - p0.x, (double)p2.x - p0.x, (double)p3.x - p0.x},
                                {(double)p1.y - p0.y, (double)p2.y - p0.y, (double)p3.y - p0.y},
                                {(double)p1.z - p0.z, (double)p2.z - p0.z, (double)p3.z - p0.z}};
        const float *B = d.tet_B + 9 * (size_t)j;
        double D[3][3];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s)
                D[r][s] = E[r][0] * B[s] + E[r][1] * B[3 + s] + E[r][2] * B[6 + s];
        const double tr = D[0][0] + D[1][1] + D[2][2];
        const double m2 = (D[0][0] * D[1][1] - D[0][1] * D[1][0]) + (D[0][0] * D[2][2] - D[0][2] * D[2][0]) +
                          (D[1][1] * D[2][2] - D[1][2] * D[2][1]);
        const double det = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                           D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                           D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
        double dd = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) dd += D[r][s] * D[r][s];
        const double mu = d.tet_mu[j], lam = d.tet_lam[j];
        const double jma = tr + m2 + det - mu / lam;  // J - alpha
        // tr F^T F - 3 = 2 tr D + |D|^2
        e += (double)d.tet_V[j] * (0.5 * mu * (2.0 * tr + dd) + 0.5 * lam * jma * jma);
    }
    block_sum_store(e, partials + blockIdx.x);
}

// self-contact energy k_c d^2 / 2 of every current pair with d > 0
__global__ void __launch_bounds__(EB) k_energy_contacts(Dev d, int n_surf, int n_edges, double kc, double *partials) {
    double e = 0.0;
    for (int k = blockIdx.x * EB + threadIdx.x; k < n_surf; k += gridDim.x * EB) {
        const int a = d.surf[k];
        const int T = d.contact[a];
        if (T < 0) continue;
        float3 n, w;
        const double dep = geom::pair_depth(d, a, d.tri[T], n, w);
        if (dep > 0.0) e += 0.5 * kc * dep * dep;
    }
    // edge-edge pairs, held by their edges (n_edges = 0 when there are none)
    for (int k = blockIdx.x * EB + threadIdx.x; k < n_edges; k += gridDim.x * EB) {
        const int f = d.ee_partner[k];
        if (f < 0) continue;
        const int4 ev = d.edge_v[k], fv = d.edge_v[f];
        const float4 prm = d.ee_prm[k], nv = d.ee_nrm[k];
        const double cw[4] = {-(1.0 - prm.x), -(double)prm.x, 1.0 - prm.y, (double)prm.y};
        const int vid[4] = {ev.x, ev.y, fv.x, fv.y};
        double dep = 0.0;
        for (int j = 0; j < 4; ++j) {
            const float4 X = d.rest[vid[j]], u = d.u[vid[j]];
            dep += cw[j] * (((double)X.x + u.x) * nv.x + ((double)X.y + u.y) * nv.y + ((double)X.z + u.z) * nv.z);
        }
        if (dep > 0.0) e += 0.5 * kc * dep * dep;
    }
    block_sum_store(e, partials + blockIdx.x);
}

__global__ void k_reduce_partials(const double *partials, int n, double *out) {
    double e = 0.0;
    for (int i = threadIdx.x; i < n; i += EB) e += partials[i];
    block_sum_store(e, out);
}

__global__ void k_set_log_young(Dev d, const float *log_young, int n_tets) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tets) return;
    const float E = expf(log_young[i]);
    const float nu = d.tet_nu[i];
    const float mu = E / (2.f * (1.f + nu));
    d.tet_mu[i] = mu;
    d.tet_lam[i] = E * nu / ((1.f + nu) * (1.f - 2.f * nu)) + mu;
}

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

int num_sms() {
    int dev = 0, n = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

void launch_predict(const Dev &d, int n, int n_free, float h, float3 g, int init_mode, bool cheby,
                    bool has_sub, cudaStream_t s) {
    const float gnorm = sqrtf(g.x * g.x + g.y * g.y + g.z * g.z);
    k_predict<<<blocks_for(n, 256), 256, 0, s>>>(d, n, n_free, h, g, gnorm, init_mode, cheby ? 1 : 0,
                                                  has_sub ? 1 : 0);
}

// the sweep instance with the optional epilogue parts
static bool needs_ext(const SweepParams &p) { return p.line_search || p.n_sub > 0; }

template <int L, bool EXT>
static unsigned persist_grid(int block) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_persist<L, EXT>, block, 0) != cudaSuccess ||
        occ < 1)
        occ = 1;
    return (unsigned)(num_sms() * occ);
}

template <bool EXT>
static void launch_persist_ext(const Dev &d, const SweepParams &p, int lanes, int block, long long threads,
                              cudaStream_t s) {
    const unsigned need = blocks_for(threads, block);
    switch (lanes) {
    case 4: k_sweep_persist<4, EXT><<<std::min(need, persist_grid<4, EXT>(block)), block, 0, s>>>(d, p, threads); break;
    case 8: k_sweep_persist<8, EXT><<<std::min(need, persist_grid<8, EXT>(block)), block, 0, s>>>(d, p, threads); break;
    case 16:
        k_sweep_persist<16, EXT><<<std::min(need, persist_grid<16, EXT>(block)), block, 0, s>>>(d, p, threads);
        break;
    default:
        k_sweep_persist<32, EXT><<<std::min(need, persist_grid<32, EXT>(block)), block, 0, s>>>(d, p, threads);
        break;
    }
}

void launch_sweep_persist(const Dev &d, const SweepParams &p, int lanes, int block, cudaStream_t s) {
    const long long threads = (long long)(p.vend - p.vbegin) * lanes;
    if (threads <= 0) return;
    if (needs_ext(p))
        launch_persist_ext<true>(d, p, lanes, block, threads, s);
    else
        launch_persist_ext<false>(d, p, lanes, block, threads, s);
}

template <int L, bool EXT>
static unsigned rest_grid(int block) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_rest<L, EXT>, block, 0) != cudaSuccess || occ < 1)
        occ = 1;
    return (unsigned)(num_sms() * occ);
}

template <bool EXT>
static void launch_rest_ext(const Dev &d, const SweepParams &p, int lanes, int block, long long threads,
                           cudaStream_t s) {
    const unsigned need = blocks_for(threads, block);
    switch (lanes) {
    case 4: k_sweep_rest<4, EXT><<<std::min(need, rest_grid<4, EXT>(block)), block, 0, s>>>(d, p, threads); break;
    case 8: k_sweep_rest<8, EXT><<<std::min(need, rest_grid<8, EXT>(block)), block, 0, s>>>(d, p, threads); break;
    case 16: k_sweep_rest<16, EXT><<<std::min(need, rest_grid<16, EXT>(block)), block, 0, s>>>(d, p, threads); break;
    default: k_sweep_rest<32, EXT><<<std::min(need, rest_grid<32, EXT>(block)), block, 0, s>>>(d, p, threads); break;
    }
}

void launch_sweep_rest(const Dev &d, const SweepParams &p, int lanes, int block, cudaStream_t s) {
    const long long threads = (long long)(p.vend - p.vbegin) * lanes;
    if (threads <= 0) return;
    if (needs_ext(p))
        launch_rest_ext<true>(d, p, lanes, block, threads, s);
    else
        launch_rest_ext<false>(d, p, lanes, block, threads, s);
}

template <int L, bool EXT>
static unsigned pair_grid(int block) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_pair<L, EXT>, block, 0) != cudaSuccess || occ < 1)
        occ = 1;
    return (unsigned)(num_sms() * occ);
}

template <bool EXT>
static void launch_pair_ext(const Dev &d, const SweepParams &p, int lanes, int block, long long threads,
                            cudaStream_t s) {
    const unsigned need = blocks_for(threads, block);
    switch (lanes) {
    case 4: k_sweep_pair<4, EXT><<<std::min(need, pair_grid<4, EXT>(block)), block, 0, s>>>(d, p, threads); break;
    case 8: k_sweep_pair<8, EXT><<<std::min(need, pair_grid<8, EXT>(block)), block, 0, s>>>(d, p, threads); break;
    case 16: k_sweep_pair<16, EXT><<<std::min(need, pair_grid<16, EXT>(block)), block, 0, s>>>(d, p, threads); break;
    default: k_sweep_pair<32, EXT><<<std::min(need, pair_grid<32, EXT>(block)), block, 0, s>>>(d, p, threads); break;
    }
}

void launch_sweep_pair(const Dev &d, const SweepParams &p, int lanes, int block, cudaStream_t s) {
    const long long threads = (long long)(p.vend - p.vbegin) * lanes;
    if (threads <= 0) return;
    if (needs_ext(p))
        launch_pair_ext<true>(d, p, lanes, block, threads, s);
    else
        launch_pair_ext<false>(d, p, lanes, block, threads, s);
}

template <bool EXT>
static unsigned rows_grid() {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_rows<EXT>, 256, kRowSmem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    return (unsigned)(num_sms() * occ);
}

void launch_sweep_rows(const Dev &d, const SweepParams &p, cudaStream_t s) {
    const int ng = p.gend - p.gbegin;
    if (ng <= 0) return;
    // above the 48 KB default of dynamic shared memory; the attribute is per device
    static std::mutex mu;
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;  // the caller reads the error
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!attr_set[dev]) {
            if (cudaFuncSetAttribute(k_sweep_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRowSmem) != cudaSuccess ||
                cudaFuncSetAttribute(k_sweep_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRowSmem) != cudaSuccess)
                return;  // left in cudaGetLastError for the caller
            attr_set[dev] = true;
        }
    }
    const unsigned need = (unsigned)((ng + kRowWarps - 1) / kRowWarps);
    if (needs_ext(p))
        k_sweep_rows<true><<<std::min(need, rows_grid<true>()), 256, kRowSmem, s>>>(d, p);
    else
        k_sweep_rows<false><<<std::min(need, rows_grid<false>()), 256, kRowSmem, s>>>(d, p);
}

int rows_per_group(int iterations) { return (iterations + kRowIters - 1) / kRowIters; }
size_t row_record_bytes() { return (size_t)kRowBytes; }

void launch_build_rows(const Dev &d, int vbegin, int vend, int gbegin, int gend, cudaStream_t s) {
    if (gend > gbegin)
        k_build_rows<<<std::min<long long>(blocks_for(32LL * (gend - gbegin), 256), 148 * 16), 256, 0, s>>>(
            d, vbegin, vend, gbegin, gend);
}

void launch_sweep_scatter(const Dev &d, const SweepParams &p, int sbegin, int send, int lanes, int block,
                          cudaStream_t s) {
    const long long threads = (long long)(p.vend - p.vbegin) * lanes;
    if (threads <= 0) return;
    if (send > sbegin) k_scatter_slots<<<blocks_for(send - sbegin, 256), 256, 0, s>>>(d, p, sbegin, send - sbegin);
    const unsigned grid = blocks_for(threads, block);
    switch (lanes) {
    case 4: k_scatter_reduce<4><<<grid, block, 0, s>>>(d, p, sbegin); break;
    case 8: k_scatter_reduce<8><<<grid, block, 0, s>>>(d, p, sbegin); break;
    case 16: k_scatter_reduce<16><<<grid, block, 0, s>>>(d, p, sbegin); break;
    default: k_scatter_reduce<32><<<grid, block, 0, s>>>(d, p, sbegin); break;
    }
}

void launch_sweep(const Dev &d, const SweepParams &p, int lanes, int block, cudaStream_t s) {
    const long long threads = (long long)(p.vend - p.vbegin) * lanes;
    if (threads <= 0) return;
    const unsigned grid = blocks_for(threads, block);
    if (p.self_collision) {
        if (needs_ext(p)) {
            switch (lanes) {
            case 4: k_sweep_sc<4, true><<<grid, block, 0, s>>>(d, p); break;
            case 8: k_sweep_sc<8, true><<<grid, block, 0, s>>>(d, p); break;
            case 16: k_sweep_sc<16, true><<<grid, block, 0, s>>>(d, p); break;
            default: k_sweep_sc<32, true><<<grid, block, 0, s>>>(d, p); break;
            }
            return;
        }
        switch (lanes) {
        case 4: k_sweep_sc<4, false><<<grid, block, 0, s>>>(d, p); break;
        case 8: k_sweep_sc<8, false><<<grid, block, 0, s>>>(d, p); break;
        case 16: k_sweep_sc<16, false><<<grid, block, 0, s>>>(d, p); break;
        default: k_sweep_sc<32, false><<<grid, block, 0, s>>>(d, p); break;
        }
        return;
    }
    if (needs_ext(p)) {
        switch (lanes) {
        case 4: k_sweep<4, true><<<grid, block, 0, s>>>(d, p); break;
        case 8: k_sweep<8, true><<<grid, block, 0, s>>>(d, p); break;
        case 16: k_sweep<16, true><<<grid, block, 0, s>>>(d, p); break;
        default: k_sweep<32, true><<<grid, block, 0, s>>>(d, p); break;
        }
        return;
    }
    switch (lanes) {
    case 4: k_sweep<4, false><<<grid, block, 0, s>>>(d, p); break;
    case 8: k_sweep<8, false><<<grid, block, 0, s>>>(d, p); break;
    case 16: k_sweep<16, false><<<grid, block, 0, s>>>(d, p); break;
    default: k_sweep<32, false><<<grid, block, 0, s>>>(d, p); break;
    }
}

size_t sweep_pipe_smem(int maxs) { return pipe_smem_bytes(maxs); }

int sweep_pipe_chunk(int block) { return block / kPipeLanes; }

cudaError_t sweep_pipe_prepare(int block, int maxs, int *ctas_per_sm) {
    const size_t smem = pipe_smem_bytes(maxs);
    cudaError_t e;
    int occ = 0;
    if (block == 256) {
        e = cudaFuncSetAttribute(k_sweep_pipe<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_pipe<256>, 256, smem);
    } else {
        e = cudaFuncSetAttribute(k_sweep_pipe<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_pipe<128>, 128, smem);
    }
    if (e != cudaSuccess) return e;
    *ctas_per_sm = occ;
    return occ > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

void launch_sweep_pipe(const Dev &d, const SweepParams &p, int block, int maxs, int grid_cap, cudaStream_t s) {
    const int n = p.vend - p.vbegin;
    if (n <= 0) return;
    const int cv = block / kPipeLanes;
    const int nchunks = (n + cv - 1) / cv;
    const unsigned grid = (unsigned)std::max(1, std::min(nchunks, grid_cap));
    const size_t smem = pipe_smem_bytes(maxs);
    if (block == 256)
        k_sweep_pipe<256><<<grid, 256, smem, s>>>(d, p, maxs);
    else
        k_sweep_pipe<128><<<grid, 128, smem, s>>>(d, p, maxs);
}

int fused_clusters_needed(int max_colour_verts, int lanes) {
    const long long threads = (long long)max_colour_verts * lanes;
    const long long per_round = (long long)kFusedMaxCluster * kFusedThreads;
    if (threads > per_round * kFusedMaxRounds) return 0;
    return (int)std::max<long long>(1, std::min<long long>(kFusedMaxCluster,
                                                           (threads + kFusedThreads - 1) / kFusedThreads));
}

cudaError_t launch_iterate_fused(const Dev &d, const FusedParams &f, int lanes, int cluster, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster, 1, 1);
    cfg.blockDim = dim3(kFusedThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    switch (lanes) {
    case 4: return cudaLaunchKernelEx(&cfg, k_iterate_fused<4>, d, f);
    case 8: return cudaLaunchKernelEx(&cfg, k_iterate_fused<8>, d, f);
    case 16: return cudaLaunchKernelEx(&cfg, k_iterate_fused<16>, d, f);
    default: return cudaLaunchKernelEx(&cfg, k_iterate_fused<32>, d, f);
    }
}

void launch_cheby(const Dev &d, int n_free, int n, float omega, cudaStream_t s) {
    if (n_free > 0) k_cheby<<<blocks_for(n_free, 256), 256, 0, s>>>(d, n_free, n, omega);
}

void launch_finish(const Dev &d, int n, float h, float4 *tape_row, cudaStream_t s) {
    k_finish<<<blocks_for(n, 256), 256, 0, s>>>(d, n, h, tape_row);
}

void launch_scatter(const float *src, float4 *dst, const int *new_of_orig, const float4 *rest, int n,
                    cudaStream_t s) {
    k_scatter<<<blocks_for(n, 256), 256, 0, s>>>(src, dst, new_of_orig, rest, n);
}

void launch_gather(const float4 *src, float *dst, const int *new_of_orig, const float4 *rest, int n,
                   cudaStream_t s) {
    k_gather<<<blocks_for(n, 256), 256, 0, s>>>(src, dst, new_of_orig, rest, n);
}

void launch_copy_back(const Dev &d, int vbegin, int vend, bool involved_only, bool ee_on, cudaStream_t s) {
    if (vend > vbegin)
        k_copy_back<<<blocks_for(vend - vbegin, 256), 256, 0, s>>>(d, vbegin, vend, involved_only ? 1 : 0,
                                                                   ee_on ? 1 : 0);
}

cudaError_t launch_grad_norm(const Dev &d, const SweepParams &p, int n_free, double *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
    if (e != cudaSuccess || n_free <= 0) return e;
    k_grad_norm<4><<<blocks_for(4LL * n_free, 256), 256, 0, s>>>(d, p, n_free, out);
    return cudaGetLastError();
}

void launch_restore_x(const Dev &d, int n, cudaStream_t s) {
    k_restore_x<<<blocks_for(n, 256), 256, 0, s>>>(d, n);
}

static void energy_grid(int n_free, int n_tets, int n_surf, int *gv, int *gt, int *gc) {
    const int cap = 4 * 148;
    *gv = (int)std::min<long long>(cap, std::max<long long>(1, blocks_for(n_free, EB)));
    *gt = (int)std::min<long long>(cap, std::max<long long>(1, blocks_for(n_tets, EB)));
    *gc = n_surf > 0 ? (int)std::min<long long>(cap, blocks_for(n_surf, EB)) : 0;
}

int energy_partials_needed(int n_free, int n_tets, int n_surf) {
    int gv, gt, gc;
    energy_grid(n_free, n_tets, n_surf, &gv, &gt, &gc);
    return gv + gt + gc;
}

void launch_energy(const Dev &d, int n_free, int n_tets, int n_surf, double h, const SweepParams &p,
                   cudaStream_t s) {
    int gv, gt, gc;
    energy_grid(n_free, n_tets, n_surf, &gv, &gt, &gc);
    k_energy_verts<<<gv, EB, 0, s>>>(d, n_free, 1.0 / (2.0 * h * h), p, d.partials);
    k_energy_tets<<<gt, EB, 0, s>>>(d, n_tets, d.partials + gv);
    if (gc > 0)
        k_energy_contacts<<<gc, EB, 0, s>>>(d, n_surf, p.ee_on ? p.n_edges : 0, (double)p.kc, d.partials + gv + gt);
    k_reduce_partials<<<1, EB, 0, s>>>(d.partials, gv + gt + gc, d.energy_out);
}

void launch_set_log_young(const Dev &d, const float *log_young, int n_tets, cudaStream_t s) {
    k_set_log_young<<<blocks_for(n_tets, 256), 256, 0, s>>>(d, log_young, n_tets);
}

// ---- energy with library-owned scratch --------------------------------------
// vbd_energy_static runs the same three energy kernels as launch_energy, but
// its per-block partial sums live in this file-scope device array instead of
// the caller's workspace, and the total goes straight to a caller-given
// device double.  Each device that loads the library holds one copy (512 KiB)
// until the process exits; every call on that device reuses it, so calls
// that overlap on the GPU (other streams, other contexts) race on it.
namespace {
constexpr int kStaticPartials = 65536;
static __device__ __align__(256) double g_static_partials[kStaticPartials];
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
// per device: the CUDA context whose module the cached address belongs to
struct StaticScratch {
    unsigned long long ctx_id;
    double *ptr;
};
StaticScratch g_static[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (0 if none).  Taken
// from the driver through the runtime's entry-point query, so the library
// needs no link against the driver library.
cudaError_t current_context_id(unsigned long long *id) {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    *id = 0;
    if (!get_current || !get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorSymbolNotFound;
        get_current = (PFN_cuCtxGetCurrent_v4000)f1;
        get_id = (PFN_cuCtxGetId_v12000)f2;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    if (!ctx) return cudaSuccess;
    if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}
}  // namespace

int energy_static_capacity() { return kStaticPartials; }

int energy_static_partials_needed(int n_free, int n_tets, int n_surf) {
    const long long gv = std::max<long long>(1, blocks_for(n_free, EB));
    const long long gt = std::max<long long>(1, blocks_for(n_tets, EB));
    const long long gc = n_surf > 0 ? blocks_for(n_surf, EB) : 0;
    return (int)std::min<long long>(gv + gt + gc, 0x7fffffffLL);
}

// Device address of g_static_partials in the current device's current
// context.  The symbol name is only a host-side handle; kernels must be given
// this address.  It is looked up once per (device, context): the module, and
// so the array, is loaded per context, and a context made after a reset of
// the device (cudaDeviceReset, then new work) may place it elsewhere, so the
// cached address is keyed by the context's unique id and looked up again
// when that id changes.  The first call in a context does the lookup, so it
// should precede any stream capture.
cudaError_t energy_static_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);  // also guards the entry points' first lookup
    unsigned long long id = 0;
    e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    if (id == 0 || !g_static[dev].ptr || g_static[dev].ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_partials);  // makes the runtime's context current if none was
        if (e != cudaSuccess) return e;
        if (id == 0) {
            e = current_context_id(&id);
            if (e != cudaSuccess) return e;
        }
        g_static[dev].ptr = (double *)p;
        g_static[dev].ctx_id = id;
    }
    *out = g_static[dev].ptr;
    return cudaSuccess;
}

cudaError_t launch_energy_static(const Dev &d, int n_free, int n_tets, int n_surf, double h,
                                 const SweepParams &p, double *G_out, cudaStream_t s) {
    const int gv = std::max(1, (int)blocks_for(n_free, EB));
    const int gt = std::max(1, (int)blocks_for(n_tets, EB));
    const int gc = n_surf > 0 ? (int)blocks_for(n_surf, EB) : 0;
    if ((long long)gv + gt + gc > kStaticPartials) return cudaErrorInvalidValue;
    double *part = nullptr;
    cudaError_t e = energy_static_scratch(&part);
    if (e != cudaSuccess) return e;
    // every partial slot [0, gv + gt + gc) is written before the final sum reads it
    k_energy_verts<<<gv, EB, 0, s>>>(d, n_free, 1.0 / (2.0 * h * h), p, part);
    k_energy_tets<<<gt, EB, 0, s>>>(d, n_tets, part + gv);
    if (gc > 0)
        k_energy_contacts<<<gc, EB, 0, s>>>(d, n_surf, p.ee_on ? p.n_edges : 0, (double)p.kc, part + gv + gt);
    k_reduce_partials<<<1, EB, 0, s>>>(part, gv + gt + gc, G_out);
    return cudaGetLastError();
}

}  // namespace vbd

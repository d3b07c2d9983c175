// vbd_adjoint.cu -- reverse pass through converged VBD steps (no paper
// counterpart: the paper has no derivatives; this follows from applying the
// implicit function theorem to dG/dx = 0 of Eq. 2, with y from Eq. 3 and the
// velocity update of Eq. 6).
//
// Positions are displacements u = x - X (tape rows included).  The sweep
// evaluates the tet through its current edge vectors (see k_adj_sweep), the
// parameter gradient from F = I + D as in the forward sweep.
// For a recorded step t with end positions x_{t+1} and H = M/h^2 + d2E/dx2
// (+ the ground and wall penalty Hessians), going backwards:
//   r = xbar_{t+1} + vbar_{t+1} / h,   H lam = r   (colour-ordered block GS),
//   xbar_t = M/h^2 lam - vbar_{t+1}/h,  vbar_t = M/h lam,
//   d L / d log E_j -= sum_{i in tet j} lam_i . dE_j/dx_i.
// The block Gauss-Seidel sweep reuses the forward's slot layout: per slot it
// forms the tet's off-diagonal blocks H_ik (k = the three other vertices)
// applied to lam_k, then one lane solves the 3x3 system for lam_i with the
// diagonal block H_ii that k_adj_diag computed once for the step.  Vertices
// of one colour share no tet, so the in-place update is an exact
// Gauss-Seidel sweep.  Each vertex's recorded displacement and lam sit in one
// 32-byte record (Dev::lam), so a neighbour costs one 256-bit gather.
#include "vbd_kernels.h"

#include <algorithm>

namespace vbd {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) {
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// F v with F given by its columns f0, f1, f2
__device__ __forceinline__ float3 mulF(float3 f0, float3 f1, float3 f2, float3 v) {
    return make_float3(v.x * f0.x + v.y * f1.x + v.z * f2.x, v.x * f0.y + v.y * f1.y + v.z * f2.y,
                       v.x * f0.z + v.y * f1.z + v.z * f2.z);
}

// Dev::lam holds a 32-byte record per vertex: [2i] the recorded displacement
// of the step being solved, [2i+1] lam_i.  One 256-bit load brings both
// (non-coherent path: a colour pass reads only other colours' records, and
// the cache does not outlive the launch), with an L2 evict-last policy so
// that the records stay in L2 while the slot stream passes.
__device__ __forceinline__ void ld_xlam(const float4 *rec, float3 &x, float3 &l) {
    float xw, lw;
    asm("{\n\t.reg .b64 pol;\n\tcreatepolicy.fractional.L2::evict_last.b64 pol, 1.0;\n\t"
        "ld.global.nc.L2::cache_hint.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], pol;\n\t}"
        : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(xw), "=f"(l.x), "=f"(l.y), "=f"(l.z), "=f"(lw)
        : "l"(rec));
}

// 1 / det_g of a slot in one MUFU instruction (relative error below 2^-22;
// det_g of a valid tet is far from zero and from the denormal range).  The
// volume V = |1 / det_g| / 6 comes from the same value.
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int L>
__device__ __forceinline__ float sub_reduce(float v) {
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

struct AdjAcc {
    float q0, q1, q2;                      // sum_k H_ik lam_k (off-diagonal part)
};

// F = I + D restricted to what the adjoint needs: D from the displacements
// (columns D0..D2), tr D, cof(D) columns q0..q2 and J - 1.
struct DForm {
    float3 D0, D1, D2, q0, q1, q2;
    float tr, jm1;
    // cof(F) v = v + (tr D) v - D^T v + cof(D) v
    __device__ __forceinline__ float3 cof(float3 v) const {
        return make_float3(v.x + tr * v.x - dot(D0, v) + v.x * q0.x + v.y * q1.x + v.z * q2.x,
                           v.y + tr * v.y - dot(D1, v) + v.x * q0.y + v.y * q1.y + v.z * q2.y,
                           v.z + tr * v.z - dot(D2, v) + v.x * q0.z + v.y * q1.z + v.z * q2.z);
    }
    // D v
    __device__ __forceinline__ float3 dmul(float3 v) const { return mulF(D0, D1, D2, v); }
};

__device__ __forceinline__ DForm make_dform(const float3 d[3], const float3 g[3]) {
    DForm f;
    f.D0 = make_float3(0.f, 0.f, 0.f);
    f.D1 = f.D0;
    f.D2 = f.D0;
    for (int k = 0; k < 3; ++k) {
        f.D0.x += d[k].x * g[k].x; f.D0.y += d[k].y * g[k].x; f.D0.z += d[k].z * g[k].x;
        f.D1.x += d[k].x * g[k].y; f.D1.y += d[k].y * g[k].y; f.D1.z += d[k].z * g[k].y;
        f.D2.x += d[k].x * g[k].z; f.D2.y += d[k].y * g[k].z; f.D2.z += d[k].z * g[k].z;
    }
    f.tr = f.D0.x + f.D1.y + f.D2.z;
    const float m2 = (f.D0.x * f.D1.y - f.D1.x * f.D0.y) + (f.D0.x * f.D2.z - f.D2.x * f.D0.z) +
                     (f.D1.y * f.D2.z - f.D2.y * f.D1.z);
    f.q0 = cross(f.D1, f.D2);
    f.q1 = cross(f.D2, f.D0);
    f.q2 = cross(f.D0, f.D1);
    f.jm1 = f.tr + m2 + dot(f.D0, f.q0);
    return f;
}

// H_ii of every free vertex at the step's recorded positions, once per step:
// sum over its tets of V (mu |g_i|^2 I + lam c_i c_i^T) with c_i = cof(F) g_i
// in the edge form of k_adj_sweep (below), plus m_i/h^2 I and the ground and
// wall penalty Hessians (Eq. 12, Sec. 3.4).  It does not change while the
// sweeps solve for lam, so they read it from Dev::hdiag (h00 h01 h02 h11 |
// h12 h22) instead of rebuilding it from every slot at every sweep.
template <int L>
__global__ void __launch_bounds__(128, 8) k_adj_diag(Dev d, const float4 *__restrict__ xs, SweepParams p) {
    const int lane = threadIdx.x & (L - 1);
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int vi = p.vbegin + (int)(gt / L);
    const bool active = vi < p.vend;
    float3 ui = make_float3(0.f, 0.f, 0.f);
    int s0 = 0, s1 = 0;
    if (active) {
        ui = f3(xs[vi]);
        s0 = d.slot_off[vi];
        s1 = d.slot_off[vi + 1];
    }
    const float2 vm = (active && !p.per_tet_mat) ? __ldg(d.vmat + vi) : make_float2(0.f, 0.f);
    float h00 = 0.f, h01 = 0.f, h02 = 0.f, h11 = 0.f, h12 = 0.f, h22 = 0.f;
    for (int s = s0 + lane; s < s1; s += L) {
        const int4 r0 = __ldcs(d.s0 + s);
        const float4 r1 = __ldcs(d.s1 + s);
        const float4 r2 = __ldcs(d.s2 + s);
        const float3 ga = make_float3(__int_as_float(r0.w), r1.x, r1.y);
        const float3 gb = make_float3(r1.z, r1.w, r2.x);
        const float3 gc = make_float3(r2.y, r2.z, r2.w);
        const float3 da = sub(f3(__ldg(xs + r0.x)), ui), db = sub(f3(__ldg(xs + r0.y)), ui),
                     dc = sub(f3(__ldg(xs + r0.z)), ui);
        const float3 gbc = cross(gb, gc);
        const float detg = dot(ga, gbc);
        const float inv = rcp_fast(detg);
        const float3 ea = gbc, eb = cross(gc, ga), ec = cross(ga, gb);
        const float3 ya = make_float3(fmaf(ea.x, inv, da.x), fmaf(ea.y, inv, da.y), fmaf(ea.z, inv, da.z));
        const float3 yb = make_float3(fmaf(eb.x, inv, db.x), fmaf(eb.y, inv, db.y), fmaf(eb.z, inv, db.z));
        const float3 yc = make_float3(fmaf(ec.x, inv, dc.x), fmaf(ec.y, inv, dc.y), fmaf(ec.z, inv, dc.z));
        const float3 Xa = cross(yb, yc), Xb = cross(yc, ya), Xc = cross(ya, yb);
        const float V = fabsf(inv) * (1.0f / 6.0f);
        float2 mat = vm;
        if (p.per_tet_mat) {
            const int j = __ldcs(d.slot_tet + s);
            mat = make_float2(__ldg(d.tet_mu + j), __ldg(d.tet_lam + j));
        }
        const float Vmu = V * mat.x, Vlam = V * mat.y;
        const float3 ci = make_float3(-detg * (Xa.x + Xb.x + Xc.x), -detg * (Xa.y + Xb.y + Xc.y),
                                      -detg * (Xa.z + Xb.z + Xc.z));
        const float3 gi = make_float3(-(ga.x + gb.x + gc.x), -(ga.y + gb.y + gc.y), -(ga.z + gb.z + gc.z));
        const float dd = Vmu * dot(gi, gi);
        h00 += dd + Vlam * ci.x * ci.x;
        h11 += dd + Vlam * ci.y * ci.y;
        h22 += dd + Vlam * ci.z * ci.z;
        h01 += Vlam * ci.x * ci.y;
        h02 += Vlam * ci.x * ci.z;
        h12 += Vlam * ci.y * ci.z;
    }
    h00 = sub_reduce<L>(h00); h01 = sub_reduce<L>(h01); h02 = sub_reduce<L>(h02);
    h11 = sub_reduce<L>(h11); h12 = sub_reduce<L>(h12); h22 = sub_reduce<L>(h22);
    if (!(active && lane == 0)) return;
    const float mh2 = d.mass[vi] * p.inv_h2;
    h00 += mh2;
    h11 += mh2;
    h22 += mh2;
    if (p.n_planes > 0) {  // ground and wall penalty Hessians (Eq. 12, Sec. 3.4)
        const float4 X = d.rest[vi];
        for (int k = 0; k < p.n_planes; ++k) {
            const float4 pl = p.planes[k];
            const float pen = pl.w - (pl.x * (X.x + ui.x) + pl.y * (X.y + ui.y) + pl.z * (X.z + ui.z));
            if (pen > 0.f) {
                h00 += p.kc * pl.x * pl.x; h11 += p.kc * pl.y * pl.y; h22 += p.kc * pl.z * pl.z;
                h01 += p.kc * pl.x * pl.y; h02 += p.kc * pl.x * pl.z; h12 += p.kc * pl.y * pl.z;
            }
        }
    }
    d.hdiag[2 * vi] = make_float4(h00, h01, h02, h11);
    d.hdiag[2 * vi + 1] = make_float4(h12, h22, 0.f, 0.f);
}

// Per slot the sweep needs only products of H with lam, never P(F) itself, so
// it works with the tet's current edge vectors y_k = x_k - x_i (k = a, b, c,
// the slot's three other vertices) instead of F = I + D.  With B the inverse
// rest edge matrix (rows g_a, g_b, g_c), det_g = det B, and the rest edges
// e_k = (g_{k+1} x g_{k+2}) / det_g (cyclic; the columns of B^-1):
//   J          = det_g  y_a . (y_b x y_c)
//   cof(F) g_a = det_g (y_b x y_c), cyclic, so c_i = cof(F) g_i
//              = -det_g (y_b - y_a) x (y_c - y_a)
//   cof F : dF = det_g sum_k lam_k . (y_{k+1} x y_{k+2})        (dF = sum_k lam_k g_k^T)
//   dcof(F)[dF] g_i = -det_g [(lam_b - lam_a) x (y_c - y_a) + (y_b - y_a) x (lam_c - lam_a)]
//   dF g_i     = sum_k lam_k (g_k . g_i)
// and sum_k H_ik lam_k = V [mu dF g_i + lam (cof F : dF) c_i + lam (J - alpha) dcof(F)[dF] g_i].
// J - 1 now comes from a determinant near 1, but only J - alpha = (J - 1) -
// mu/lam enters, whose size is set by mu/lam, so its rounding stays at the
// FP32 level; no step takes a difference of nearly equal O(1) numbers.
// MODE 0: one Gauss-Seidel update of lam_i; MODE 1: r - (H lam)_i of the
// subspace-constrained vertices into rhs (lam unchanged); MODE 2: over all
// free vertices at once, max_i |r_i - (H lam)_i| (projected onto the
// subspace of a constrained vertex) and max_i |r_i| into res_out[0], [1]
// (FP64, atomic max of the non-negative doubles' bit patterns).
// launched with 128 threads, VBD_ADJ_MIN_BLOCKS resident CTAs per SM (8:
// held to 64 registers)
#ifndef VBD_ADJ_MIN_BLOCKS
#define VBD_ADJ_MIN_BLOCKS 8
#endif
template <int L, int MODE>
__device__ __forceinline__ void adj_body(const Dev &d, const float4 *__restrict__ xs, const SweepParams &p,
                                         long long gt, float &res_acc, float &r_acc) {
    const int lane = threadIdx.x & (L - 1);
    const int vi = p.vbegin + (int)(gt / L);
    const bool active = vi < p.vend;
    float3 ui = make_float3(0.f, 0.f, 0.f);
    int s0 = 0, s1 = 0;
    if (active) {
        ui = f3(xs[vi]);
        s0 = d.slot_off[vi];
        s1 = d.slot_off[vi + 1];
    }
    const float2 vm = (active && !p.per_tet_mat) ? __ldg(d.vmat + vi) : make_float2(0.f, 0.f);
    AdjAcc a = {0.f, 0.f, 0.f};
    for (int s = s0 + lane; s < s1; s += L) {
        const int4 r0 = __ldcs(d.s0 + s);
        const float4 r1 = __ldcs(d.s1 + s);
        const float4 r2 = __ldcs(d.s2 + s);
        const float3 ga = make_float3(__int_as_float(r0.w), r1.x, r1.y);
        const float3 gb = make_float3(r1.z, r1.w, r2.x);
        const float3 gc = make_float3(r2.y, r2.z, r2.w);
        float3 xa, xb, xc, la, lb, lc;  // other colours only
        ld_xlam(d.lam + 2 * (size_t)r0.x, xa, la);
        ld_xlam(d.lam + 2 * (size_t)r0.y, xb, lb);
        ld_xlam(d.lam + 2 * (size_t)r0.z, xc, lc);
        const float3 da = sub(xa, ui), db = sub(xb, ui), dc = sub(xc, ui);
        const float3 gbc = cross(gb, gc);
        const float detg = dot(ga, gbc);
        const float inv = rcp_fast(detg);
        // current edges y_k = e_k + (u_k - u_i)
        const float3 ea = gbc, eb = cross(gc, ga), ec = cross(ga, gb);
        const float3 ya = make_float3(fmaf(ea.x, inv, da.x), fmaf(ea.y, inv, da.y), fmaf(ea.z, inv, da.z));
        const float3 yb = make_float3(fmaf(eb.x, inv, db.x), fmaf(eb.y, inv, db.y), fmaf(eb.z, inv, db.z));
        const float3 yc = make_float3(fmaf(ec.x, inv, dc.x), fmaf(ec.y, inv, dc.y), fmaf(ec.z, inv, dc.z));
        const float3 Xa = cross(yb, yc), Xb = cross(yc, ya), Xc = cross(ya, yb);
        const float V = fabsf(inv) * (1.0f / 6.0f);
        float2 mat = vm;
        if (p.per_tet_mat) {
            const int j = __ldcs(d.slot_tet + s);
            mat = make_float2(__ldg(d.tet_mu + j), __ldg(d.tet_lam + j));
        }
        const float Vmu = V * mat.x, Vlam = V * mat.y;
        const float J = detg * dot(ya, Xa);
        const float3 ci = make_float3(-detg * (Xa.x + Xb.x + Xc.x), -detg * (Xa.y + Xb.y + Xc.y),
                                      -detg * (Xa.z + Xb.z + Xc.z));
        const float sc = detg * (dot(la, Xa) + dot(lb, Xb) + dot(lc, Xc));
        const float3 lba = sub(lb, la), lca = sub(lc, la), yba = sub(yb, ya), yca = sub(yc, ya);
        const float3 w1 = cross(lba, yca), w2 = cross(yba, lca);
        const float3 gi = make_float3(-(ga.x + gb.x + gc.x), -(ga.y + gb.y + gc.y), -(ga.z + gb.z + gc.z));
        const float pa = dot(ga, gi), pb = dot(gb, gi), pc = dot(gc, gi);
        const float3 dFg = make_float3(la.x * pa + lb.x * pb + lc.x * pc, la.y * pa + lb.y * pb + lc.y * pc,
                                       la.z * pa + lb.z * pb + lc.z * pc);
        const float kJ = -(Vlam * (J - 1.0f) - Vmu) * detg;  // V lam (J - alpha) times -det_g of w
        const float ks = Vlam * sc;
        a.q0 += Vmu * dFg.x + ks * ci.x + kJ * (w1.x + w2.x);
        a.q1 += Vmu * dFg.y + ks * ci.y + kJ * (w1.y + w2.y);
        a.q2 += Vmu * dFg.z + ks * ci.z + kJ * (w1.z + w2.z);
    }
    a.q0 = sub_reduce<L>(a.q0); a.q1 = sub_reduce<L>(a.q1); a.q2 = sub_reduce<L>(a.q2);
    const bool owner = active && lane == 0;
    float res_max = 0.f, r_max = 0.f;
    if (owner) {
        const float4 r = d.rhs[vi];
        const float b0 = r.x - a.q0, b1 = r.y - a.q1, b2 = r.z - a.q2;
        const float4 hA = d.hdiag[2 * vi], hB = d.hdiag[2 * vi + 1];  // H_ii of k_adj_diag
        const float h00 = hA.x, h01 = hA.y, h02 = hA.z, h11 = hA.w, h12 = hB.x, h22 = hB.y;
        const int sub = p.n_sub > 0 ? d.sub_id[vi] : -1;
        if (MODE != 0) {
            // r - (H lam)_i = b - H_ii lam_i
            const float4 l = d.lam[2 * (size_t)vi + 1];
            float e0 = b0 - (h00 * l.x + h01 * l.y + h02 * l.z), e1 = b1 - (h01 * l.x + h11 * l.y + h12 * l.z),
                  e2 = b2 - (h02 * l.x + h12 * l.y + h22 * l.z);
            if (MODE == 1) {
                // the part of xbar that follows x_t across a constrained vertex's fixed directions
                if (sub >= 0) d.rhs[vi] = make_float4(e0, e1, e2, 0.f);
            } else {
                if (sub >= 0) {  // only Q^T (r - H lam) is solved for: project onto span(Q)
                    const float4 qa = d.sub_q[2 * sub], qb = d.sub_q[2 * sub + 1];
                    const float z0 = qa.x * e0 + qa.y * e1 + qa.z * e2;
                    const float z1 = qa.w < 1.5f ? 0.f : qb.x * e0 + qb.y * e1 + qb.z * e2;
                    e0 = qa.x * z0 + qb.x * z1;
                    e1 = qa.y * z0 + qb.y * z1;
                    e2 = qa.z * z0 + qb.z * z1;
                }
                // a non-finite component reports as +inf (fmaxf alone would drop a NaN)
                res_max = (isfinite(e0) && isfinite(e1) && isfinite(e2))
                              ? fmaxf(fabsf(e0), fmaxf(fabsf(e1), fabsf(e2))) : INFINITY;
                r_max = (isfinite(r.x) && isfinite(r.y) && isfinite(r.z))
                            ? fmaxf(fabsf(r.x), fmaxf(fabsf(r.y), fabsf(r.z))) : INFINITY;
            }
        } else {
            float l0, l1, l2;
            if (sub >= 0) {
                // reduced block (Sec. 3.4): lam_i = Q (Q^T H_ii Q)^-1 Q^T b
                const float4 qa = d.sub_q[2 * sub], qb = d.sub_q[2 * sub + 1];
                const float ha0 = h00 * qa.x + h01 * qa.y + h02 * qa.z;
                const float ha1 = h01 * qa.x + h11 * qa.y + h12 * qa.z;
                const float ha2 = h02 * qa.x + h12 * qa.y + h22 * qa.z;
                const float A00 = qa.x * ha0 + qa.y * ha1 + qa.z * ha2;
                const float c0 = qa.x * b0 + qa.y * b1 + qa.z * b2;
                float z0, z1 = 0.f;
                if (qa.w < 1.5f) {
                    z0 = c0 / A00;
                } else {
                    const float A01 = qb.x * ha0 + qb.y * ha1 + qb.z * ha2;
                    const float A11 = qb.x * (h00 * qb.x + h01 * qb.y + h02 * qb.z) +
                                      qb.y * (h01 * qb.x + h11 * qb.y + h12 * qb.z) +
                                      qb.z * (h02 * qb.x + h12 * qb.y + h22 * qb.z);
                    const float c1 = qb.x * b0 + qb.y * b1 + qb.z * b2;
                    const float inv2 = 1.f / (A00 * A11 - A01 * A01);
                    z0 = (A11 * c0 - A01 * c1) * inv2;
                    z1 = (A00 * c1 - A01 * c0) * inv2;
                }
                l0 = qa.x * z0 + qb.x * z1;
                l1 = qa.y * z0 + qb.y * z1;
                l2 = qa.z * z0 + qb.z * z1;
            } else {
                const float a00 = h11 * h22 - h12 * h12, a01 = h02 * h12 - h01 * h22, a02 = h01 * h12 - h02 * h11;
                const float a11 = h00 * h22 - h02 * h02, a12 = h01 * h02 - h00 * h12, a22 = h00 * h11 - h01 * h01;
                const float det = h00 * a00 + h01 * a01 + h02 * a02;
                const float invd = 1.f / det;
                l0 = (a00 * b0 + a01 * b1 + a02 * b2) * invd;
                l1 = (a01 * b0 + a11 * b1 + a12 * b2) * invd;
                l2 = (a02 * b0 + a12 * b1 + a22 * b2) * invd;
            }
            if (!(isfinite(l0) && isfinite(l1) && isfinite(l2)))
                atomicAdd(d.counters + 0, 1ull);
            else
                d.lam[2 * (size_t)vi + 1] = make_float4(l0, l1, l2, 0.f);
        }
    }
    if (MODE == 2) {  // running maxima of this thread over its grid-stride turns
        res_acc = fmaxf(res_acc, res_max);
        r_acc = fmaxf(r_acc, r_max);
    }
}

// Persistent grid: 148 x resident CTAs walk the colour's vertices with a
// grid stride (every thread of a CTA makes the same number of turns, so the
// warp-wide reduction of mode 2 sees full warps).  MODE = SweepParams::adj_residual,
// one instance each, so that the sweep (mode 0) carries no residual code.
template <int L, int MODE>
__global__ void __launch_bounds__(128, VBD_ADJ_MIN_BLOCKS) k_adj_sweep(Dev d, const float4 *__restrict__ xs, SweepParams p,
                                                      double *res_out, long long threads) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    float res_acc = 0.f, r_acc = 0.f;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < threads; base += stride)
        adj_body<L, MODE>(d, xs, p, base + threadIdx.x, res_acc, r_acc);
    if (MODE == 2) {
        // every thread of the CTA made the same number of turns, so the whole
        // warp is here: one warp reduction and two atomics per warp
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            res_acc = fmaxf(res_acc, __shfl_xor_sync(FULL, res_acc, off));
            r_acc = fmaxf(r_acc, __shfl_xor_sync(FULL, r_acc, off));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMax((unsigned long long *)res_out, (unsigned long long)__double_as_longlong((double)res_acc));
            atomicMax((unsigned long long *)res_out + 1, (unsigned long long)__double_as_longlong((double)r_acc));
        }
    }
}

// xbar, vbar <- seed; lam <- 0; gtheta <- 0 is done by the host (memset).
__global__ void k_adj_seed(Dev d, const float *dL_dx, int n) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int i = d.new_of_orig[o];
    d.xbar[i] = make_float4(dL_dx[3 * o], dL_dx[3 * o + 1], dL_dx[3 * o + 2], 0.f);
    d.vbar[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// r = xbar + vbar / h on free vertices; lam = 0 everywhere (pinned stay 0)
// beside the step's recorded displacement in the vertex's (x, lam) record.
__global__ void k_adj_rhs(Dev d, const float4 *__restrict__ xs, int n, int n_free, float inv_h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    d.lam[2 * (size_t)i] = xs[i];
    d.lam[2 * (size_t)i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i >= n_free) return;
    const float4 xb = d.xbar[i], vb = d.vbar[i];
    d.rhs[i] = make_float4(xb.x + vb.x * inv_h, xb.y + vb.y * inv_h, xb.z + vb.z * inv_h, 0.f);
}

// xbar_t = M/h^2 lam - vbar/h (+ r - (H lam)_i, stored in rhs, for a
// subspace-constrained vertex), vbar_t = M/h lam (free vertices; pinned 0)
__global__ void k_adj_post_verts(Dev d, int n, int n_free, float h, int has_sub) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i >= n_free) {
        d.xbar[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        d.vbar[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float m = d.mass[i];
    const float4 l = d.lam[2 * (size_t)i + 1], vb = d.vbar[i];
    const float a = m / (h * h), b = m / h, c = 1.f / h;
    float4 xb = make_float4(a * l.x - c * vb.x, a * l.y - c * vb.y, a * l.z - c * vb.z, 0.f);
    if (has_sub && d.sub_id[i] >= 0) {
        const float4 e = d.rhs[i];
        xb.x += e.x; xb.y += e.y; xb.z += e.z;
    }
    d.xbar[i] = xb;
    d.vbar[i] = make_float4(b * l.x, b * l.y, b * l.z, 0.f);
}

// gtheta_j -= sum_k lam_k . V P g_k at the recorded positions (dE_j/dlogE_j = E_j),
// V P g_k = V mu (D g_k - c'_k) + V lam (J - 1) (g_k + c'_k),  c'_k = cof(F) g_k - g_k
__global__ void k_adj_post_tets(Dev d, const float4 *__restrict__ xs, int n_tets) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_tets) return;
    const int4 t = d.tet_v[j];
    const int id[4] = {t.x, t.y, t.z, t.w};
    const float *B = d.tet_B + 9 * (size_t)j;
    float3 g[3];
    g[0] = make_float3(B[0], B[1], B[2]);
    g[1] = make_float3(B[3], B[4], B[5]);
    g[2] = make_float3(B[6], B[7], B[8]);
    const float3 g0 = make_float3(-(g[0].x + g[1].x + g[2].x), -(g[0].y + g[1].y + g[2].y),
                                  -(g[0].z + g[1].z + g[2].z));
    const float3 u0 = f3(xs[id[0]]);
    float3 e[3];
    for (int k = 0; k < 3; ++k) e[k] = sub(f3(xs[id[k + 1]]), u0);
    const DForm F = make_dform(e, g);
    const float mu = d.tet_mu[j], lam = d.tet_lam[j], V = d.tet_V[j];
    float acc = 0.f;
    for (int k = 0; k < 4; ++k) {
        const float3 gk = k == 0 ? g0 : g[k - 1];
        const float3 l = f3(d.lam[2 * (size_t)id[k] + 1]);
        const float3 c = F.cof(gk);                  // g_k + c'_k
        const float3 Dg = F.dmul(gk);
        const float3 cp = make_float3(c.x - gk.x, c.y - gk.y, c.z - gk.z);
        acc += V * (mu * (dot(Dg, l) - dot(cp, l)) + lam * F.jm1 * dot(c, l));
    }
    d.gtheta[j] -= acc;
}

__global__ void k_adj_out(Dev d, float *dL_dv0, int n) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const float4 a = d.vbar[d.new_of_orig[o]];
    dL_dv0[3 * o] = a.x;
    dL_dv0[3 * o + 1] = a.y;
    dL_dv0[3 * o + 2] = a.z;
}

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// SMs x resident CTAs of k_adj_sweep<lanes, MODE> at this block size on the
// current device (0 if the query fails: the launch then covers every vertex at once)
template <int MODE>
long long adj_persist_grid(int lanes, int block) {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    cudaError_t e;
    switch (lanes) {
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adj_sweep<4, MODE>, block, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adj_sweep<8, MODE>, block, 0); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adj_sweep<16, MODE>, block, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adj_sweep<32, MODE>, block, 0); break;
    }
    if (e != cudaSuccess || occ < 1) return 0;
    return (long long)sms * occ;
}

template <int MODE>
void launch_adj_sweep_mode(const Dev &d, const float4 *xs, const SweepParams &p, int lanes, int block,
                           long long threads, cudaStream_t s, double *res_out) {
    const long long need = (long long)blocks_for(threads, block);
    const long long cap = adj_persist_grid<MODE>(lanes, block);
    const unsigned grid = (unsigned)(cap > 0 ? std::min(need, cap) : need);
    switch (lanes) {
    case 4: k_adj_sweep<4, MODE><<<grid, block, 0, s>>>(d, xs, p, res_out, threads); break;
    case 8: k_adj_sweep<8, MODE><<<grid, block, 0, s>>>(d, xs, p, res_out, threads); break;
    case 16: k_adj_sweep<16, MODE><<<grid, block, 0, s>>>(d, xs, p, res_out, threads); break;
    default: k_adj_sweep<32, MODE><<<grid, block, 0, s>>>(d, xs, p, res_out, threads); break;
    }
}

}  // namespace

void launch_adj_seed(const Dev &d, const float *dL_dx, int n, cudaStream_t s) {
    k_adj_seed<<<blocks_for(n, 256), 256, 0, s>>>(d, dL_dx, n);
}

void launch_adj_rhs(const Dev &d, const float4 *xs, int n, int n_free, float inv_h, cudaStream_t s) {
    k_adj_rhs<<<blocks_for(n, 256), 256, 0, s>>>(d, xs, n, n_free, inv_h);
}

void launch_adj_sweep(const Dev &d, const float4 *xs, const SweepParams &p, int lanes, int block,
                      cudaStream_t s, double *res_out) {
    const long long threads = (long long)(p.vend - p.vbegin) * lanes;
    if (threads <= 0) return;
    switch (p.adj_residual) {
    case 0: launch_adj_sweep_mode<0>(d, xs, p, lanes, block, threads, s, res_out); break;
    case 1: launch_adj_sweep_mode<1>(d, xs, p, lanes, block, threads, s, res_out); break;
    default: launch_adj_sweep_mode<2>(d, xs, p, lanes, block, threads, s, res_out); break;
    }
}

void launch_adj_diag(const Dev &d, const float4 *xs, const SweepParams &p, int lanes, int block, cudaStream_t s) {
    const long long threads = (long long)(p.vend - p.vbegin) * lanes;
    if (threads <= 0) return;
    const unsigned grid = blocks_for(threads, block);
    switch (lanes) {
    case 4: k_adj_diag<4><<<grid, block, 0, s>>>(d, xs, p); break;
    case 8: k_adj_diag<8><<<grid, block, 0, s>>>(d, xs, p); break;
    case 16: k_adj_diag<16><<<grid, block, 0, s>>>(d, xs, p); break;
    default: k_adj_diag<32><<<grid, block, 0, s>>>(d, xs, p); break;
    }
}

void launch_adj_post(const Dev &d, const float4 *xs, int n, int n_free, int n_tets, float h, bool has_sub,
                     cudaStream_t s) {
    // tets first: they read lam, which the vertex pass does not change
    k_adj_post_tets<<<blocks_for(n_tets, 256), 256, 0, s>>>(d, xs, n_tets);
    k_adj_post_verts<<<blocks_for(n, 256), 256, 0, s>>>(d, n, n_free, h, has_sub ? 1 : 0);
}

void launch_adj_out(const Dev &d, float *dL_dlogE, float *dL_dv0, int n, int n_tets, cudaStream_t s) {
    if (dL_dv0) k_adj_out<<<blocks_for(n, 256), 256, 0, s>>>(d, dL_dv0, n);
    if (dL_dlogE) cudaMemcpyAsync(dL_dlogE, d.gtheta, sizeof(float) * (size_t)n_tets,
                                  cudaMemcpyDeviceToDevice, s);
}

}  // namespace vbd

// vbd_adjoint.cu -- reverse pass through converged VBD steps (no paper
// counterpart: the paper has no derivatives; this follows from applying the
// implicit function theorem to dG/dx = 0 of Eq. 2, with y from Eq. 3 and the
// velocity update of Eq. 6).
//
// Positions are displacements u = x - X (tape rows included), and the element
// is evaluated from F = I + D as in the forward sweep.
// For a recorded step t with end positions x_{t+1} and H = M/h^2 + d2E/dx2
// (+ the ground and wall penalty Hessians), going backwards:
//   r = xbar_{t+1} + vbar_{t+1} / h,   H lam = r   (colour-ordered block GS),
//   xbar_t = M/h^2 lam - vbar_{t+1}/h,  vbar_t = M/h lam,
//   d L / d log E_j -= sum_{i in tet j} lam_i . dE_j/dx_i.
// The block Gauss-Seidel sweep reuses the forward's slot layout: per slot it
// forms the tet's off-diagonal blocks H_ik (k = the three other vertices)
// applied to lam_k, and the vertex's diagonal block, then one lane solves
// the 3x3 system for lam_i.  Vertices of one colour share no tet, so the
// in-place update is an exact Gauss-Seidel sweep.
#include "vbd_kernels.h"

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

template <int L>
__device__ __forceinline__ float sub_reduce(float v) {
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

struct AdjAcc {
    float q0, q1, q2;                      // sum_k H_ik lam_k (off-diagonal part)
    float h00, h01, h02, h11, h12, h22;    // elastic diagonal block
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

template <int L>
// launched with 128 threads and held to 64 registers (8 CTAs per SM; a 12-byte
// spill), measured 1.7 % faster than 70 registers at 7 CTAs
__global__ void __launch_bounds__(128, 8) k_adj_sweep(Dev d, const float4 *__restrict__ xs, SweepParams p) {
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
    AdjAcc a = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int s = s0 + lane; s < s1; s += L) {
        const int4 r0 = __ldcs(d.s0 + s);
        const float4 r1 = __ldcs(d.s1 + s);
        const float4 r2 = __ldcs(d.s2 + s);
        const int nb[3] = {r0.x, r0.y, r0.z};
        float3 g[3];
        g[0] = make_float3(__int_as_float(r0.w), r1.x, r1.y);
        g[1] = make_float3(r1.z, r1.w, r2.x);
        g[2] = make_float3(r2.y, r2.z, r2.w);
        // tet volume from the gradients; mu, lambda of the vertex, or of the
        // tet when materials differ around vertices (after vbd_set_log_young)
        const float V = __frcp_rn(6.0f * fabsf(dot(g[0], cross(g[1], g[2]))));
        float2 mat = vm;
        if (p.per_tet_mat) {
            const int j = __ldcs(d.slot_tet + s);
            mat = make_float2(__ldg(d.tet_mu + j), __ldg(d.tet_lam + j));
        }
        const float Vmu = V * mat.x, Vlam = V * mat.y;
        const float3 gi = make_float3(-(g[0].x + g[1].x + g[2].x), -(g[0].y + g[1].y + g[2].y),
                                      -(g[0].z + g[1].z + g[2].z));
        float3 e[3], lk[3];
        for (int k = 0; k < 3; ++k) {
            e[k] = sub(f3(__ldg(xs + nb[k])), ui);
            lk[k] = f3(d.lam[nb[k]]);  // written by other colours' launches only
        }
        const DForm F = make_dform(e, g);
        const float3 ci = F.cof(gi);
        const float kJ = Vlam * F.jm1 - Vmu;  // V lam (J - alpha)
        // sum_k H_ik lam_k = V [mu dF g_i + lam (cof F : dF) c_i + lam (J - alpha) dcof(F)[dF] g_i]
        // with the direction dF = sum_k lam_k g_k^T (columns dF0..dF2); the last
        // term equals sum_k (F (g_k x g_i)) x lam_k, the skew part of the blocks.
        float3 dF0 = make_float3(0.f, 0.f, 0.f), dF1 = dF0, dF2 = dF0;
        for (int k = 0; k < 3; ++k) {
            dF0.x += lk[k].x * g[k].x; dF0.y += lk[k].y * g[k].x; dF0.z += lk[k].z * g[k].x;
            dF1.x += lk[k].x * g[k].y; dF1.y += lk[k].y * g[k].y; dF1.z += lk[k].z * g[k].y;
            dF2.x += lk[k].x * g[k].z; dF2.y += lk[k].y * g[k].z; dF2.z += lk[k].z * g[k].z;
        }
        const float3 dFg = mulF(dF0, dF1, dF2, gi);
        // cof F : dF, with cof(F) e_c = (1 + tr D) e_c - D^T e_c + cof(D) e_c
        const float trdF = dF0.x + dF1.y + dF2.z;
        const float trdFD = dF0.x * F.D0.x + dF0.y * F.D1.x + dF0.z * F.D2.x +
                            dF1.x * F.D0.y + dF1.y * F.D1.y + dF1.z * F.D2.y +
                            dF2.x * F.D0.z + dF2.y * F.D1.z + dF2.z * F.D2.z;
        const float sc = (1.f + F.tr) * trdF - trdFD + dot(dF0, F.q0) + dot(dF1, F.q1) + dot(dF2, F.q2);
        // dcof(F)[dF] g_i: cof F has columns f1 x f2, f2 x f0, f0 x f1 (f_c = e_c + D_c)
        const float3 f0 = make_float3(1.f + F.D0.x, F.D0.y, F.D0.z);
        const float3 f1 = make_float3(F.D1.x, 1.f + F.D1.y, F.D1.z);
        const float3 f2 = make_float3(F.D2.x, F.D2.y, 1.f + F.D2.z);
        const float3 c0 = cross(dF1, f2), c0b = cross(f1, dF2);
        const float3 c1 = cross(dF2, f0), c1b = cross(f2, dF0);
        const float3 c2 = cross(dF0, f1), c2b = cross(f0, dF1);
        const float3 w = make_float3(gi.x * (c0.x + c0b.x) + gi.y * (c1.x + c1b.x) + gi.z * (c2.x + c2b.x),
                                     gi.x * (c0.y + c0b.y) + gi.y * (c1.y + c1b.y) + gi.z * (c2.y + c2b.y),
                                     gi.x * (c0.z + c0b.z) + gi.y * (c1.z + c1b.z) + gi.z * (c2.z + c2b.z));
        float3 q = make_float3(Vmu * dFg.x + kJ * w.x, Vmu * dFg.y + kJ * w.y, Vmu * dFg.z + kJ * w.z);
        q.x += Vlam * ci.x * sc; q.y += Vlam * ci.y * sc; q.z += Vlam * ci.z * sc;
        a.q0 += q.x; a.q1 += q.y; a.q2 += q.z;
        const float dd = Vmu * dot(gi, gi);
        a.h00 += dd + Vlam * ci.x * ci.x;
        a.h11 += dd + Vlam * ci.y * ci.y;
        a.h22 += dd + Vlam * ci.z * ci.z;
        a.h01 += Vlam * ci.x * ci.y;
        a.h02 += Vlam * ci.x * ci.z;
        a.h12 += Vlam * ci.y * ci.z;
    }
    a.q0 = sub_reduce<L>(a.q0); a.q1 = sub_reduce<L>(a.q1); a.q2 = sub_reduce<L>(a.q2);
    a.h00 = sub_reduce<L>(a.h00); a.h01 = sub_reduce<L>(a.h01); a.h02 = sub_reduce<L>(a.h02);
    a.h11 = sub_reduce<L>(a.h11); a.h12 = sub_reduce<L>(a.h12); a.h22 = sub_reduce<L>(a.h22);
    if (!(active && lane == 0)) return;
    const float mh2 = d.mass[vi] * p.inv_h2;
    const float4 r = d.rhs[vi];
    const float b0 = r.x - a.q0, b1 = r.y - a.q1, b2 = r.z - a.q2;
    float h00 = a.h00 + mh2, h11 = a.h11 + mh2, h22 = a.h22 + mh2, h01 = a.h01, h02 = a.h02, h12 = a.h12;
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
    const int sub = p.n_sub > 0 ? d.sub_id[vi] : -1;
    if (p.adj_residual) {
        // after the sweeps: r - (H lam)_i = b - H_ii lam_i of a constrained vertex,
        // the part of xbar that follows x_t across its constrained directions
        if (sub >= 0) {
            const float4 l = d.lam[vi];
            d.rhs[vi] = make_float4(b0 - (h00 * l.x + h01 * l.y + h02 * l.z), b1 - (h01 * l.x + h11 * l.y + h12 * l.z),
                                    b2 - (h02 * l.x + h12 * l.y + h22 * l.z), 0.f);
        }
        return;
    }
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
        const float inv = 1.f / det;
        l0 = (a00 * b0 + a01 * b1 + a02 * b2) * inv;
        l1 = (a01 * b0 + a11 * b1 + a12 * b2) * inv;
        l2 = (a02 * b0 + a12 * b1 + a22 * b2) * inv;
    }
    if (!(isfinite(l0) && isfinite(l1) && isfinite(l2))) {
        atomicAdd(d.counters + 0, 1ull);
        return;
    }
    d.lam[vi] = make_float4(l0, l1, l2, 0.f);
}

// xbar, vbar <- seed; lam <- 0; gtheta <- 0 is done by the host (memset).
__global__ void k_adj_seed(Dev d, const float *dL_dx, int n) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int i = d.new_of_orig[o];
    d.xbar[i] = make_float4(dL_dx[3 * o], dL_dx[3 * o + 1], dL_dx[3 * o + 2], 0.f);
    d.vbar[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// r = xbar + vbar / h on free vertices; lam = 0 everywhere (pinned stay 0).
__global__ void k_adj_rhs(Dev d, int n, int n_free, float inv_h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    d.lam[i] = make_float4(0.f, 0.f, 0.f, 0.f);
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
    const float4 l = d.lam[i], vb = d.vbar[i];
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
        const float3 l = f3(d.lam[id[k]]);
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

}  // namespace

void launch_adj_seed(const Dev &d, const float *dL_dx, int n, cudaStream_t s) {
    k_adj_seed<<<blocks_for(n, 256), 256, 0, s>>>(d, dL_dx, n);
}

void launch_adj_rhs(const Dev &d, int n, int n_free, float inv_h, cudaStream_t s) {
    k_adj_rhs<<<blocks_for(n, 256), 256, 0, s>>>(d, n, n_free, inv_h);
}

void launch_adj_sweep(const Dev &d, const float4 *xs, const SweepParams &p, int lanes, int block,
                      cudaStream_t s) {
    const long long threads = (long long)(p.vend - p.vbegin) * lanes;
    if (threads <= 0) return;
    const unsigned grid = blocks_for(threads, block);
    switch (lanes) {
    case 4: k_adj_sweep<4><<<grid, block, 0, s>>>(d, xs, p); break;
    case 8: k_adj_sweep<8><<<grid, block, 0, s>>>(d, xs, p); break;
    case 16: k_adj_sweep<16><<<grid, block, 0, s>>>(d, xs, p); break;
    default: k_adj_sweep<32><<<grid, block, 0, s>>>(d, xs, p); break;
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

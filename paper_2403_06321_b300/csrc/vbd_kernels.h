// vbd_kernels.h -- device data layout and kernel launchers of the VBD library
// (internal; the public boundary is include/vbd.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vbd {

// Device arrays, all carved out of the caller's workspace.  Vertices are in
// colour-major order: free vertices of colour 0, colour 1, ..., then pinned
// vertices.  Tets keep the caller's order.
// Positions are kept as displacements from the rest shape, u = x - X, so
// that FP32 resolves small strains at any distance from the origin; every
// quantity below that is a position (u, ut, ym, cheb, tape) is a displacement.
struct Dev {
    float4 *u;        // current displacement; .w = 1 once the vertex was in contact this step
    float4 *ut;       // u^t (start of step)
    float4 *v;        // v^t
    float4 *vprev;    // v^{t-1}
    float4 *ym;       // inertia target y - X (Eq. 3) in .xyz, m_i / h^2 in .w
    float4 *rest;     // rest position X (FP32), used to form x = X + u
    float4 *unew;     // block-Jacobi target (x^new of Algorithm 1)
    float4 *cheb[2];  // Chebyshev history (Eq. 18), roles alternate with iteration parity
    float *mass;      // lumped mass
    int *slot_off;    // n_free + 1: slots of free vertex i are [slot_off[i], slot_off[i+1])
    int *color_begin; // n_colors + 1: free vertices of colour c are [color_begin[c], color_begin[c+1])
    // incidence slots (one per (free vertex, incident tet)), 48 bytes each:
    int4 *s0;         // other three vertex ids, bits of g_a.x
    float4 *s1;       // g_a.yz, g_b.xy
    float4 *s2;       // g_b.z, g_c.xyz
    float2 *vmat;     // per free vertex: (mu, lambda) shared by all its tets
    int *slot_vtx;    // own vertex of each slot (two-phase scatter sweep only)
    float4 *scr0, *scr1;  // scatter sweep scratch per slot of one colour: f0 f1 f2 h00 | h01 h02 h11 h12
    float *scr2;      //                                               h22
    // warp rows (variant 7, carved with vbd_params.warp_rows): the slot records again, in rows of
    // 64 entries (two iterations of 32 lanes) per group of 8 consecutive vertices of a colour
    // (k_sweep_rows), padding id -1; a row is 192 float4: the entries' s0 words (ids as float
    // bits), then s1, then s2
    float4 *wrow;
    int *group_row;   // n_groups + 1: first row of each group (groups of all colours in colour order)
    int *slot_tet;    // caller tet id of each slot
    int *slot_loc;    // local index (0..3) of the slot's own vertex in that tet
    // subspace constraints (Sec. 3.4), when any vertex has one
    int *sub_id;      // n_free: index of the vertex's constraint, or -1
    float4 *sub_q;    // 2 per constraint: q_1 (.w = L) and q_2, an orthonormal basis of the subspace
    // per tet (caller order)
    int4 *tet_v;      // vertex ids (internal numbering)
    float *tet_B;     // 9 per tet: inverse rest edge matrix, row-major
    float *tet_V, *tet_nu, *tet_mu, *tet_lam;
    int *new_of_orig; // N
    float *stage[3];  // 3N each, state exchange with caller order
    unsigned long long *counters;  // [0] non-finite updates, [1] det skips, [2] pipeline wait time-outs,
                                   // [3] self-collision pairs found, [4] positions beyond the collision grid
    double *partials; // energy partial sums
    double *energy_out;
    double *gnorm;    // 2: max |dG/dx_i| (bits of a non-negative double, atomic max) and spare
    double *adj_res;  // 2 per tape step: max |r - H lam| and max |r| after the step's adjoint sweeps
    float4 *tape;     // tape_steps * N displacements
    // adjoint
    float4 *lam;      // 2N with a tape: per vertex a 32-byte record, [2i] the recorded displacement
                      // of the step being solved, [2i+1] lam_i (one 256-bit gather brings both)
    float4 *rhs, *xbar, *vbar;
    float4 *hdiag;    // 2N: each free vertex's diagonal block H_ii of the current adjoint step
                      // (h00 h01 h02 h11 | h12 h22 . .); carved with a tape
    float *gtheta;    // T
    // self-collision (vertex-triangle pairs, Sec. 3.5); carved only when enabled
    int4 *tri;        // boundary triangles: internal vertex ids, outward at rest (.w unused)
    int *surf;        // internal ids of the boundary vertices
    int *ring_off;    // n_surf + 1
    int *ring;        // sorted ids of every vertex sharing a tet with surf[k] (itself included)
    int *contact;     // N: triangle paired with the vertex by the last detection, -1 none
    int *rev_off;     // n_free + 1: pairs in which free vertex i is a triangle corner
    int *rev;         // 3 n_surf: the pairs' vertices, ascending per corner
    int *rev_fill;    // n_free
    float4 *tri_sphere;  // n_tris: centroid and radius of each triangle's bounding ball at this step
    float4 *tet_sphere;  // T: the same for the tets
    int *cell_start;  // n_buckets + 1: triangles of each hash bucket (by centroid cell)
    int *cell_fill;   // n_buckets
    int *cell_tri;    // n_tris
    float4 *cell_tri_sph; // n_tris: the sphere of each cell_tri entry, in table order
    int *tet_start;   // n_tet_buckets + 1: tets of each hash bucket (by centroid cell)
    int *tet_fill;    // n_tet_buckets
    int *cell_tet;    // T
    float4 *cell_tet_sph; // T: the sphere of each cell_tet entry, in table order
    int *scan_tmp;    // block totals of the prefix sums
    unsigned *cell_size;  // bits (float) of the largest centroid-to-corner distance: [0] triangles, [1] tets,
                          // [2] the largest half path of a boundary vertex (CCD)
    float4 *contact_w;    // N: a CCD pair's impact weights (.w = 1); .w = 0 for a DCD pair or none
    // edge-edge CCD pairs (Sec. 3.5), held by the edge that found them
    int4 *edge_v;         // n_edges boundary edges: p0, p1 (internal ids), their boundary (ring) indices
    float4 *edge_sphere;  // n_edges: bounding sphere of the edge's motion at the last CCD
    int *edge_start;      // n_edge_buckets + 1: edges of each hash bucket
    int *edge_fill;       // n_edge_buckets
    int *cell_edge;       // n_edges
    float4 *cell_edge_sph; // n_edges: edge_sphere of each cell_edge entry, in table order
    int *ee_partner;      // n_edges: the other edge of the held pair, or -1
    int *ee_found;        // n_edges: the edge hit first at the last CCD, or -1
    float4 *ee_prm;       // n_edges: s, u of the held pair, .z = 1 if carried from the previous step
    float4 *ee_hit;       // n_edges: s, u of ee_found
    float4 *ee_nrm;       // n_edges: the held pair's frozen normal
    int *ee_off;          // n_free + 1: edge-edge items of each free vertex
    int *ee_vfill;        // n_free
    int *ee_item;         // 4 n_edges: 4 * (holding edge) + role of the vertex (0, 1 edge a; 2, 3 edge b)
};

// static half-spaces of the unilateral constraints (Sec. 3.4): the ground and up to six walls
constexpr int kMaxPlanes = 7;

struct SweepParams {
    int vbegin, vend;
    int gbegin, gend; // warp-row groups of the colour (variant 7)
    float4 planes[kMaxPlanes];  // xyz unit normal, w offset: the allowed side is x.n >= w
    int n_planes;     // planes in use (ground first when on, then the walls)
    int n_sub;        // subspace-constrained vertices (Sec. 3.4); > 0 reads Dev::sub_id
    int adj_residual; // adjoint only: 1 store r - (H lam)_i of constrained vertices in Dev::rhs, 2 max-reduce
                      // |r - H lam| and |r| over all free vertices; lam unchanged in both
    int ee_on;        // edge-edge pairs exist (CCD on): the sweep reads Dev::ee_off
    int n_edges;      // boundary edges (energy of the edge-edge pairs)
    float kc;         // collision stiffness (Eq. 12)
    float det_eps;
    float kd_over_h;  // Rayleigh damping k_d / h
    float inv_h2;     // 1/h^2 (adjoint only)
    float mu_c;       // ground friction coefficient (Eqs. 13-16)
    float eps_h;      // eps_v * h: tangential displacement where f1 reaches 1
    int line_search;  // backtracking on G_i (Sec. 3.2)
    int per_tet_mat;  // 1: mu, lambda per tet (via slot_tet); 0: per vertex (vmat)
    int to_unew;      // every vertex writes to d.unew instead of updating d.u in place (block Jacobi)
    int self_collision;  // add the vertex-triangle contact forces of the current pairs
    int stall_test;   // TMA-staged sweep only: each CTA's first chunk also waits on a barrier that
                      // nothing arrives at, so its bounded wait runs out (tests of the time-out report)
};

// the fused iteration loop (one launch of one thread-block cluster per vbd_iterate)
struct FusedParams {
    SweepParams p;    // vbegin / vend unused: each colour range comes from Dev::color_begin
    int n_colors, first_n, iters, cheby, n_free;
    double rho;
};
constexpr int kFusedThreads = 512;
constexpr int kFusedMaxCluster = 8;   // portable cluster size
constexpr int kFusedMaxRounds = 2;    // passes of the CTAs over the largest colour

// sizes of the self-collision arrays
struct CollideDims {
    int n_tris, n_surf, n_buckets;
    int n_tets, n_tet_buckets;
    float radius;     // detection distance
    int n_edges, n_edge_buckets;  // boundary edges and their hash (edge-edge CCD)
    int ee_on;        // edge-edge pairs tracked (CCD on)
};

int num_sms();

void launch_predict(const Dev &d, int n, int n_free, float h, float3 g, int init_mode,
                    bool cheby, bool has_sub, cudaStream_t s);
void launch_sweep(const Dev &d, const SweepParams &p, int lanes, int block, cudaStream_t s);
// persistent grid-stride form of launch_sweep (grid = SMs x resident CTAs)
void launch_sweep_persist(const Dev &d, const SweepParams &p, int lanes, int block, cudaStream_t s);
// persistent sweep over compact slots (shape gradients from the rest positions)
void launch_sweep_rest(const Dev &d, const SweepParams &p, int lanes, int block, cudaStream_t s);
// variant 6: compact slots, two slots per lane in packed FP32
void launch_sweep_pair(const Dev &d, const SweepParams &p, int lanes, int block, cudaStream_t s);
// variant 7: warp rows streamed by per-warp bulk copies (4 lanes, 256 threads)
void launch_sweep_rows(const Dev &d, const SweepParams &p, cudaStream_t s);
// rows of a warp-row group that needs `iterations` iterations of 4 lanes, and the bytes of a row
int rows_per_group(int iterations);
size_t row_record_bytes();
// fills Dev::wrow for the groups [gbegin, gend) of one colour from the slot records
void launch_build_rows(const Dev &d, int vbegin, int vend, int gbegin, int gend, cudaStream_t s);
// two-phase tet-scatter-into-slots form; slots [sbegin, send) are the colour's
void launch_sweep_scatter(const Dev &d, const SweepParams &p, int sbegin, int send, int lanes, int block,
                          cudaStream_t s);
// pipelined sweep (TMA bulk copies of each chunk's slots into shared memory);
// maxs = slot capacity of one stage, chunks of block/8 vertices
size_t sweep_pipe_smem(int maxs);
int sweep_pipe_chunk(int block);
cudaError_t sweep_pipe_prepare(int block, int maxs, int *ctas_per_sm);
void launch_sweep_pipe(const Dev &d, const SweepParams &p, int block, int maxs, int grid_cap, cudaStream_t s);
void launch_cheby(const Dev &d, int n_free, int n, float omega, cudaStream_t s);
// CTAs of the cluster for the fused loop, or 0 when the largest colour does not fit
int fused_clusters_needed(int max_colour_verts, int lanes);
cudaError_t launch_iterate_fused(const Dev &d, const FusedParams &f, int lanes, int cluster, cudaStream_t s);
void launch_finish(const Dev &d, int n, float h, float4 *tape_row, cudaStream_t s);
// caller order <-> internal order; with `rest` non-null the caller array holds
// positions and the internal one displacements (u = x - X)
void launch_scatter(const float *src, float4 *dst, const int *new_of_orig, const float4 *rest, int n,
                    cudaStream_t s);
void launch_gather(const float4 *src, float *dst, const int *new_of_orig, const float4 *rest, int n,
                   cudaStream_t s);
void launch_restore_x(const Dev &d, int n, cudaStream_t s);
void launch_copy_back(const Dev &d, int vbegin, int vend, bool involved_only, bool ee_on, cudaStream_t s);
// n_surf > 0 adds the self-contact energy of the current pairs
// max_i |dG/dx_i| over the free vertices into *out (device double), asynchronous
cudaError_t launch_grad_norm(const Dev &d, const SweepParams &p, int n_free, double *out, cudaStream_t s);
void launch_energy(const Dev &d, int n_free, int n_tets, int n_surf, double h, const SweepParams &p,
                   cudaStream_t s);
int energy_partials_needed(int n_free, int n_tets, int n_surf);
// energy with its scratch in a static device array (see vbd_energy_static)
int energy_static_capacity();
int energy_static_partials_needed(int n_free, int n_tets, int n_surf);
cudaError_t launch_energy_static(const Dev &d, int n_free, int n_tets, int n_surf, double h,
                                 const SweepParams &p, double *G_out, cudaStream_t s);

// self-collision detection at x = X + u (vbd_collide.cu): fills d.contact,
// d.rev_off and d.rev; counters[3] += pairs found
int scan_tmp_needed(int n);
void launch_detect(const Dev &d, const CollideDims &c, int n_free, cudaStream_t s);
// vertex-triangle CCD along x^t (Dev::ut) -> the current iterate (Dev::u), Sec. 3.5
void launch_ccd(const Dev &d, const CollideDims &c, int n_free, cudaStream_t s);
void launch_set_log_young(const Dev &d, const float *log_young, int n_tets, cudaStream_t s);

// adjoint
void launch_adj_rhs(const Dev &d, const float4 *xs, int n, int n_free, float inv_h, cudaStream_t s);
// H_ii of the free vertices [p.vbegin, p.vend) at the recorded positions xs, into Dev::hdiag
void launch_adj_diag(const Dev &d, const float4 *xs, const SweepParams &p, int lanes, int block, cudaStream_t s);
void launch_adj_sweep(const Dev &d, const float4 *xs, const SweepParams &p, int lanes, int block,
                      cudaStream_t s, double *res_out = nullptr);
void launch_adj_post(const Dev &d, const float4 *xs, int n, int n_free, int n_tets, float h, bool has_sub,
                     cudaStream_t s);
void launch_adj_seed(const Dev &d, const float *dL_dx, int n, cudaStream_t s);
void launch_adj_out(const Dev &d, float *dL_dlogE, float *dL_dv0, int n, int n_tets,
                    cudaStream_t s);

}  // namespace vbd

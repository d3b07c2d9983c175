/*
 * vbd.h -- C ABI of the B300 (sm_103a) Vertex Block Descent library.
 *
 * Vertex Block Descent (Chen, Liu, Yang, Yuksel, ACM TOG 43(4), 2024)
 * integrates elastic tetrahedral bodies with implicit Euler written as the
 * minimisation of the variational energy G of Eqs. 1-2, by block coordinate
 * descent over vertices: Gauss-Seidel passes over vertex colours (Sec. 3.9),
 * each vertex taking one Newton step on its local energy G_i (Eqs. 4-5, 7-9).
 * One time step is Algorithm 1.
 *
 * Conventions for every entry point:
 *  - Returns a vbd_status; nothing throws across the ABI.  On failure the
 *    message of vbd_last_error() says why; the context stays usable unless
 *    the status is VBD_ERR_CUDA.
 *  - Host inputs to vbd_create_mesh / vbd_color are copied; the caller may
 *    free them on return.
 *  - The library allocates no device memory.  The caller allocates one
 *    workspace of vbd_workspace_size() bytes (256-byte aligned) and lends it
 *    with vbd_bind(); it must outlive the binding (until vbd_destroy or the
 *    next vbd_bind).
 *  - All device work is asynchronous on the stream given to vbd_bind()
 *    (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *    Calls marked "synchronising" wait for that stream.
 *  - Vertex and tet arrays are in the caller's order; the internal
 *    colour-major renumbering is never visible.
 *  - Float arrays of positions and velocities are 3*n_verts floats (x,y,z
 *    interleaved).  Pointers marked "host or device" may be either: with
 *    unified addressing the library tells them apart itself.
 *  - Units are SI; the default ground plane is z = 0 with +z up.
 */
#ifndef VBD_H
#define VBD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VBD_OK = 0,
    VBD_ERR_INVALID_ARG = 1,   /* NULL pointer, size or range error */
    VBD_ERR_BAD_MESH = 2,      /* tet index out of range, degenerate rest tet, bad material */
    VBD_ERR_BAD_COLORING = 3,  /* two vertices of one tet share a colour */
    VBD_ERR_NOT_COLORED = 4,   /* vbd_color() has not run */
    VBD_ERR_WORKSPACE = 5,     /* not bound, or workspace too small / misaligned */
    VBD_ERR_CUDA = 6,          /* a CUDA runtime call failed */
    VBD_ERR_NONFINITE = 7,     /* a kernel met a non-finite position or solve */
    VBD_ERR_NO_TAPE = 8,       /* vbd_backward without recorded steps */
    VBD_ERR_STATE = 9,         /* call out of order (e.g. vbd_iterate before vbd_begin_step) */
    VBD_ERR_TIMEOUT = 10,      /* a bounded wait inside a kernel gave up; results are invalid */
    VBD_ERR_RANGE = 11         /* self-collision met positions beyond its grid's exact range */
} vbd_status;

typedef struct vbd_ctx vbd_ctx;

/* One mesh, or the union of n_meshes independent meshes (batched mode):
 * mesh b owns vertices [vert_offset[b], vert_offset[b+1]) and tets
 * [tet_offset[b], tet_offset[b+1]); tets index the global vertex range.
 * Meshes share no tet, so the union is swept in one launch per colour; they
 * interact only through self-collision pairs, when that is on. */
typedef struct {
    int32_t n_meshes;             /* >= 1 */
    const int32_t *vert_offset;   /* host, n_meshes+1, or NULL when n_meshes == 1 */
    const int32_t *tet_offset;    /* host, n_meshes+1, or NULL when n_meshes == 1 */
    int32_t n_verts;              /* N >= 1 */
    int32_t n_tets;               /* T >= 1 */
    const double *rest_pos;       /* host, 3N: rest (material) positions */
    const int32_t *tets;          /* host, 4T: vertex ids in [0, N) */
    const float *young;           /* host, T: Young's modulus E > 0 [Pa] */
    const float *poisson;         /* host, T: Poisson ratio in (-1, 0.5) */
    const float *density;         /* host, T: mass density > 0 [kg/m^3] */
    const uint8_t *pinned;        /* host, N: 1 = fixed vertex, or NULL (Sec. 3.4: a bilateral
                                     constraint that fixes a vertex is met by never updating it) */
} vbd_mesh_desc;

typedef struct {
    float gravity[3];        /* a_ext of Eq. 3 [m/s^2] */
    int32_t ground_on;       /* ground half-space penalty (Eq. 12) on/off */
    float ground_height;     /* plane {x : x . n = ground_height} */
    float ground_normal[3];  /* n, need not be unit length */
    float k_c;               /* collision stiffness of Eq. 12 [N/m] */
    float cheby_rho;         /* spectral radius of Eq. 19; 0 disables acceleration */
    int32_t init_mode;       /* Sec. 3.7: 0 previous position, 1 inertia,
                                2 inertia + acceleration, 3 adaptive (default) */
    float det_eps;           /* Sec. 3.2 skip when |det H_i| <= det_eps |tr H_i / 3|^3 */
    float k_d;               /* Rayleigh damping coefficient of Eqs. 10-11 (0 = off) */
    int32_t tape_steps;      /* steps of positions recorded for vbd_backward (0 = none) */
    float mu_c;              /* ground friction coefficient of Eqs. 13-16 (0 = off) */
    float eps_v;             /* friction velocity threshold of Eq. 15 [m/s] */
    int32_t line_search;     /* 1: local backtracking on G_i after each Newton step (Sec. 3.2) */
    int32_t jacobi;          /* 1: block Jacobi, every vertex against the previous iterate */
    int32_t self_collision;  /* 1: vertex-triangle contact between boundary elements (Sec. 3.5) */
    float dcd_radius;        /* detection distance r of the self-collision pairs [m] */
    int32_t scatter_sweep;   /* 1: carve the buffers of the two-phase scatter sweep (variant 3 of
                                vbd_set_launch); enlarges the workspace, so set it before vbd_bind */
    int32_t xnew_copy_back;  /* 1: every colour pass writes x^new and copies it back, as Algorithm 1
                                prints it; without self-collision the default in-place writes give
                                the same positions bit for bit (no two vertices of one colour share
                                a tet), so this exists to check that */
    int32_t n_walls;         /* world-box walls in use, 0..VBD_MAX_WALLS */
    float walls[6][4];       /* wall k: normal walls[k][0..2] (need not be unit length) and offset
                                walls[k][3]; the allowed side is {x : x . n/|n| >= offset} */
    int32_t ccd_interval;    /* > 0 (with self_collision): vertex-triangle CCD before iterations
                                1, 1 + ccd_interval, ... of each step (Sec. 3.5); 0 = DCD only */
    int32_t ccd_edges;       /* 1: that CCD also pairs crossing boundary edges (Sec. 3.5, where
                                both kinds are used); a separate switch so that the vertex-
                                triangle CCD can run alone */
    int32_t warp_rows;       /* 1: carve and fill the warp-row copy of the slot records that sweep
                                variant 7 of vbd_set_launch streams (about the size of the slot
                                records again); set before vbd_bind */
} vbd_params;

#define VBD_MAX_WALLS 6

/* Library defaults: gravity (0,0,-9.8), ground off at z = 0 with n = +z,
 * k_c = 1e7, no acceleration, adaptive init, det_eps = 1e-12, no damping,
 * no friction (mu_c = 0, eps_v = 1e-3 m/s).  Friction acts on vertices in
 * ground contact: the ground is static, so the tangential part u of
 * x_i - x_i^t is the sliding displacement, the normal-force magnitude
 * k_c d scales it, and the force -mu_c k_c d f1(|u|) u/|u| (f1 of Eq. 15)
 * with Hessian mu_c k_c d f1(|u|)/|u| (I - n n^T) (Eq. 16) joins Eqs. 8-9.
 * World-box walls (none by default; Sec. 3.4 treats such unilateral
 * constraints as potentials) are static half-spaces like the ground: a
 * vertex at depth d = offset - x.n/|n| > 0 gets the same penalty (k_c) and
 * friction (mu_c, eps_v), and the terms of the ground and of every wall add
 * up.
 * line_search (off by default, as in the paper's results): after the Newton
 * step dx, alpha = 1, 1/2, ..., 1/128 is tried and the first alpha with
 * G_i(x + alpha dx) <= G_i(x) kept (no move if none), G_i being inertia,
 * elasticity and the ground and wall penalties (Eq. 4, Eq. 12).  G_i is exactly quadratic
 * in x_i apart from the penalty's kink, so the test is evaluated in closed
 * form without revisiting the tets.  jacobi (off by default): one pass per
 * iteration over all free vertices, each solved against the previous
 * iterate and written to an auxiliary buffer copied back after the pass
 * (the x^new of Algorithm 1 applied to all vertices at once); colours are
 * then not used.
 * self_collision (off by default; dcd_radius 0.01 m): at the start of every
 * step (on x^t) each boundary vertex a that has penetrated, i.e. lies in
 * (or on) a tet it is not a vertex of, is paired with the nearest boundary
 * triangle that shares no tet with it and lies within dcd_radius
 * (triangles within 1e-5 dcd_radius of the nearest distance count as tied;
 * the lowest index wins).  Boundary triangles are the tet
 * faces owned by one tet, oriented outward at rest.  The detection grid
 * works in FP32 with cells of about the element size: positions must stay
 * within 65536 cells of the origin (else vbd_sync_status reports
 * VBD_ERR_RANGE).  During the step a pair
 * with depth d = (q - x_a).n > 0 (q the nearest point of the triangle, w its
 * barycentric weights, n the unit normal at the current positions) adds the
 * penalty of Eq. 12 with the same k_c: k_c d n and k_c n n^T to vertex a,
 * -k_c d w_k n and k_c w_k^2 n n^T to corner k.  With mu_c > 0 the pairs
 * get friction as well (Eqs. 13-16): the contact points moved by
 * (x_a - x_a^t) - sum_k w_k (x_k - x_k^t) since the step start, u is its
 * tangential part, c = mu_c k_c d f1(|u|)/|u|, and vertex a gets -c u with
 * c (I - n n^T), corner k +w_k c u with w_k^2 c (I - n n^T).  Every colour pass then
 * solves its vertices against the pass-start positions and copies them back
 * (x^new of Algorithm 1), because a contact can couple two vertices of one
 * colour; the pipelined sweep is not used.
 * ccd_interval = n_col > 0 adds the CCD of Sec. 3.5: before iterations 1,
 * 1 + n_col, 1 + 2 n_col, ... each boundary vertex without a step-start
 * pair is swept along its straight path from x^t to the current iterate
 * against the boundary triangles that share no tet with it (their corners
 * moving the same way); the earliest time at which it lies in a closed
 * triangle (the coplanarity cubic's first admissible root; impacts within
 * 1e-5 in time are tied, the lowest index wins) gives a pair that acts
 * through the impact point, whose barycentric weights stay fixed, with the
 * triangle's current normal and the same penalty and friction.  Each CCD
 * replaces the previous CCD pairs; step-start pairs stay.  With ccd_edges
 * the same CCD sweeps the boundary edges (edges of boundary triangles) against each
 * other (partners share no tet): the first time two segments cross (the
 * coplanarity cubic's first root with both crossing parameters in [0, 1];
 * segments within about 6 degrees of parallel are not paired)
 * makes a pair held by the edge that found it (each edge keeps its first
 * hit, 1e-5 ties to the lowest index; a pair found from both edges is held
 * by the lower one).  Its contact points keep their parameters and its
 * normal n is the edges' unit common perpendicular where the CCD found them
 * crossed, oriented along x_b - x_a, frozen; d = (x_b - x_a).n > 0 adds the penalty of Eq. 12 (no
 * friction), -k_c d c_v n and k_c c_v^2 n n^T with c = (-(1 - s), -s,
 * 1 - u, u) for the four vertices.  A pair still penetrated at the next
 * step start is carried into that step.  Needs dcd_radius > 0; not
 * available with line_search; enlarges the workspace, so set it before
 * vbd_bind. */
void vbd_default_params(vbd_params *out);

/* Sizes of a created context (filled after vbd_color for the colour data). */
typedef struct {
    int32_t n_verts, n_tets, n_meshes;
    int32_t n_free;          /* vertices that are not pinned */
    int32_t n_colors;        /* 0 before vbd_color */
    int64_t n_slots;         /* (free vertex, incident tet) pairs streamed per iteration */
    int32_t lanes_per_vertex, block_threads;   /* current sweep launch shape */
    int32_t pipeline;        /* sweep variant of vbd_set_launch (0 plain, 1 TMA-staged, 2 persistent,
                                3 two-phase scatter, 4 fused loop, 5 compact slots, 6 compact slots
                                two per lane in packed FP32, 7 warp rows) */
    int32_t pipe_stage_slots; /* slot capacity of one pipeline stage */
    int32_t pipe_ctas_per_sm; /* resident CTAs per SM of the pipelined sweep */
    int32_t use_graph;       /* vbd_iterate replays a CUDA graph */
    int32_t n_surface_tris;  /* boundary triangles (0 until self-collision needed them) */
    int32_t n_surface_verts; /* vertices of those triangles */
} vbd_info;

/* Creates a context from host arrays (copied).  Computes per-tet rest data
 * in FP64 (inverse rest edge matrix and volume, lumped vertex masses
 * m_i = sum_j rho_j V_j / 4) and the stable neo-Hookean parameters
 * (Sec. 5 material; mu = E/(2(1+nu)), lambda = E nu/((1+nu)(1-2nu)) + mu,
 * alpha = 1 + mu/lambda).  VBD_ERR_BAD_MESH for an out-of-range index, a
 * rest tet with |det Dm| <= 1e-12 L^3, or a material outside its range.
 * *out receives the context (NULL on failure); free it with vbd_destroy. */
vbd_status vbd_create_mesh(const vbd_mesh_desc *desc, const vbd_params *params, vbd_ctx **out);

/* Vertex colouring of Sec. 3.9: no tet may hold two vertices of one colour.
 * colors = host array of N colour ids in [0, 4096) to validate and use, or
 * NULL for the library's greedy colouring (vertices by decreasing number of
 * distinct neighbours, ties by lower id, smallest free colour).  Renumbers
 * vertices colour-major and builds the incidence-slot arrays.  Invalidates
 * a previous binding (call vbd_bind again).  VBD_ERR_BAD_COLORING when the
 * given colouring is invalid.  *n_colors_out may be NULL. */
vbd_status vbd_color(vbd_ctx *ctx, const int32_t *colors, int32_t *n_colors_out);

/* Host copy of the colouring in use (N ints, caller order). */
vbd_status vbd_get_colors(const vbd_ctx *ctx, int32_t *colors_out);

vbd_status vbd_get_info(const vbd_ctx *ctx, vbd_info *out);

/* Boundary triangles used by self-collision (Sec. 3.5): *n_tris_out
 * receives their count and, when tris_out is not NULL, tris_out (host,
 * 3 * count ints) their caller vertex ids, each outward at rest, in
 * ascending order of the sorted id triple.  Builds the surface if needed.
 * VBD_ERR_NOT_COLORED before vbd_color. */
vbd_status vbd_get_surface(vbd_ctx *ctx, int32_t *n_tris_out, int32_t *tris_out);

/* Bytes of device workspace needed with the current colouring and params
 * (tape_steps enlarges it).  VBD_ERR_NOT_COLORED before vbd_color. */
vbd_status vbd_workspace_size(const vbd_ctx *ctx, size_t *bytes);

/* Lends the device workspace (256-byte aligned, >= vbd_workspace_size
 * bytes) and the stream; uploads the static mesh data and sets the state to
 * x = rest positions, v = v_prev = 0.  Asynchronous on `stream`. */
vbd_status vbd_bind(vbd_ctx *ctx, void *device_workspace, size_t bytes, void *stream);

/* Replaces the parameters.  Changing tape_steps requires a new vbd_bind. */
vbd_status vbd_set_params(vbd_ctx *ctx, const vbd_params *params);

/* Bilateral subspace constraints (Sec. 3.4): vertex[k] (caller id, not
 * pinned, each at most once) moves only within x^t + span(Q_k) during every
 * step, Q_k an orthonormal basis of a line (dim[k] = 1, dir[3k..3k+2] its
 * direction) or of a plane (dim[k] = 2, dir its normal); directions need
 * not be unit length.  The vertex's local step solves the reduced system
 * Q^T H Q dz = Q^T f (1x1 or 2x2, with the Sec. 3.2 singular test on it)
 * and moves by Q dz; its initial guess is projected onto x^t + span(Q).  A
 * vertex placed on a fixed line or plane therefore stays on it.  Host
 * arrays of n entries; n = 0 removes all constraints.  Must be called
 * before vbd_bind (the tables live in the workspace), else VBD_ERR_STATE;
 * VBD_ERR_INVALID_ARG for an index out of range, a pinned or repeated
 * vertex, a dimension other than 1 or 2, or a zero or non-finite
 * direction.  vbd_backward covers them: their block of H lam = r is the
 * reduced one, and their xbar keeps r - (H lam)_i, the part that follows
 * x^t across the constrained directions. */
vbd_status vbd_set_subspaces(vbd_ctx *ctx, int32_t n, const int32_t *vertex, const int32_t *dim,
                             const float *dir);

/* Sets x^t, v^t and v^{t-1} (3N floats each, caller order, host or device).
 * v_prev == NULL means v^{t-1} = v^t (zero estimated acceleration, the
 * first-step convention of Sec. 3.7 (d)).  v_prev goes beyond the plain
 * (x, v) state: the adaptive initial guess of Eq. 17 reads the previous
 * velocity, so a saved (x, v, v_prev) resumes a run bit for bit.  Clears the
 * tape. */
vbd_status vbd_set_state(vbd_ctx *ctx, const float *x, const float *v, const float *v_prev);

/* Copies x and v (3N floats each, caller order, host or device; either may
 * be NULL) on the bound stream.  For host destinations the call waits for
 * the stream (synchronising). */
vbd_status vbd_get_state(vbd_ctx *ctx, float *x, float *v);

/* Replaces the per-tet Young's moduli by exp(log_young) (T floats, caller
 * tet order, host or device), Poisson ratios unchanged. */
vbd_status vbd_set_log_young(vbd_ctx *ctx, const float *log_young);

/* One time step of Algorithm 1 with step size h and `iters` iterations:
 * vbd_begin_step + vbd_iterate + vbd_end_step. */
vbd_status vbd_step(vbd_ctx *ctx, float h, int32_t iters);

/* Start of Algorithm 1: y = x^t + h v^t + h^2 a_ext (Eq. 3) and the
 * initial guess of Sec. 3.7 (pinned vertices keep x^t). */
vbd_status vbd_begin_step(vbd_ctx *ctx, float h);

/* Algorithm 1 iteration loop: for n = 1..iters, one Gauss-Seidel pass per
 * colour in ascending colour order, each vertex solving H_i dx = f_i (Eqs.
 * 7-9, damping Eqs. 10-11, ground penalty Eq. 12, singular skip Sec. 3.2),
 * then, if cheby_rho > 0, the Chebyshev update of Eqs. 18-19 skipping
 * vertices that touched the ground during this step (Sec. 3.8).  Replays a
 * CUDA graph of the whole loop when graphs are enabled (default). */
vbd_status vbd_iterate(vbd_ctx *ctx, int32_t iters);

/* One Gauss-Seidel pass over the vertices of one colour (in place; vertices
 * of one colour share no tet, so in-place writes equal the x^new copy-back
 * of Algorithm 1 on this path; with self-collision the pass writes x^new
 * and copies it back, see vbd_default_params). */
vbd_status vbd_sweep_color(vbd_ctx *ctx, int32_t color);

/* Chebyshev update (Eq. 18) after iteration n (1-based) of the current step. */
vbd_status vbd_accelerate(vbd_ctx *ctx, int32_t n);

/* End of Algorithm 1: v^{t+1} = (x^{t+1} - x^t)/h (Eq. 6); records x
 * on the tape when tape_steps > 0. */
vbd_status vbd_end_step(vbd_ctx *ctx);

/* FP64 variational energy G(x) of Eq. 2 for the current x and the inertia
 * target y of the current step (free vertices; ground and wall penalties
 * included when on; self-contact pairs included).  Synchronising. */
vbd_status vbd_energy(vbd_ctx *ctx, double *G_out);

/* FP64 energy G(x), as vbd_energy, for callers that cannot allocate device
 * memory.  The paper has no counterpart; it exists for hosts that own every
 * byte of device memory themselves (a fixed pool handed out at start-up, a
 * real-time loop where cudaMalloc's implicit synchronisation is not
 * allowed) and so cannot grant this diagnostic scratch of its own.  Its
 * scratch (per-block partial sums) is a 512 KiB array inside the library,
 * one per CUDA context that loads it, kept until the process exits; nothing
 * is allocated.  G_out: device pointer to one double, written asynchronously
 * on the bound stream (not synchronising).  The first call in a context
 * looks up that context's copy of the array (a context made after a device
 * reset gets a fresh lookup); make it before any stream capture.  Calls that
 * overlap on the GPU (several streams at once) race on the shared array.
 * VBD_ERR_INVALID_ARG when the partial sums needed, ceil(free vertices /
 * 256) + ceil(tets / 256), plus ceil(boundary triangles / 256) when
 * self-collision is on, exceed 65536 (about 16.7 million elements in all),
 * or when G_out is not device memory. */
vbd_status vbd_energy_static(vbd_ctx *ctx, double *G_out);

/* Self-collision pairs of the current step (found by vbd_begin_step on
 * x^t): contact_out (host, N ints, caller order) receives for each vertex
 * the index of its paired triangle in the vbd_get_surface list, or -1.
 * VBD_ERR_STATE when the binding has no self-collision arrays.
 * Synchronising. */
vbd_status vbd_get_contacts(vbd_ctx *ctx, int32_t *contact_out);

/* Boundary edges and their edge-edge pairs (Sec. 3.5; pairs exist only with
 * ccd_interval > 0).  n_edges_out receives the number of boundary edges
 * (edges of the boundary triangles); edges_out (host, 2 per edge, may be
 * NULL) their caller vertex ids (lower id first), in ascending order;
 * partner_out (host, one per edge, may be NULL) for each edge the edge with
 * which it holds a pair, or -1.  Each pair is held by one of its edges.
 * VBD_ERR_STATE without a boundary surface (self_collision off when
 * vbd_color ran) or, for partner_out, without the self-collision arrays in
 * the bound workspace.  Synchronising when partner_out is given. */
vbd_status vbd_get_edge_pairs(vbd_ctx *ctx, int32_t *n_edges_out, int32_t *edges_out, int32_t *partner_out);

/* Waits for the stream and reads the device counters: VBD_ERR_TIMEOUT if a
 * bounded wait inside the pipelined sweep gave up (the step's results are
 * then invalid), else VBD_ERR_NONFINITE if any solve produced a non-finite
 * update since the last call (that update was not applied), else
 * VBD_ERR_RANGE if the self-collision detection met positions beyond its
 * grid's range (its pairs may then be incomplete).  det_skips
 * receives the singular-Hessian skips, contacts the self-collision pairs
 * found by detection, both summed since the last call; either may be NULL.
 * Synchronising. */
vbd_status vbd_sync_status(vbd_ctx *ctx, int64_t *det_skips, int64_t *contacts);

/* Adjoint of the recorded steps (tape_steps > 0; no paper counterpart, the
 * paper has no derivatives): treats every recorded step as converged
 * (dG/dx = 0 of Eq. 2) and, backwards over the steps, solves H lam = r with
 * `adj_iters` colour-ordered block Gauss-Seidel sweeps, H the Hessian of G
 * at the recorded positions.  Inputs: dL_dxT (3N floats, caller order,
 * device): dL/dx of the final positions.  Outputs (device, overwritten):
 * dL_dlogE (T floats, caller tet order): dL/d log E per tet; dL_dv0 (3N):
 * dL/dv at the first recorded step; either may be NULL.  Needs k_d = 0 and
 * mu_c = 0 (damping and friction are not variational).  With graphs on
 * (vbd_set_graph, the default) the step loop is captured once per tape
 * length, adj_iters and recorded step sizes and replayed by later calls;
 * it touches only the workspace, so the three buffers may differ from call
 * to call.  Synchronises only to read the tape length. */
vbd_status vbd_backward(vbd_ctx *ctx, const float *dL_dxT, float *dL_dlogE, float *dL_dv0,
                        int32_t adj_iters);

/* Convergence of the last vbd_backward (no paper counterpart): the adjoint
 * treats every recorded step as converged and solves H lam = r by a fixed
 * number of block Gauss-Seidel sweeps, so it reports how far each solve got.
 * After the sweeps of each step one more pass over all free vertices takes
 * max_i |r_i - (H lam)_i| and max_i |r_i| (per vertex in FP32, reduced in
 * FP64; for a subspace-constrained vertex the part within its subspace).
 * rel_out (host, n >= the number of recorded steps, else
 * VBD_ERR_INVALID_ARG) receives, per recorded step t in forward order,
 * max |r - H lam| / max |r| (0 when r = 0).  VBD_ERR_NO_TAPE before any
 * vbd_backward.  Synchronising. */
vbd_status vbd_adjoint_residuals(vbd_ctx *ctx, double *rel_out, int32_t n);

/* Convergence of the current step's iterate (no paper counterpart; a report
 * on how far the fixed iteration count of Algorithm 1 left the minimiser of
 * G, Eqs. 1-2): *grad_inf_out = max over free vertices of |dG/dx_i|, the
 * force residual of Eq. 8 with the ground and wall penalties of Eq. 12 at
 * the current x and the inertia target y of the current (or last) step, in
 * newtons; self-contact, damping and friction terms are not included (the
 * last two are not part of G).  Per vertex in FP32 like the sweep, reduced
 * in FP64.  force_scale_out (may be NULL) receives max_i m_i |a_ext|, the
 * largest weight, as a scale.  VBD_ERR_STATE before the first step.
 * Synchronising. */
vbd_status vbd_gradient_norm(vbd_ctx *ctx, double *grad_inf_out, double *force_scale_out);

/* Sweep launch shape and kernel variant.  variant:
 *  0  plain: one thread group of lanes_per_vertex in {4, 8, 16, 32} per
 *     vertex, loading its slot records from global memory, block_threads in
 *     {64, 128, 256}, one CTA per block of vertices;
 *  1  TMA-staged: persistent CTAs of block_threads in {128, 256} stage each
 *     chunk of block_threads/8 vertices' slot records in shared memory with
 *     TMA bulk copies, two chunks ahead, 8 lanes per vertex
 *     (lanes_per_vertex is ignored);
 *  2  persistent: variant 0's kernel on a grid of (SMs x resident CTAs)
 *     that strides over the colour's vertices (default, with 4 lanes and
 *     256 threads: the fastest measured on B300);
 *  3  two-phase tet-scatter-into-slots: one thread per incidence writes that
 *     tet's force and Hessian block on its vertex to a scratch slot, then a
 *     per-vertex kernel adds them up and solves (needs scatter_sweep = 1 at
 *     bind time, else VBD_ERR_STATE);
 *  4  fused loop for small meshes: each vbd_iterate is one launch of one
 *     thread-block cluster (up to 8 CTAs of 512 threads) that runs every
 *     colour pass and the Chebyshev update, the CTAs meeting at the
 *     hardware cluster barrier between passes (block_threads is ignored;
 *     VBD_ERR_INVALID_ARG when the largest colour exceeds two rounds of the
 *     cluster, 2048 vertices with 4 lanes);
 *  5  compact slots: variant 2's persistent grid reading only the 16-byte
 *     neighbour-id word of each slot and recomputing the shape gradients
 *     and volume from the FP32 rest positions (three more gathered
 *     positions per slot, a third of the streamed bytes; on B300 as fast as
 *     2 on a 1M-vertex cube and 7 % faster on a 33M-vertex one, where it
 *     stays below the power cap that throttles 2);
 *  6  compact slots, two per lane: variant 5's data and persistent grid,
 *     each lane evaluating two of its slots at once in packed FP32
 *     (sm_100+ pair instructions: half the FP32 instructions, both slots'
 *     gathers in flight together);
 *  7  warp rows: variant 2's arithmetic with 4 lanes (lanes_per_vertex and
 *     block_threads are ignored: 4 and 256) on a persistent grid whose warps
 *     each stream their next 64 slot records, copied at bind into one
 *     3,072-byte row per two iterations, into a ring of two shared-memory
 *     stages by bulk copies (TMA), every wait bounded (VBD_ERR_TIMEOUT as
 *     for variant 1); needs warp_rows = 1 at bind time, else VBD_ERR_STATE;
 *     with per-tet materials (vbd_set_log_young, mixed materials) its passes
 *     run variant 2.  On B300 slower than 2 (the ring's bookkeeping).
 * All variants give the same positions: 0, 2 and 4 bit for bit with equal
 * lanes (7 too, with 4), 1 equals 0 with 8 lanes, and 3 agrees to FP32 rounding (each
 * incidence's terms are rounded before they are summed); 5 differs from 0
 * by the rounding of the rest positions to FP32 (about 2e-7 of the
 * bounding-box diagonal after one iteration of a 1M-vertex cube), and 6
 * from 5 by its explicit fused multiply-adds and the order of its sums
 * (each lane adds its even and odd slots separately).  Self-collision passes always use the
 * plain form with contacts, and block Jacobi the plain form.  0 keeps a
 * shape value, a negative variant keeps the variant.  Must not be called
 * during stream capture. */
vbd_status vbd_set_launch(vbd_ctx *ctx, int32_t lanes_per_vertex, int32_t block_threads, int32_t variant);

/* Test hook for the time-out report of the TMA-staged sweep (variant 1):
 * while enabled, each CTA's first chunk, once its bulk copies have landed,
 * also waits on a spare barrier at which nothing arrives, so that wait runs
 * out after about 2 s of SM clock; the CTA records the time-out, waits
 * (bounded) for every copy it has issued and leaves, and the next
 * vbd_sync_status returns VBD_ERR_TIMEOUT.  Nothing faults, no copy is left
 * in flight, and the context stays usable.  Other variants ignore it. */
vbd_status vbd_debug_stall_pipeline(vbd_ctx *ctx, int32_t enable);

/* Enables (1) or disables (0) CUDA-graph replay of vbd_iterate's loop and of
 * vbd_backward's step loop (on by default; replay equals the eager launches
 * bit for bit). */
vbd_status vbd_set_graph(vbd_ctx *ctx, int32_t enable);

/* Times every applicable sweep launch shape of vbd_set_launch on the bound
 * stream, each for `iters` iterations of a step of size h begun from the
 * current state (one warm-up run, then the best of two to seven timed runs,
 * as many as fit in about 2 ms of timing; with the context's CUDA-graph
 * setting, so small meshes are timed as they will run), and keeps the
 * fastest (Sec. 3.9's colour passes are what
 * is timed; the paper fixes one launch shape, this picks it per mesh).
 * Between steps only (VBD_ERR_STATE inside one).  Everything the timing
 * steps overwrite is put back: x (from x^t; v and v^{t-1} are never
 * touched), the inertia target of the last step (so vbd_energy reads the
 * same G), the device counters of vbd_sync_status, and the host-side step
 * state.  The shapes differ in rounding (see vbd_set_launch), so the
 * chosen shape can change the last bits of later results; all of them
 * meet the same accuracy.  A failing call stops the search, keeps the
 * previous shape and returns its status.  With self-collision on, the
 * pass kernel is fixed: returns VBD_OK at once with *best_ms_per_iter = 0.
 * Synchronising.  best_ms_per_iter (may be NULL) receives the best time
 * per iteration in ms. */
vbd_status vbd_autotune(vbd_ctx *ctx, float h, int32_t iters, float *best_ms_per_iter);

/* vbd_autotune with flags: VBD_TUNE_SAME_ARITHMETIC restricts the search to
 * shapes whose positions equal those of the current shape bit for bit
 * (variants 0, 2 and 4 with the current lane count, variant 7 when that
 * count is 4, and variant 1 when it is 8; variants 3, 5 and 6 only among their
 * own block sizes), so tuning
 * cannot change any result.  Other bits: VBD_ERR_INVALID_ARG. */
#define VBD_TUNE_SAME_ARITHMETIC 1
vbd_status vbd_autotune_ex(vbd_ctx *ctx, float h, int32_t iters, int32_t flags, float *best_ms_per_iter);

/* Message of the last failed call on this context (static storage owned by
 * the context; valid until the next call).  Never NULL. */
const char *vbd_last_error(const vbd_ctx *ctx);

/* Releases host memory and CUDA graphs.  The workspace is the caller's. */
void vbd_destroy(vbd_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif

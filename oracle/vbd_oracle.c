/*
 * vbd_oracle.c -- serial FP64 CPU oracle for Vertex Block Descent.
 *
 * TEST INFRASTRUCTURE ONLY (see vbd_oracle.h).  Plain loops, FP64, no
 * blocking, fusion or reordering beyond what the paper states, so each
 * routine can be read against the paper equation it cites.  The same file
 * built with -fopenmp (liboracle_omp.so, used only to time the multi-core
 * CPU baseline) solves the vertices of one colour on several threads, which
 * Sec. 3.9 allows because they share no force element; its results equal
 * the serial build's bit for bit.
 *
 * Readings of points the paper leaves open (each pinned by a test):
 *  - Material: Sec. 5 uses the stable neo-Hookean model of Smith et al.
 *    (2018) with its logarithmic term dropped, and prints no formula:
 *        Psi(F) = mu/2 (tr F^T F - 3) + lam/2 (J - alpha)^2,
 *        alpha  = 1 + mu/lam   (the unique value making F = I stress free).
 *  - Lame mapping from (E, nu): mu = E/(2(1+nu)),
 *        lam = E nu/((1+nu)(1-2nu)) + mu, so the small-strain limit of Psi
 *        is linear elasticity with the textbook Lame pair.
 *  - Mass: lumped, m_i = sum over tets j containing i of rho_j V_j / 4.
 *  - Singular-Hessian skip (Sec. 3.2): |det H| <= det_eps * |tr H / 3|^3.
 *  - Contact (Eq. 12) with a ground half-space: x_b is the projection of
 *    the vertex on the plane, d = max(0, height - x.n), n held constant.
 *  - Subspace constraints (Sec. 3.4, bilateral): a constrained vertex moves
 *    in x^t + span(Q) with Q an orthonormal 3 x L basis (L = 1 line, 2
 *    plane); its local step solves Q^T H Q dz = Q^T f (dx = Q dz) with the
 *    singular test of Sec. 3.2 on the L x L matrix, and its initial guess is
 *    projected onto x^t + span(Q).  The subspace moves with x^t, so a vertex
 *    placed on a fixed line or plane stays on it.
 *  - World-box walls (Sec. 3.4 treats unilateral constraints as potentials):
 *    each wall is one more static half-space with the ground's penalty,
 *    stiffness k_c and friction (mu_c, eps_v); their terms add up.
 *  - Colouring (Sec. 3.9 gives no algorithm): greedy, vertices visited by
 *    decreasing number of distinct neighbours, ties by lower id, each
 *    taking the smallest colour unused by its neighbours.
 *  - Chebyshev (Eqs. 18-19): x^(0) is the initial guess; a vertex that
 *    saw contact in any iteration of the step, including the current one,
 *    keeps its Gauss-Seidel result (Sec. 3.8 collision skip).
 *  - First step: the caller passes v^{t-1} = v^t, so the adaptive
 *    acceleration estimate is 0.
 *  - Line search (Sec. 3.2, optional): on the variational part of G_i
 *    (inertia, elasticity, ground penalty; Eq. 4), try alpha = 1, 1/2, ...,
 *    1/128 along the Newton step and keep the first with G_i not above its
 *    current value; if none, the vertex does not move.
 *  - Block Jacobi: every vertex of an iteration solves against the previous
 *    iterate, and all moves are applied after the pass (x^new + copy-back
 *    of Algorithm 1 over all vertices at once); colours are not used.
 *  - Self-collision (Sec. 3.5, vertex-triangle only, DCD only): at the start
 *    of the step a boundary vertex that has already penetrated, i.e. lies
 *    inside (or on) a tet it does not belong to, is paired with the nearest
 *    boundary triangle within dcd_radius, skipping triangles that touch the
 *    vertex or one of its tet neighbours.  At every evaluation the closest point x_b
 *    on that triangle, its barycentric weights w and the unit normal n are
 *    recomputed from the current positions; with d = (x_b - x_a).n > 0 the
 *    penalty k_c d^2 / 2 of Eq. 12 (n held constant) gives the vertex
 *    +k_c d n and the triangle corners -k_c d w_k n, Hessians k_c n n^T and
 *    k_c w_k^2 n n^T.  These elements may join two vertices of one colour,
 *    so colour passes then use x^new and a copy-back (Algorithm 1): every
 *    vertex of the pass solves against the positions at its start.
 *  - Vertex-triangle CCD (Sec. 3.5): before every ccd_interval-th iteration
 *    (iterations 1, 1 + n_col, ...) each boundary vertex without a
 *    step-start pair is swept against the boundary triangles that share no
 *    tet with it, along the straight paths from x^t to the current iterate.
 *    Its impact is the earliest root t in [0, 1] of the coplanarity cubic
 *    at which it lies in the closed triangle (impacts within 1e-5 in t are
 *    tied; the lowest triangle index wins).  The pair keeps the impact
 *    point's barycentric weights w (the contact point is sum w_k x_k) and
 *    uses the triangle's current normal, with the penalty and friction of
 *    the DCD pairs; each CCD replaces the previous CCD pairs.
 *  - Edge-edge CCD (Sec. 3.5), in the same calls when ccd_edges is set:
 *    boundary edges (edges of
 *    boundary triangles) are swept against each other (candidates: none of
 *    the other edge's vertices shares a tet with one of its own); the
 *    impact is the first root of the coplanarity cubic at which the two
 *    segments cross (segments within about 6 degrees of parallel are not
 *    paired: their crossing point is ill-conditioned).  Each edge keeps the edge it hits first (1e-5 ties, the
 *    lowest index); each hit is one pair, counted once.  The contact points
 *    x_a, x_b keep their impact parameters, and the normal n is the unit
 *    common perpendicular e x g of the two edges at the detection positions
 *    (the current iterate, where the edges have crossed), oriented along
 *    x_b - x_a there, and frozen for the pair's life.  The paper takes n
 *    along x_b - x_a; for two lines that vector lies along e x g, which
 *    stays well conditioned when the crossing is shallow, and freezing n
 *    makes d = (x_b - x_a).n change sign when the edges are back across.  d = max(0, (x_b - x_a).n) with
 *    the penalty of Eq. 12; no friction on these pairs.  Neither CCD (from
 *    x^t) nor the vertex DCD can see two edges that are already crossed, so
 *    a pair still penetrated (d > 0) at the next step start is carried into
 *    that step, as the DCD's vertex pairs are; a carried pair ends at the
 *    first step start where d <= 0.
 *  - Ground friction (Eqs. 13-16): the ground is static, so the relative
 *    displacement is delta = x_i - x_i^t; u = its tangential part.  lambda
 *    is read as the normal-force magnitude k_c d >= 0 (as printed, the
 *    collision-gradient sign would push the vertex along its motion), so
 *    the force -mu lambda f1(|u|) u/|u| opposes the sliding and the
 *    Hessian term mu lambda f1(|u|)/|u| (I - n n^T) is positive
 *    semidefinite; |u| is not differentiated (Eq. 16).
 */
#include "vbd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_model {
    int n_verts, n_tets;
    int *tets;           /* 4T */
    double *B;           /* 9T: inverse rest edge matrix, row-major */
    double *V;           /* T : rest volume */
    double *mu, *lam;    /* T : stable neo-Hookean parameters */
    double *poisson;     /* T */
    double *mass;        /* N */
    unsigned char *pinned;
    int *inc_off;        /* N+1: vertex -> incident tets */
    int *inc_tet;        /* 4T */
    int *inc_loc;        /* 4T: local index (0..3) of the vertex in that tet */
    int n_tris;          /* boundary triangles, oriented outward at rest */
    int *tris;           /* 3 * n_tris */
    unsigned char *on_surface; /* N */
    int *contact;        /* N: triangle hit by the vertex (DCD at x^t), or -1 */
    double *contact_w;   /* 3N: impact weights of a CCD pair (fixed for the pair's life) */
    unsigned char *contact_ccd; /* N: 1 = the vertex's pair came from CCD, 0 = from the DCD */
    int n_edges;         /* boundary edges (edges of boundary triangles), ascending (lo, hi) */
    int *edges;          /* 2 * n_edges */
    /* edge-edge pairs, held by the edge that found them (Sec. 3.5 CCD) */
    int *ee_partner;     /* n_edges: the other edge of the pair this edge holds, or -1 */
    unsigned char *ee_carried; /* n_edges: 1 = the pair was still penetrated at the step start */
    double *ee_su;       /* 2 per edge: impact parameters s on this edge, u on the partner */
    double *ee_n;        /* 3 per edge: contact normal, frozen at detection */
    int *sub_dim;        /* N: L of the vertex's subspace constraint (Sec. 3.4), 3 = none */
    double *sub_basis;   /* 9N: orthonormal basis q_1..q_L of that subspace, 3 doubles each */
};

/* ------------------------------------------------------------------ */
/* small 3x3 helpers (row-major)                                        */
/* ------------------------------------------------------------------ */
static double det3(const double A[9]) {
    return A[0] * (A[4] * A[8] - A[5] * A[7])
         - A[1] * (A[3] * A[8] - A[5] * A[6])
         + A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* adjugate (transpose of the cofactor matrix): A * adj(A) = det(A) I */
static void adj3(const double A[9], double R[9]) {
    R[0] = A[4] * A[8] - A[5] * A[7];
    R[1] = A[2] * A[7] - A[1] * A[8];
    R[2] = A[1] * A[5] - A[2] * A[4];
    R[3] = A[5] * A[6] - A[3] * A[8];
    R[4] = A[0] * A[8] - A[2] * A[6];
    R[5] = A[2] * A[3] - A[0] * A[5];
    R[6] = A[3] * A[7] - A[4] * A[6];
    R[7] = A[1] * A[6] - A[0] * A[7];
    R[8] = A[0] * A[4] - A[1] * A[3];
}

static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* ------------------------------------------------------------------ */
/* materials and the tetrahedral element                                */
/* ------------------------------------------------------------------ */
void orc_lame(double E, double nu, double *mu, double *lam) {
    *mu = E / (2.0 * (1.0 + nu));
    *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)) + *mu;
}

/* Rest edge matrix Dm = [X1-X0, X2-X0, X3-X0] (columns), B = Dm^{-1},
 * V = |det Dm| / 6.  Returns 1 for a degenerate rest tet. */
int orc_rest_tet(const double X[12], double B[9], double *V) {
    double Dm[9], A[9], L = 0.0;
    for (int a = 0; a < 3; ++a) {
        double len2 = 0.0;
        for (int r = 0; r < 3; ++r) {
            Dm[r * 3 + a] = X[(a + 1) * 3 + r] - X[r];
            len2 += Dm[r * 3 + a] * Dm[r * 3 + a];
        }
        if (len2 > L) L = len2;
    }
    L = sqrt(L);
    double d = det3(Dm);
    if (!(fabs(d) > 1e-12 * L * L * L)) return 1;
    adj3(Dm, A);
    for (int k = 0; k < 9; ++k) B[k] = A[k] / d;
    *V = fabs(d) / 6.0;
    return 0;
}

/* Deformation gradient F = Ds B with Ds = [x1-x0, x2-x0, x3-x0]. */
void orc_tet_F(const double x[12], const double B[9], double F[9]) {
    double Ds[9];
    for (int a = 0; a < 3; ++a)
        for (int r = 0; r < 3; ++r) Ds[r * 3 + a] = x[(a + 1) * 3 + r] - x[r];
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) {
            double acc = 0.0;
            for (int a = 0; a < 3; ++a) acc += Ds[r * 3 + a] * B[a * 3 + s];
            F[r * 3 + s] = acc;
        }
}

/* cof F = dJ/dF: columns f1 x f2, f2 x f0, f0 x f1 (f_s = column s of F). */
void orc_cofactor(const double F[9], double C[9]) {
    double f[3][3], c[3];
    for (int s = 0; s < 3; ++s)
        for (int r = 0; r < 3; ++r) f[s][r] = F[r * 3 + s];
    for (int s = 0; s < 3; ++s) {
        cross3(f[(s + 1) % 3], f[(s + 2) % 3], c);
        for (int r = 0; r < 3; ++r) C[r * 3 + s] = c[r];
    }
}

double orc_nh_psi(const double F[9], double mu, double lam) {
    double Ic = 0.0;
    for (int k = 0; k < 9; ++k) Ic += F[k] * F[k];
    double alpha = 1.0 + mu / lam;
    double J = det3(F);
    return 0.5 * mu * (Ic - 3.0) + 0.5 * lam * (J - alpha) * (J - alpha);
}

/* First Piola-Kirchhoff stress P = dPsi/dF = mu F + lam (J - alpha) cof F. */
void orc_nh_pk1(const double F[9], double mu, double lam, double P[9]) {
    double C[9];
    orc_cofactor(F, C);
    double alpha = 1.0 + mu / lam;
    double J = det3(F);
    for (int k = 0; k < 9; ++k) P[k] = mu * F[k] + lam * (J - alpha) * C[k];
}

/* g_k = dF/dx_k (as F = sum_k x_k g_k^T): rows of B, g_0 = -(g_1+g_2+g_3). */
static void shape_grad(const double B[9], int k, double g[3]) {
    if (k == 0) {
        for (int s = 0; s < 3; ++s) g[s] = -(B[s] + B[3 + s] + B[6 + s]);
    } else {
        for (int s = 0; s < 3; ++s) g[s] = B[(k - 1) * 3 + s];
    }
}

double orc_tet_energy(const double x[12], const double B[9], double V, double mu, double lam) {
    double F[9];
    orc_tet_F(x, B, F);
    return V * orc_nh_psi(F, mu, lam);
}

/* dE/dx_k = V P g_k */
void orc_tet_grad(const double x[12], const double B[9], double V, double mu, double lam,
                  double grad[12]) {
    double F[9], P[9], g[3];
    orc_tet_F(x, B, F);
    orc_nh_pk1(F, mu, lam, P);
    for (int k = 0; k < 4; ++k) {
        shape_grad(B, k, g);
        for (int r = 0; r < 3; ++r)
            grad[k * 3 + r] = V * (P[r * 3 + 0] * g[0] + P[r * 3 + 1] * g[1] + P[r * 3 + 2] * g[2]);
    }
}

/* d^2E/(dx_k dx_l) = V [ mu (g_k.g_l) I + lam c_k c_l^T
 *                        + lam (J - alpha) [F (g_l x g_k)]_x ],  c = cof(F) g.
 * The skew term is the derivative of cof(F) g_k along x_l; it vanishes for
 * k == l because J is affine in any single vertex. */
void orc_tet_hess_block(const double x[12], const double B[9], double V, double mu, double lam,
                        int k, int l, double Hkl[9]) {
    double F[9], C[9], gk[3], gl[3], ck[3], cl[3], gx[3], a[3];
    orc_tet_F(x, B, F);
    orc_cofactor(F, C);
    double alpha = 1.0 + mu / lam;
    double J = det3(F);
    shape_grad(B, k, gk);
    shape_grad(B, l, gl);
    for (int r = 0; r < 3; ++r) {
        ck[r] = C[r * 3 + 0] * gk[0] + C[r * 3 + 1] * gk[1] + C[r * 3 + 2] * gk[2];
        cl[r] = C[r * 3 + 0] * gl[0] + C[r * 3 + 1] * gl[1] + C[r * 3 + 2] * gl[2];
    }
    cross3(gl, gk, gx);
    for (int r = 0; r < 3; ++r) a[r] = F[r * 3 + 0] * gx[0] + F[r * 3 + 1] * gx[1] + F[r * 3 + 2] * gx[2];
    double skew[9] = {0.0, -a[2], a[1], a[2], 0.0, -a[0], -a[1], a[0], 0.0};
    double gg = dot3(gk, gl);
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s)
            Hkl[r * 3 + s] = V * ((r == s ? mu * gg : 0.0) + lam * ck[r] * cl[s]
                                  + lam * (J - alpha) * skew[r * 3 + s]);
}

void orc_tet_hess(const double x[12], const double B[9], double V, double mu, double lam,
                  double H[144]) {
    double blk[9];
    for (int k = 0; k < 4; ++k)
        for (int l = 0; l < 4; ++l) {
            orc_tet_hess_block(x, B, V, mu, lam, k, l, blk);
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s) H[(k * 3 + r) * 12 + l * 3 + s] = blk[r * 3 + s];
        }
}

/* ------------------------------------------------------------------ */
/* vertex graph colouring (Sec. 3.9)                                    */
/* ------------------------------------------------------------------ */
static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

static int cmp_edge(const void *pa, const void *pb) {
    const int *a = (const int *)pa, *b = (const int *)pb;
    if (a[0] != b[0]) return (a[0] > b[0]) - (a[0] < b[0]);
    return (a[1] > b[1]) - (a[1] < b[1]);
}

static int cmp_face(const void *pa, const void *pb) {
    const int *x = (const int *)pa, *y = (const int *)pb;
    for (int k = 0; k < 3; ++k)
        if (x[k] != y[k]) return (x[k] > y[k]) - (x[k] < y[k]);
    return 0;
}

static int *g_deg_for_sort;
static int cmp_visit(const void *a, const void *b) {
    int i = *(const int *)a, j = *(const int *)b;
    if (g_deg_for_sort[i] != g_deg_for_sort[j]) return g_deg_for_sort[j] - g_deg_for_sort[i];
    return (i > j) - (i < j);
}

/* Returns the number of colours, or -1 on bad input. */
int orc_color_greedy(int n, int t, const int *tets, int *colors) {
    for (int k = 0; k < 4 * t; ++k)
        if (tets[k] < 0 || tets[k] >= n) return -1;
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
    for (int j = 0; j < t; ++j)
        for (int a = 0; a < 4; ++a) cnt[tets[4 * j + a] + 1] += 3;
    for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int *nbr = (int *)malloc(sizeof(int) * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
    int *fill = (int *)calloc((size_t)n, sizeof(int));
    for (int j = 0; j < t; ++j)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                if (a != b) {
                    int i = tets[4 * j + a];
                    nbr[cnt[i] + fill[i]++] = tets[4 * j + b];
                }
    /* sort and de-duplicate each list; degree = distinct neighbours */
    int *deg = (int *)calloc((size_t)n, sizeof(int));
    for (int i = 0; i < n; ++i) {
        int *L = nbr + cnt[i];
        int m = cnt[i + 1] - cnt[i];
        qsort(L, (size_t)m, sizeof(int), cmp_int);
        int u = 0;
        for (int k = 0; k < m; ++k)
            if (u == 0 || L[k] != L[u - 1]) L[u++] = L[k];
        deg[i] = u;
    }
    int *order = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) order[i] = i;
    g_deg_for_sort = deg;
    qsort(order, (size_t)n, sizeof(int), cmp_visit);
    for (int i = 0; i < n; ++i) colors[i] = -1;
    int n_colors = 0;
    unsigned char *used = (unsigned char *)calloc(4096, 1);
    for (int q = 0; q < n; ++q) {
        int i = order[q];
        for (int k = 0; k < deg[i]; ++k) {
            int c = colors[nbr[cnt[i] + k]];
            if (c >= 0 && c < 4096) used[c] = 1;
        }
        int c = 0;
        while (used[c]) ++c;
        colors[i] = c;
        if (c + 1 > n_colors) n_colors = c + 1;
        for (int k = 0; k < deg[i]; ++k) {
            int cc = colors[nbr[cnt[i] + k]];
            if (cc >= 0 && cc < 4096) used[cc] = 0;
        }
    }
    free(used); free(order); free(deg); free(fill); free(nbr); free(cnt);
    return n_colors;
}

/* 1 iff no force element (tet) uses two vertices of the same colour. */
int orc_color_valid(int n, int t, const int *tets, const int *colors) {
    for (int i = 0; i < n; ++i)
        if (colors[i] < 0) return 0;
    for (int j = 0; j < t; ++j)
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (colors[tets[4 * j + a]] == colors[tets[4 * j + b]]) return 0;
    return 1;
}

/* ------------------------------------------------------------------ */
/* model                                                                */
/* ------------------------------------------------------------------ */
static void gather_tet(const orc_model *m, int j, const double *x, double out[12]) {
    for (int a = 0; a < 4; ++a)
        for (int r = 0; r < 3; ++r) out[a * 3 + r] = x[3 * m->tets[4 * j + a] + r];
}

/* status: 0 ok, 1 bad index, 2 degenerate rest tet, 3 bad material */
orc_model *orc_model_new(int n, int t, const double *rest, const int *tets,
                         const double *young, const double *poisson, const double *density,
                         const unsigned char *pinned, int *status) {
    *status = 0;
    for (int k = 0; k < 4 * t; ++k)
        if (tets[k] < 0 || tets[k] >= n) { *status = 1; return NULL; }
    for (int j = 0; j < t; ++j)
        if (!(young[j] > 0.0) || !(poisson[j] > -1.0 && poisson[j] < 0.5) || !(density[j] > 0.0)) {
            *status = 3;
            return NULL;
        }
    orc_model *m = (orc_model *)calloc(1, sizeof(orc_model));
    m->n_verts = n;
    m->n_tets = t;
    m->tets = (int *)malloc(sizeof(int) * 4 * (size_t)t + 1);
    memcpy(m->tets, tets, sizeof(int) * 4 * (size_t)t);
    m->B = (double *)malloc(sizeof(double) * 9 * (size_t)t + 1);
    m->V = (double *)malloc(sizeof(double) * (size_t)t + 1);
    m->mu = (double *)malloc(sizeof(double) * (size_t)t + 1);
    m->lam = (double *)malloc(sizeof(double) * (size_t)t + 1);
    m->poisson = (double *)malloc(sizeof(double) * (size_t)t + 1);
    m->mass = (double *)calloc((size_t)n + 1, sizeof(double));
    m->pinned = (unsigned char *)malloc((size_t)n + 1);
    memcpy(m->pinned, pinned, (size_t)n);
    for (int j = 0; j < t; ++j) {
        double X[12];
        gather_tet(m, j, rest, X);
        if (orc_rest_tet(X, m->B + 9 * (size_t)j, m->V + j)) {
            *status = 2;
            orc_model_free(m);
            return NULL;
        }
        orc_lame(young[j], poisson[j], m->mu + j, m->lam + j);
        m->poisson[j] = poisson[j];
        for (int a = 0; a < 4; ++a) m->mass[tets[4 * j + a]] += density[j] * m->V[j] / 4.0;
    }
    m->inc_off = (int *)calloc((size_t)n + 1, sizeof(int));
    for (int k = 0; k < 4 * t; ++k) m->inc_off[tets[k] + 1]++;
    for (int i = 0; i < n; ++i) m->inc_off[i + 1] += m->inc_off[i];
    m->inc_tet = (int *)malloc(sizeof(int) * 4 * (size_t)t + 1);
    m->inc_loc = (int *)malloc(sizeof(int) * 4 * (size_t)t + 1);
    int *fill = (int *)calloc((size_t)n + 1, sizeof(int));
    for (int j = 0; j < t; ++j)
        for (int a = 0; a < 4; ++a) {
            int i = tets[4 * j + a];
            int s = m->inc_off[i] + fill[i]++;
            m->inc_tet[s] = j;
            m->inc_loc[s] = a;
        }
    free(fill);
    /* boundary triangles: tet faces that occur once, oriented away from the
     * tet's fourth vertex */
    {
        int nf = 4 * t;
        int *faces = (int *)malloc(sizeof(int) * 5 * (size_t)nf + 1);  /* sorted triple, tet, local face */
        for (int j = 0; j < t; ++j)
            for (int f = 0; f < 4; ++f) {
                int q = 0, v[3];
                for (int k = 0; k < 4; ++k)
                    if (k != f) v[q++] = tets[4 * j + k];
                /* sort the triple */
                for (int x0 = 0; x0 < 3; ++x0)
                    for (int x1 = x0 + 1; x1 < 3; ++x1)
                        if (v[x1] < v[x0]) { int tmp = v[x0]; v[x0] = v[x1]; v[x1] = tmp; }
                int *r = faces + 5 * (4 * (size_t)j + f);
                r[0] = v[0]; r[1] = v[1]; r[2] = v[2]; r[3] = j; r[4] = f;
            }
        qsort(faces, (size_t)nf, 5 * sizeof(int), cmp_face);
        m->tris = (int *)malloc(sizeof(int) * 3 * (size_t)nf + 1);
        m->on_surface = (unsigned char *)calloc((size_t)n + 1, 1);
        m->n_tris = 0;
        for (int k = 0; k < nf; ++k) {
            const int *r = faces + 5 * (size_t)k;
            int dup = (k > 0 && cmp_face(r, r - 5) == 0) || (k + 1 < nf && cmp_face(r, r + 5) == 0);
            if (dup) continue;
            int j = r[3], f = r[4];
            int v[3], q = 0;
            for (int kk = 0; kk < 4; ++kk)
                if (kk != f) v[q++] = tets[4 * j + kk];
            int opp = tets[4 * j + f];
            double e0[3], e1[3], nrm[3], to[3];
            for (int c = 0; c < 3; ++c) {
                e0[c] = rest[3 * v[1] + c] - rest[3 * v[0] + c];
                e1[c] = rest[3 * v[2] + c] - rest[3 * v[0] + c];
                to[c] = rest[3 * opp + c] - rest[3 * v[0] + c];
            }
            cross3(e0, e1, nrm);
            if (dot3(nrm, to) > 0.0) { int tmp = v[1]; v[1] = v[2]; v[2] = tmp; }
            int *o = m->tris + 3 * (size_t)m->n_tris++;
            o[0] = v[0]; o[1] = v[1]; o[2] = v[2];
            m->on_surface[v[0]] = m->on_surface[v[1]] = m->on_surface[v[2]] = 1;
        }
        free(faces);
        m->contact = (int *)malloc(sizeof(int) * (size_t)n + 1);
        for (int i = 0; i < n; ++i) m->contact[i] = -1;
        m->contact_w = (double *)calloc(3 * (size_t)n + 1, sizeof(double));
        m->contact_ccd = (unsigned char *)calloc((size_t)n + 1, 1);
        /* boundary edges: the sorted vertex pairs of the boundary triangles, once each */
        int *ed = (int *)malloc(sizeof(int) * 6 * (size_t)m->n_tris + 2);
        for (int T = 0; T < m->n_tris; ++T)
            for (int k = 0; k < 3; ++k) {
                int a = m->tris[3 * T + k], b = m->tris[3 * T + (k + 1) % 3];
                ed[6 * T + 2 * k] = a < b ? a : b;
                ed[6 * T + 2 * k + 1] = a < b ? b : a;
            }
        qsort(ed, 3 * (size_t)m->n_tris, 2 * sizeof(int), cmp_edge);
        m->edges = (int *)malloc(sizeof(int) * 6 * (size_t)m->n_tris + 2);
        m->n_edges = 0;
        for (int k = 0; k < 3 * m->n_tris; ++k)
            if (k == 0 || cmp_edge(ed + 2 * k, ed + 2 * (k - 1)) != 0) {
                m->edges[2 * m->n_edges] = ed[2 * k];
                m->edges[2 * m->n_edges + 1] = ed[2 * k + 1];
                m->n_edges++;
            }
        free(ed);
        m->ee_partner = (int *)malloc(sizeof(int) * (size_t)m->n_edges + 1);
        m->ee_carried = (unsigned char *)calloc((size_t)m->n_edges + 1, 1);
        for (int e = 0; e < m->n_edges; ++e) m->ee_partner[e] = -1;
        m->ee_su = (double *)malloc(sizeof(double) * 2 * (size_t)m->n_edges + 2);
        m->ee_n = (double *)malloc(sizeof(double) * 3 * (size_t)m->n_edges + 3);
    }
    m->sub_dim = (int *)malloc(sizeof(int) * (size_t)n + 1);
    m->sub_basis = (double *)calloc(9 * (size_t)n + 1, sizeof(double));
    for (int i = 0; i < n; ++i) m->sub_dim[i] = 3;
    return m;
}

/* Bilateral subspace constraint of Sec. 3.4 on vertex i: its position is
 * kept in x^t + span(q_1..q_L), L = 1 (a line with direction dir) or L = 2
 * (a plane with normal dir); L = 3 lifts the constraint.  The basis is
 * orthonormal: for L = 2, q_1 is the coordinate axis least aligned with the
 * normal with its normal part removed, q_2 = n x q_1.  Returns 0, or 1 for
 * a bad argument (index, L, zero direction). */
int orc_model_set_subspace(orc_model *m, int i, int L, const double dir[3]) {
    if (i < 0 || i >= m->n_verts || L < 1 || L > 3) return 1;
    double *q = m->sub_basis + 9 * (size_t)i;
    m->sub_dim[i] = 3;
    if (L == 3) return 0;
    double nn = sqrt(dot3(dir, dir));
    if (!(nn > 0.0) || !isfinite(nn)) return 1;
    double d[3] = {dir[0] / nn, dir[1] / nn, dir[2] / nn};
    if (L == 1) {
        for (int r = 0; r < 3; ++r) q[r] = d[r];
    } else {
        int a = 0;
        for (int r = 1; r < 3; ++r)
            if (fabs(d[r]) < fabs(d[a])) a = r;
        double e[3] = {0.0, 0.0, 0.0};
        e[a] = 1.0;
        double en = dot3(e, d);
        for (int r = 0; r < 3; ++r) e[r] -= en * d[r];
        double el = sqrt(dot3(e, e));
        for (int r = 0; r < 3; ++r) q[r] = e[r] / el;
        cross3(d, q, q + 3);
    }
    m->sub_dim[i] = L;
    return 0;
}

/* Restricts the Newton step of a subspace-constrained vertex (Sec. 3.4):
 * in the coordinates z of x_i = x_i^t + Q z the local force and Hessian are
 * b = Q^T f and A = Q^T H Q, the L x L system A dz = b is solved, and
 * dx = Q dz.  Returns 1 when A is singular by the Sec. 3.2 test on L x L
 * matrices, |det A| <= det_eps |tr A / L|^L (dx = 0). */
static int subspace_step(const orc_model *m, const orc_params *p, int i, const double f[3], const double H[9],
                         double dx[3]) {
    const int L = m->sub_dim[i];
    const double *q = m->sub_basis + 9 * (size_t)i;
    double b[2], A[4];
    for (int a = 0; a < L; ++a) {
        b[a] = dot3(q + 3 * a, f);
        for (int c = 0; c < L; ++c) {
            double Hq[3];
            for (int r = 0; r < 3; ++r)
                Hq[r] = H[r * 3 + 0] * q[3 * c] + H[r * 3 + 1] * q[3 * c + 1] + H[r * 3 + 2] * q[3 * c + 2];
            A[a * L + c] = dot3(q + 3 * a, Hq);
        }
    }
    double dz[2];
    dx[0] = dx[1] = dx[2] = 0.0;
    if (L == 1) {
        if (fabs(A[0]) <= p->det_eps * fabs(A[0])) return 1;
        dz[0] = b[0] / A[0];
    } else {
        double det = A[0] * A[3] - A[1] * A[2];
        double tr2 = 0.5 * (A[0] + A[3]);
        if (fabs(det) <= p->det_eps * tr2 * tr2) return 1;
        dz[0] = (A[3] * b[0] - A[1] * b[1]) / det;
        dz[1] = (A[0] * b[1] - A[2] * b[0]) / det;
    }
    for (int a = 0; a < L; ++a)
        for (int r = 0; r < 3; ++r) dx[r] += q[3 * a + r] * dz[a];
    return 0;
}

void orc_model_free(orc_model *m) {
    if (!m) return;
    free(m->tets); free(m->B); free(m->V); free(m->mu); free(m->lam); free(m->poisson);
    free(m->mass); free(m->pinned); free(m->inc_off); free(m->inc_tet); free(m->inc_loc);
    free(m->tris); free(m->on_surface); free(m->contact); free(m->contact_w); free(m->contact_ccd);
    free(m->edges); free(m->ee_partner); free(m->ee_carried); free(m->ee_su); free(m->ee_n);
    free(m->sub_dim); free(m->sub_basis);
    free(m);
}

int orc_model_n_tris(const orc_model *m) { return m->n_tris; }

void orc_model_tris(const orc_model *m, int *tris) {
    memcpy(tris, m->tris, sizeof(int) * 3 * (size_t)m->n_tris);
}

void orc_model_contacts(const orc_model *m, int *contact) {
    memcpy(contact, m->contact, sizeof(int) * (size_t)m->n_verts);
}

/* Closest point q of triangle (a, b, c) to p, with barycentric weights w
 * (q = w0 a + w1 b + w2 c): the projection onto the plane if it falls
 * inside, otherwise the nearest of the closest points on the three edges. */
void orc_closest_point_tri(const double p[3], const double a[3], const double b[3], const double c[3],
                           double q[3], double w[3]) {
    double e0[3], e1[3], r[3];
    for (int k = 0; k < 3; ++k) {
        e0[k] = b[k] - a[k];
        e1[k] = c[k] - a[k];
        r[k] = p[k] - a[k];
    }
    double d00 = dot3(e0, e0), d01 = dot3(e0, e1), d11 = dot3(e1, e1);
    double d20 = dot3(r, e0), d21 = dot3(r, e1);
    double den = d00 * d11 - d01 * d01;
    double wb = (d11 * d20 - d01 * d21) / den;
    double wc = (d00 * d21 - d01 * d20) / den;
    double wa = 1.0 - wb - wc;
    if (wa >= 0.0 && wb >= 0.0 && wc >= 0.0) {
        w[0] = wa; w[1] = wb; w[2] = wc;
    } else {
        const double *P[3] = {a, b, c};
        double best = -1.0;
        for (int e = 0; e < 3; ++e) {
            const double *p0 = P[e], *p1 = P[(e + 1) % 3];
            double dd[3], pp[3];
            for (int k = 0; k < 3; ++k) { dd[k] = p1[k] - p0[k]; pp[k] = p[k] - p0[k]; }
            double tt = dot3(pp, dd) / dot3(dd, dd);
            if (tt < 0.0) tt = 0.0;
            if (tt > 1.0) tt = 1.0;
            double dist2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                double z = p0[k] + tt * dd[k] - p[k];
                dist2 += z * z;
            }
            if (best < 0.0 || dist2 < best) {
                best = dist2;
                w[0] = w[1] = w[2] = 0.0;
                w[e] = 1.0 - tt;
                w[(e + 1) % 3] = tt;
            }
        }
    }
    for (int k = 0; k < 3; ++k) q[k] = w[0] * a[k] + w[1] * b[k] + w[2] * c[k];
}

/* unit normal of boundary triangle T at positions x */
static void tri_normal(const orc_model *m, int T, const double *x, double n[3]) {
    const int *v = m->tris + 3 * (size_t)T;
    double e0[3], e1[3];
    for (int k = 0; k < 3; ++k) {
        e0[k] = x[3 * v[1] + k] - x[3 * v[0] + k];
        e1[k] = x[3 * v[2] + k] - x[3 * v[0] + k];
    }
    cross3(e0, e1, n);
    double l = sqrt(dot3(n, n));
    for (int k = 0; k < 3; ++k) n[k] /= l;
}

/* penetration depth of vertex a into its contact triangle at positions x:
 * d = (x_b - x_a).n with x_b the closest point; also returns n and w */
static double contact_depth(const orc_model *m, int a, const double *x, double n[3], double w[3]) {
    const int T = m->contact[a];
    const int *v = m->tris + 3 * (size_t)T;
    double q[3];
    if (m->contact_ccd[a]) {
        /* CCD pair: the impact point keeps its barycentric weights (Sec. 3.5) */
        for (int k = 0; k < 3; ++k) w[k] = m->contact_w[3 * (size_t)a + k];
        for (int r = 0; r < 3; ++r)
            q[r] = w[0] * x[3 * v[0] + r] + w[1] * x[3 * v[1] + r] + w[2] * x[3 * v[2] + r];
    } else {
        orc_closest_point_tri(x + 3 * a, x + 3 * v[0], x + 3 * v[1], x + 3 * v[2], q, w);
    }
    tri_normal(m, T, x, n);
    return (q[0] - x[3 * a]) * n[0] + (q[1] - x[3 * a + 1]) * n[1] + (q[2] - x[3 * a + 2]) * n[2];
}

/* 1 if point q lies in the closed tet (x[t[0]], .., x[t[3]]): its barycentric
 * coordinates, from the edge matrix E = [x1 - x0, x2 - x0, x3 - x0] by
 * Cramer's rule, are all >= 0.  0 for a flat tet. */
int orc_point_in_tet(const double *x, const int *t, const double q[3]) {
    double E[9], r[3];
    for (int k = 0; k < 3; ++k) {
        for (int c = 0; c < 3; ++c) E[3 * k + c] = x[3 * t[c + 1] + k] - x[3 * t[0] + k];
        r[k] = q[k] - x[3 * t[0] + k];
    }
    double D = det3(E);
    if (D == 0.0) return 0;
    double lam_sum = 0.0;
    for (int c = 0; c < 3; ++c) {
        double Ec[9];
        memcpy(Ec, E, sizeof(Ec));
        for (int k = 0; k < 3; ++k) Ec[3 * k + c] = r[k];
        double l = det3(Ec) / D;
        if (l < 0.0) return 0;
        lam_sum += l;
    }
    return 1.0 - lam_sum >= 0.0;
}

/* DCD at positions x (the step start), one vertex: returns the triangle
 * paired with vertex a, or -1.  A boundary vertex has penetrated
 * when it lies in a tet it is not a vertex of; it is then paired with the
 * nearest boundary triangle within dcd_radius, skipping triangles that touch
 * the vertex or a vertex sharing a tet with it.  Triangles whose distance is
 * within 1e-5 dcd_radius of the nearest count as tied (a nearest point on an
 * edge or corner is shared by several triangles; rounding must not choose)
 * and the lowest index wins. */
int orc_dcd_vertex(const orc_model *m, const orc_params *p, const double *x, int a) {
    if (!m->on_surface[a]) return -1;
    int inside = 0;
    for (int j = 0; j < m->n_tets && !inside; ++j) {
        const int *t = m->tets + 4 * (size_t)j;
        if (t[0] == a || t[1] == a || t[2] == a || t[3] == a) continue;
        inside = orc_point_in_tet(x, t, x + 3 * a);
    }
    if (!inside) return -1;
    double best = -1.0;
    for (int pass = 0; pass < 2; ++pass) {
        /* pass 0: the nearest distance; pass 1: the lowest index near it */
        for (int T = 0; T < m->n_tris; ++T) {
            const int *v = m->tris + 3 * (size_t)T;
            int adjacent = 0;  /* a triangle vertex shares a tet with a */
            for (int s = m->inc_off[a]; s < m->inc_off[a + 1] && !adjacent; ++s)
                for (int k = 0; k < 4; ++k) {
                    int w = m->tets[4 * (size_t)m->inc_tet[s] + k];
                    adjacent |= (w == v[0]) | (w == v[1]) | (w == v[2]);
                }
            if (adjacent) continue;
            double q[3], w[3];
            orc_closest_point_tri(x + 3 * a, x + 3 * v[0], x + 3 * v[1], x + 3 * v[2], q, w);
            double dv[3] = {x[3 * a] - q[0], x[3 * a + 1] - q[1], x[3 * a + 2] - q[2]};
            double dist = sqrt(dot3(dv, dv));
            if (dist > p->dcd_radius) continue;
            if (pass == 0 && (best < 0.0 || dist < best)) best = dist;
            if (pass == 1 && dist <= best + 1e-5 * p->dcd_radius) return T;
        }
        if (best < 0.0) break;
    }
    return -1;
}

static double ee_depth(const orc_model *m, int e, const double *x, int v[4], double c[4]);

void orc_dcd(orc_model *m, const orc_params *p, const double *x) {
    /* edge-edge pairs (found by CCD) that are still penetrated at x^t are
     * carried into the step; the others end */
    for (int e = 0; e < m->n_edges; ++e) {
        m->ee_carried[e] = 0;
        if (m->ee_partner[e] < 0) continue;
        int v[4];
        double c[4];
        if (ee_depth(m, e, x, v, c) > 0.0) m->ee_carried[e] = 1;
        else m->ee_partner[e] = -1;
    }
    for (int a = 0; a < m->n_verts; ++a) {
        m->contact[a] = orc_dcd_vertex(m, p, x, a);
        m->contact_ccd[a] = 0;
    }
}

/* f(t) = c0 + c1 t + c2 t^2 + c3 t^3.  Its earliest root in [t_min, 1]: the
 * interval is cut at the roots of f' into monotone pieces, and the first
 * piece that starts at a zero or changes sign is bisected to full FP64
 * precision.  Returns -1 when f has no root there; a cubic that vanishes
 * identically (coplanar motion) counts as no root. */
double orc_cubic_first_root(const double c[4], double t_min) {
    double scale = fabs(c[0]) + fabs(c[1]) + fabs(c[2]) + fabs(c[3]);
    if (!(scale > 0.0)) return -1.0;
    double cut[4];
    int nc = 0;
    cut[nc++] = t_min;
    /* roots of f' = c1 + 2 c2 t + 3 c3 t^2 inside (t_min, 1), ascending */
    double qa = 3.0 * c[3], qb = 2.0 * c[2], qc = c[1], r[2];
    int nr = 0;
    if (qa != 0.0) {
        double disc = qb * qb - 4.0 * qa * qc;
        if (disc >= 0.0) {
            double sq = sqrt(disc);
            r[0] = (-qb - sq) / (2.0 * qa);
            r[1] = (-qb + sq) / (2.0 * qa);
            if (r[0] > r[1]) { double t = r[0]; r[0] = r[1]; r[1] = t; }
            nr = 2;
        }
    } else if (qb != 0.0) {
        r[0] = -qc / qb;
        nr = 1;
    }
    for (int k = 0; k < nr; ++k)
        if (r[k] > t_min && r[k] < 1.0) cut[nc++] = r[k];
    cut[nc++] = 1.0;
    for (int k = 0; k + 1 < nc; ++k) {
        double lo = cut[k], hi = cut[k + 1];
        double flo = ((c[3] * lo + c[2]) * lo + c[1]) * lo + c[0];
        double fhi = ((c[3] * hi + c[2]) * hi + c[1]) * hi + c[0];
        if (flo == 0.0) return lo;
        if ((flo < 0.0) == (fhi < 0.0) && fhi != 0.0) continue;
        for (int it = 0; it < 200 && hi - lo > 1e-15; ++it) {
            double mid = 0.5 * (lo + hi);
            double fm = ((c[3] * mid + c[2]) * mid + c[1]) * mid + c[0];
            if (fm == 0.0) { lo = hi = mid; break; }
            if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
        }
        return hi;
    }
    return -1.0;
}

/* Time of impact of vertex a with triangle v along the linear trajectories
 * (Sec. 3.5 CCD).  With r_k(t) = x_k(t) - x_a(t) = A_k + t B_k for the three
 * corners, the vertex is in the triangle's plane where
 * f(t) = r_1 . (r_2 x r_3) = 0, a cubic whose coefficients follow from the
 * trilinear expansion in (A_k, B_k).  Its roots are visited in order; the
 * first one at which the vertex lies inside the (closed) triangle, by
 * barycentric weights of the projected point, is the impact.  Returns the
 * time or -1; w receives the weights. */
static double vt_impact(const double *x0, const double *x1, int a, const int *v, double w[3]) {
    double A[3][3], B[3][3];
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) {
            A[k][r] = x0[3 * v[k] + r] - x0[3 * a + r];
            B[k][r] = (x1[3 * v[k] + r] - x1[3 * a + r]) - A[k][r];
        }
    double t23[3], c[4], tmp[3];
    cross3(A[1], A[2], t23);
    c[0] = dot3(A[0], t23);
    c[1] = dot3(B[0], t23);
    cross3(B[1], A[2], tmp); c[1] += dot3(A[0], tmp);
    cross3(A[1], B[2], tmp); c[1] += dot3(A[0], tmp);
    cross3(B[1], A[2], tmp); c[2] = dot3(B[0], tmp);
    cross3(A[1], B[2], tmp); c[2] += dot3(B[0], tmp);
    cross3(B[1], B[2], tmp); c[2] += dot3(A[0], tmp);
    c[3] = dot3(B[0], tmp);
    double t0 = 0.0;
    for (int rep = 0; rep < 3; ++rep) {
        double t = orc_cubic_first_root(c, t0);
        if (t < 0.0) return -1.0;
        /* barycentric weights of the vertex, projected onto the triangle at t */
        double r1[3], r2[3], r3[3], n[3], e1[3], e2[3], s1[3], s2[3], s3[3];
        for (int q = 0; q < 3; ++q) {
            r1[q] = A[0][q] + t * B[0][q];
            r2[q] = A[1][q] + t * B[1][q];
            r3[q] = A[2][q] + t * B[2][q];
            e1[q] = r2[q] - r1[q];
            e2[q] = r3[q] - r1[q];
        }
        cross3(e1, e2, n);
        double nn = dot3(n, n);
        if (nn > 0.0) {
            cross3(r2, r3, s1);  /* twice the area of (a, 2, 3) along n, and so on */
            cross3(r3, r1, s2);
            cross3(r1, r2, s3);
            w[0] = dot3(s1, n) / nn;
            w[1] = dot3(s2, n) / nn;
            w[2] = dot3(s3, n) / nn;
            if (w[0] >= 0.0 && w[1] >= 0.0 && w[2] >= 0.0) return t;
        }
        /* not inside at this root: look for the next one */
        t0 = t + 1e-12;
        if (t0 >= 1.0) return -1.0;
    }
    return -1.0;
}

int orc_ccd_vertex(const orc_model *m, const double *x0, const double *x1, int a, double *toi, double wout[3]) {
    if (!m->on_surface[a]) return -1;
    double best = 2.0;
    int best_T = -1;
    for (int T = 0; T < m->n_tris; ++T) {
        const int *v = m->tris + 3 * (size_t)T;
        int adjacent = 0;  /* a triangle vertex shares a tet with a */
        for (int s = m->inc_off[a]; s < m->inc_off[a + 1] && !adjacent; ++s)
            for (int k = 0; k < 4; ++k) {
                int q = m->tets[4 * (size_t)m->inc_tet[s] + k];
                adjacent |= (q == v[0]) | (q == v[1]) | (q == v[2]);
            }
        if (adjacent) continue;
        double w[3];
        double t = vt_impact(x0, x1, a, v, w);
        /* earliest impact; impacts within 1e-5 of it count as tied and the
         * lowest triangle index wins (triangles are visited in order) */
        if (t >= 0.0 && t < best - 1e-5) {
            best = t;
            best_T = T;
            for (int k = 0; k < 3; ++k) wout[k] = w[k];
        }
    }
    if (best_T >= 0 && toi) *toi = best;
    return best_T;
}

/* Time of impact of edges (p0, p1) and (q0, q1) moving linearly (Sec. 3.5
 * CCD): with A_k + t B_k the positions of p1, q0, q1 relative to p0, the
 * four points are coplanar where the cubic (p1 - p0) . ((q0 - p0) x
 * (q1 - p0)) vanishes; its roots are visited in order and the first at
 * which the segments cross (in their common plane, p0 + s (p1 - p0) =
 * q0 + u (q1 - q0) with s, u in [0, 1]) is the impact.  Segments within
 * about 6 degrees of parallel (|e x g| < 0.1 |e| |g|) count as no
 * crossing: their crossing point is ill-conditioned, and the vertex-triangle
 * pairs of their end points take them.  Returns t or -1; s, u receive the
 * parameters. */
double orc_ee_impact(const double *x0, const double *x1, int p0, int p1, int q0, int q1, double *s_out,
                     double *u_out) {
    const int id[3] = {p1, q0, q1};
    double A[3][3], B[3][3];
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) {
            A[k][r] = x0[3 * id[k] + r] - x0[3 * p0 + r];
            B[k][r] = (x1[3 * id[k] + r] - x1[3 * p0 + r]) - A[k][r];
        }
    double t23[3], c[4], tmp[3];
    cross3(A[1], A[2], t23);
    c[0] = dot3(A[0], t23);
    c[1] = dot3(B[0], t23);
    cross3(B[1], A[2], tmp); c[1] += dot3(A[0], tmp);
    cross3(A[1], B[2], tmp); c[1] += dot3(A[0], tmp);
    cross3(B[1], A[2], tmp); c[2] = dot3(B[0], tmp);
    cross3(A[1], B[2], tmp); c[2] += dot3(B[0], tmp);
    cross3(B[1], B[2], tmp); c[2] += dot3(A[0], tmp);
    c[3] = dot3(B[0], tmp);
    double t0 = 0.0;
    for (int rep = 0; rep < 3; ++rep) {
        double t = orc_cubic_first_root(c, t0);
        if (t < 0.0) return -1.0;
        double e[3], w[3], g[3], n[3], wg[3], we[3];
        for (int r = 0; r < 3; ++r) {
            e[r] = A[0][r] + t * B[0][r];               /* p1 - p0 */
            w[r] = A[1][r] + t * B[1][r];               /* q0 - p0 */
            g[r] = (A[2][r] + t * B[2][r]) - w[r];      /* q1 - q0 */
        }
        cross3(e, g, n);
        double nn = dot3(n, n);
        /* edges within about 6 degrees of parallel (|e x g| < 0.1 |e| |g|)
         * have an ill-conditioned crossing point: not paired */
        if (nn > 0.01 * dot3(e, e) * dot3(g, g)) {
            cross3(w, g, wg);
            cross3(w, e, we);
            double s = dot3(wg, n) / nn, u = dot3(we, n) / nn;
            if (s >= 0.0 && s <= 1.0 && u >= 0.0 && u <= 1.0) {
                *s_out = s;
                *u_out = u;
                return t;
            }
        }
        t0 = t + 1e-12;
        if (t0 >= 1.0) return -1.0;
    }
    return -1.0;
}

/* whether vertex q shares a tet with vertex a (or is a) */
static int shares_tet(const orc_model *m, int a, int q) {
    for (int s = m->inc_off[a]; s < m->inc_off[a + 1]; ++s)
        for (int k = 0; k < 4; ++k)
            if (m->tets[4 * (size_t)m->inc_tet[s] + k] == q) return 1;
    return a == q;
}

/* Edge-edge CCD: each boundary edge that holds no carried pair takes the
 * boundary edge it hits first (ties within 1e-5 in time: the lowest index),
 * among edges none of whose vertices shares a tet with one of its own.  The
 * pair is held by the finding edge, unless the partner found this edge too
 * with a lower index (it then holds it) or the partner already holds the
 * same pair as a carried one.  The contact points keep their impact
 * parameters; the normal is the edges' unit common perpendicular at x1,
 * oriented along x_b - x_a there and frozen for the pair's life (a pair
 * with x_b - x_a perpendicular to it there is dropped). */
int orc_ee_first_hit(const orc_model *m, const double *x0, const double *x1, int e, double *s_out,
                     double *u_out) {
    const int p0 = m->edges[2 * e], p1 = m->edges[2 * e + 1];
    double best = 2.0;
    int found = -1;
    for (int f = 0; f < m->n_edges; ++f) {
        const int q0 = m->edges[2 * f], q1 = m->edges[2 * f + 1];
        if (shares_tet(m, p0, q0) || shares_tet(m, p0, q1) || shares_tet(m, p1, q0) || shares_tet(m, p1, q1))
            continue;
        double s, u;
        double t = orc_ee_impact(x0, x1, p0, p1, q0, q1, &s, &u);
        if (t >= 0.0 && t < best - 1e-5) {
            best = t;
            found = f;
            *s_out = s;
            *u_out = u;
        }
    }
    return found;
}

static void ee_ccd(orc_model *m, const double *x0, const double *x1) {
    int *found = (int *)malloc(sizeof(int) * (size_t)m->n_edges + 1);
    double *su = (double *)malloc(sizeof(double) * 2 * (size_t)m->n_edges + 2);
    for (int e = 0; e < m->n_edges; ++e) {
        found[e] = -1;
        if (m->ee_carried[e]) continue;
        found[e] = orc_ee_first_hit(m, x0, x1, e, su + 2 * e, su + 2 * e + 1);
    }
    for (int e = 0; e < m->n_edges; ++e) {
        if (m->ee_carried[e]) continue;
        const int f = found[e];
        m->ee_partner[e] = -1;
        if (f < 0) continue;
        if (found[f] == e && f < e) continue;                   /* held by f */
        if (m->ee_carried[f] && m->ee_partner[f] == e) continue;  /* already carried by f */
        const int v[4] = {m->edges[2 * e], m->edges[2 * e + 1], m->edges[2 * f], m->edges[2 * f + 1]};
        const double s = su[2 * e], u = su[2 * e + 1];
        /* the normal: the common perpendicular e x g of the two edges at x1,
         * pointing along x_b - x_a (for two lines x_b - x_a lies along it) */
        double dlt[3], ee[3], gg[3], nrm[3];
        for (int r = 0; r < 3; ++r) {
            dlt[r] = ((1.0 - u) * x1[3 * v[2] + r] + u * x1[3 * v[3] + r]) -
                     ((1.0 - s) * x1[3 * v[0] + r] + s * x1[3 * v[1] + r]);
            ee[r] = x1[3 * v[1] + r] - x1[3 * v[0] + r];
            gg[r] = x1[3 * v[3] + r] - x1[3 * v[2] + r];
        }
        cross3(ee, gg, nrm);
        double side = dot3(nrm, dlt), len = sqrt(dot3(nrm, nrm));
        if (!(len > 0.0) || side == 0.0) continue;
        if (side < 0.0) len = -len;
        m->ee_partner[e] = f;
        m->ee_su[2 * (size_t)e] = s;
        m->ee_su[2 * (size_t)e + 1] = u;
        for (int r = 0; r < 3; ++r) m->ee_n[3 * (size_t)e + r] = nrm[r] / len;
    }
    free(found);
    free(su);
}

/* Depth of the edge-edge pair held by edge e at positions x, its four
 * vertices v and their derivative weights: d = (x_b - x_a) . n with
 * x_a = (1 - s) p0 + s p1 on edge e, x_b = (1 - u) q0 + u q1 on the partner
 * and n frozen, so dd/dx_v = c_v n with c = (-(1 - s), -s, 1 - u, u). */
static double ee_depth(const orc_model *m, int e, const double *x, int v[4], double c[4]) {
    const int f = m->ee_partner[e];
    v[0] = m->edges[2 * e]; v[1] = m->edges[2 * e + 1];
    v[2] = m->edges[2 * f]; v[3] = m->edges[2 * f + 1];
    const double s = m->ee_su[2 * (size_t)e], u = m->ee_su[2 * (size_t)e + 1];
    c[0] = -(1.0 - s); c[1] = -s; c[2] = 1.0 - u; c[3] = u;
    double d = 0.0;
    for (int j = 0; j < 4; ++j)
        for (int r = 0; r < 3; ++r) d += c[j] * x[3 * v[j] + r] * m->ee_n[3 * (size_t)e + r];
    return d;
}

void orc_ccd_edges(orc_model *m, const double *x0, const double *x1) { ee_ccd(m, x0, x1); }

int orc_ccd(orc_model *m, const double *x0, const double *x1) {
    int n = 0;
    for (int a = 0; a < m->n_verts; ++a) {
        if (m->contact[a] >= 0 && !m->contact_ccd[a]) continue;  /* keeps its step-start pair */
        double toi, w[3];
        int T = orc_ccd_vertex(m, x0, x1, a, &toi, w);
        m->contact[a] = T;
        m->contact_ccd[a] = T >= 0;
        if (T >= 0) {
            for (int k = 0; k < 3; ++k) m->contact_w[3 * (size_t)a + k] = w[k];
            ++n;
        }
    }
    return n;
}

void orc_model_contact_weights(const orc_model *m, double *w, unsigned char *is_ccd) {
    for (int a = 0; a < m->n_verts; ++a) {
        is_ccd[a] = m->contact_ccd ? m->contact_ccd[a] : 0;
        for (int k = 0; k < 3; ++k) w[3 * (size_t)a + k] = m->contact_w ? m->contact_w[3 * (size_t)a + k] : 0.0;
    }
}

int orc_model_n_verts(const orc_model *m) { return m->n_verts; }
int orc_model_n_tets(const orc_model *m) { return m->n_tets; }

void orc_model_mass(const orc_model *m, double *mass) {
    memcpy(mass, m->mass, sizeof(double) * (size_t)m->n_verts);
}

void orc_model_tet_data(const orc_model *m, double *B, double *V, double *mu, double *lam) {
    memcpy(B, m->B, sizeof(double) * 9 * (size_t)m->n_tets);
    memcpy(V, m->V, sizeof(double) * (size_t)m->n_tets);
    memcpy(mu, m->mu, sizeof(double) * (size_t)m->n_tets);
    memcpy(lam, m->lam, sizeof(double) * (size_t)m->n_tets);
}

/* Per-tet Young's modulus given as log E (the differentiable parameter). */
void orc_model_set_log_young(orc_model *m, const double *log_young) {
    for (int j = 0; j < m->n_tets; ++j) orc_lame(exp(log_young[j]), m->poisson[j], m->mu + j, m->lam + j);
}

/* ------------------------------------------------------------------ */
/* time step                                                            */
/* ------------------------------------------------------------------ */

/* Eq. 3: y = x^t + h v^t + h^2 a_ext */
void orc_inertia_target(const orc_model *m, const orc_params *p, double h,
                        const double *xt, const double *vt, double *y) {
    for (int i = 0; i < m->n_verts; ++i)
        for (int r = 0; r < 3; ++r) y[3 * i + r] = xt[3 * i + r] + h * vt[3 * i + r] + h * h * p->gravity[r];
}

/* Sec. 3.7 initialisation options (a)-(d); pinned vertices keep x^t. */
void orc_initial_guess(const orc_model *m, const orc_params *p, double h,
                       const double *xt, const double *vt, const double *vprev, double *x) {
    const double *g = p->gravity;
    double gnorm = sqrt(dot3(g, g));
    for (int i = 0; i < m->n_verts; ++i) {
        const double *xi = xt + 3 * i, *vi = vt + 3 * i, *wi = vprev + 3 * i;
        double *out = x + 3 * i;
        if (m->pinned[i]) {
            for (int r = 0; r < 3; ++r) out[r] = xi[r];
            continue;
        }
        double atil = 0.0; /* factor on a_ext */
        switch (p->init_mode) {
        case 0:
            for (int r = 0; r < 3; ++r) out[r] = xi[r];
            continue;
        case 1: atil = 0.0; break;
        case 2: atil = 1.0; break;
        default: {
            /* a^t = (v^t - v^{t-1})/h, its component along a_ext / |a_ext| */
            if (gnorm > 0.0) {
                double a_ext_comp = 0.0;
                for (int r = 0; r < 3; ++r) a_ext_comp += (vi[r] - wi[r]) / h * g[r] / gnorm;
                if (a_ext_comp > gnorm) atil = 1.0;
                else if (a_ext_comp < 0.0) atil = 0.0;
                else atil = a_ext_comp / gnorm;
            }
        }
        }
        for (int r = 0; r < 3; ++r) out[r] = xi[r] + h * vi[r] + h * h * atil * g[r];
        if (m->sub_dim[i] < 3) {
            /* a subspace-constrained vertex starts on x^t + span(Q) (Sec. 3.4) */
            const double *q = m->sub_basis + 9 * (size_t)i;
            double d[3] = {out[0] - xi[0], out[1] - xi[1], out[2] - xi[2]};
            for (int r = 0; r < 3; ++r) out[r] = xi[r];
            for (int a = 0; a < m->sub_dim[i]; ++a) {
                double c = dot3(q + 3 * a, d);
                for (int r = 0; r < 3; ++r) out[r] += c * q[3 * a + r];
            }
        }
    }
}

/* The static half-spaces of the unilateral constraints (Sec. 3.4): the ground
 * (when on) and the world-box walls, as unit normals nh and offsets c; the
 * allowed side is x.nh >= c.  Returns their number. */
static int contact_planes(const orc_params *p, double nh[1 + ORC_MAX_WALLS][3],
                          double c[1 + ORC_MAX_WALLS]) {
    int k = 0;
    if (p->ground_on) {
        double nn = sqrt(dot3(p->ground_normal, p->ground_normal));
        for (int r = 0; r < 3; ++r) nh[k][r] = p->ground_normal[r] / nn;
        c[k++] = p->ground_height;
    }
    for (int w = 0; w < p->n_walls && w < ORC_MAX_WALLS; ++w) {
        const double *n = p->walls + 4 * w;
        double nn = sqrt(dot3(n, n));
        for (int r = 0; r < 3; ++r) nh[k][r] = n[r] / nn;
        c[k++] = n[3];
    }
    return k;
}

/* G_i of Eq. 4 (inertia + incident tets) plus the contact penalties of Eq. 12
 * (ground, walls, self-contact pairs). */
double orc_local_energy(const orc_model *m, const orc_params *p, double h, int i,
                        const double *x, const double *y) {
    double d2 = 0.0;
    for (int r = 0; r < 3; ++r) d2 += (x[3 * i + r] - y[3 * i + r]) * (x[3 * i + r] - y[3 * i + r]);
    double G = m->mass[i] / (2.0 * h * h) * d2;
    for (int s = m->inc_off[i]; s < m->inc_off[i + 1]; ++s) {
        int j = m->inc_tet[s];
        double xs[12];
        gather_tet(m, j, x, xs);
        G += orc_tet_energy(xs, m->B + 9 * (size_t)j, m->V[j], m->mu[j], m->lam[j]);
    }
    double nh[1 + ORC_MAX_WALLS][3], c[1 + ORC_MAX_WALLS];
    int np = contact_planes(p, nh, c);
    for (int k = 0; k < np; ++k) {
        double d = c[k] - dot3(x + 3 * i, nh[k]);
        if (d > 0.0) G += 0.5 * p->k_c * d * d;
    }
    if (p->self_collision)
        for (int a = 0; a < m->n_verts; ++a) {
            if (m->contact[a] < 0) continue;
            const int *v = m->tris + 3 * (size_t)m->contact[a];
            if (a != i && v[0] != i && v[1] != i && v[2] != i) continue;
            double nn[3], w[3];
            double d = contact_depth(m, a, x, nn, w);
            if (d > 0.0) G += 0.5 * p->k_c * d * d;
        }
    if (p->self_collision)
        for (int e = 0; e < m->n_edges; ++e) {
            if (m->ee_partner[e] < 0) continue;
            int v[4];
            double cw[4];
            double d = ee_depth(m, e, x, v, cw);
            if (v[0] != i && v[1] != i && v[2] != i && v[3] != i) continue;
            if (d > 0.0) G += 0.5 * p->k_c * d * d;
        }
    return G;
}

/* Friction of one self-contact pair (Sec. 3.6, Eqs. 13-16), lagged: the
 * contact points move by delta = (x_a - x_a^t) - sum_k w_k (x_k - x_k^t)
 * (x_b = sum_k w_k x_k with this evaluation's weights), u is its part
 * tangent to n, and the pair's normal force magnitude lambda = k_c d scales
 * the potential mu_c lambda f0(|u|).  A vertex whose delta derivative is
 * s I (s = 1 for the colliding vertex, -w_k for corner k) gets the force
 * -s c u and the Hessian s^2 c (I - n n^T), c = mu_c lambda f1(|u|)/|u|. */
static void pair_friction(const orc_model *m, const orc_params *p, double h, int a, const int *v,
                          const double w[3], const double n[3], double lambda_n, const double *x,
                          const double *xt, double s, double f[3], double H[9]) {
    double dlt[3];
    for (int r = 0; r < 3; ++r) {
        dlt[r] = x[3 * a + r] - xt[3 * a + r];
        for (int k = 0; k < 3; ++k) dlt[r] -= w[k] * (x[3 * v[k] + r] - xt[3 * v[k] + r]);
    }
    double dn = dot3(dlt, n);
    double ut[3] = {dlt[0] - dn * n[0], dlt[1] - dn * n[1], dlt[2] - dn * n[2]};
    double um = sqrt(dot3(ut, ut));
    double eh = p->eps_v * h;
    double f1_over_u = (um < eh) ? (2.0 / eh - um / (eh * eh)) : 1.0 / um;
    double c = p->mu_c * lambda_n * f1_over_u;
    for (int r = 0; r < 3; ++r) {
        f[r] -= s * c * ut[r];
        for (int q = 0; q < 3; ++q) H[r * 3 + q] += s * s * c * ((r == q ? 1.0 : 0.0) - n[r] * n[q]);
    }
    (void)m;
}

/* Vertex-triangle penalty (Eq. 12) with the step's DCD pairs acting on
 * vertex i, as the colliding vertex and as a corner of a hit triangle: adds
 * forces to f and Hessians to H; with mu_c > 0 and xt given, the pairs'
 * friction too (h is the step size).  Returns 1 if any pair penetrates. */
int orc_self_contact(const orc_model *m, const orc_params *p, double h, int i, const double *x,
                     const double *xt, double f[3], double H[9]) {
    int hit = 0;
    double nn[3], w[3];
    const int friction = p->mu_c > 0.0 && xt != NULL;
    if (m->contact[i] >= 0) {
        double d = contact_depth(m, i, x, nn, w);
        if (d > 0.0) {
            hit = 1;
            for (int r = 0; r < 3; ++r) {
                f[r] += p->k_c * d * nn[r];
                for (int c = 0; c < 3; ++c) H[r * 3 + c] += p->k_c * nn[r] * nn[c];
            }
            if (friction)
                pair_friction(m, p, h, i, m->tris + 3 * (size_t)m->contact[i], w, nn, p->k_c * d, x, xt, 1.0,
                              f, H);
        }
    }
    for (int a = 0; a < m->n_verts; ++a) {
        if (m->contact[a] < 0) continue;
        const int *v = m->tris + 3 * (size_t)m->contact[a];
        int corner = (v[0] == i) ? 0 : (v[1] == i) ? 1 : (v[2] == i) ? 2 : -1;
        if (corner < 0) continue;
        double d = contact_depth(m, a, x, nn, w);
        if (d > 0.0) {
            hit = 1;
            double wk = w[corner];
            for (int r = 0; r < 3; ++r) {
                f[r] -= p->k_c * d * wk * nn[r];
                for (int c = 0; c < 3; ++c) H[r * 3 + c] += p->k_c * wk * wk * nn[r] * nn[c];
            }
            if (friction) pair_friction(m, p, h, a, v, w, nn, p->k_c * d, x, xt, -wk, f, H);
        }
    }
    for (int e = 0; e < m->n_edges; ++e) {  /* edge-edge pairs (Sec. 3.5), no friction */
        if (m->ee_partner[e] < 0) continue;
        int v[4];
        double c[4];
        double d = ee_depth(m, e, x, v, c);
        int j = (v[0] == i) ? 0 : (v[1] == i) ? 1 : (v[2] == i) ? 2 : (v[3] == i) ? 3 : -1;
        if (j < 0) continue;
        if (d > 0.0) {
            hit = 1;
            const double *n = m->ee_n + 3 * (size_t)e;
            for (int r = 0; r < 3; ++r) {
                f[r] -= p->k_c * d * c[j] * n[r];
                for (int q = 0; q < 3; ++q) H[r * 3 + q] += p->k_c * c[j] * c[j] * n[r] * n[q];
            }
        }
    }
    return hit;
}

/* Friction of Eqs. 13-16 against a static half-space with unit normal nh,
 * for one vertex in contact: adds the force to f and its approximate
 * Hessian to H.  f1 (Eq. 15) blends static and dynamic friction over
 * tangential displacements below eps_v h; f1(u)/u is evaluated in closed
 * form so that u = 0 is regular. */
static void plane_friction(const orc_params *p, double h, const double nh[3], const double xi[3],
                           const double xti[3], double lambda_n, double f[3], double H[9]) {
    double dlt[3] = {xi[0] - xti[0], xi[1] - xti[1], xi[2] - xti[2]};
    double dn = dot3(dlt, nh);
    double ut[3] = {dlt[0] - dn * nh[0], dlt[1] - dn * nh[1], dlt[2] - dn * nh[2]};
    double um = sqrt(dot3(ut, ut));
    double eh = p->eps_v * h;
    double f1_over_u = (um < eh) ? (2.0 / eh - um / (eh * eh)) : 1.0 / um;
    double c = p->mu_c * lambda_n * f1_over_u;
    for (int r = 0; r < 3; ++r) {
        f[r] -= c * ut[r];
        for (int s = 0; s < 3; ++s) H[r * 3 + s] += c * ((r == s ? 1.0 : 0.0) - nh[r] * nh[s]);
    }
}

/* Ground friction (Eqs. 13-16) for one vertex in ground contact. */
void orc_ground_friction(const orc_params *p, double h, const double xi[3], const double xti[3],
                         double lambda_n, double f[3], double H[9]) {
    const double *n = p->ground_normal;
    double nn = sqrt(dot3(n, n));
    double nh[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
    plane_friction(p, h, nh, xi, xti, lambda_n, f, H);
}

/* Local Newton step for vertex i (Eqs. 7-9, damping Eqs. 10-11, contact
 * Eq. 12, analytic 3x3 solve and singular skip of Sec. 3.2).  Returns 1 if
 * the vertex is skipped (dx = 0). */
int orc_vertex_solve(const orc_model *m, const orc_params *p, double h, int i,
                     const double *x, const double *y, const double *xt,
                     double dx[3], int *in_contact) {
    double f[3], H[9], Hel[9];
    double mh2 = m->mass[i] / (h * h);
    for (int r = 0; r < 3; ++r) f[r] = -mh2 * (x[3 * i + r] - y[3 * i + r]);
    for (int k = 0; k < 9; ++k) Hel[k] = 0.0;
    for (int s = m->inc_off[i]; s < m->inc_off[i + 1]; ++s) {
        int j = m->inc_tet[s], a = m->inc_loc[s];
        double xs[12], grad[12], Hb[9];
        gather_tet(m, j, x, xs);
        orc_tet_grad(xs, m->B + 9 * (size_t)j, m->V[j], m->mu[j], m->lam[j], grad);
        orc_tet_hess_block(xs, m->B + 9 * (size_t)j, m->V[j], m->mu[j], m->lam[j], a, a, Hb);
        for (int r = 0; r < 3; ++r) f[r] -= grad[3 * a + r];
        for (int k = 0; k < 9; ++k) Hel[k] += Hb[k];
    }
    for (int k = 0; k < 9; ++k) H[k] = (1.0 + p->k_d / h) * Hel[k];
    H[0] += mh2; H[4] += mh2; H[8] += mh2;
    if (p->k_d != 0.0) {
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) f[r] -= p->k_d / h * Hel[r * 3 + s] * (x[3 * i + s] - xt[3 * i + s]);
    }
    *in_contact = 0;
    double nh[1 + ORC_MAX_WALLS][3], c[1 + ORC_MAX_WALLS];
    int np = contact_planes(p, nh, c);
    for (int k = 0; k < np; ++k) {
        double d = c[k] - dot3(x + 3 * i, nh[k]);
        if (d > 0.0) {
            *in_contact = 1;
            for (int r = 0; r < 3; ++r) {
                f[r] += p->k_c * d * nh[k][r];
                for (int s = 0; s < 3; ++s) H[r * 3 + s] += p->k_c * nh[k][r] * nh[k][s];
            }
            if (p->mu_c > 0.0) plane_friction(p, h, nh[k], x + 3 * i, xt + 3 * i, p->k_c * d, f, H);
        }
    }
    if (p->self_collision && orc_self_contact(m, p, h, i, x, xt, f, H)) *in_contact = 1;
    if (m->sub_dim[i] < 3) {
        if (subspace_step(m, p, i, f, H, dx)) return 1;
    } else {
        double det = det3(H);
        double tr3 = (H[0] + H[4] + H[8]) / 3.0;
        if (fabs(det) <= p->det_eps * fabs(tr3 * tr3 * tr3)) {
            dx[0] = dx[1] = dx[2] = 0.0;
            return 1;
        }
        double A[9];
        adj3(H, A);
        for (int r = 0; r < 3; ++r) dx[r] = (A[r * 3 + 0] * f[0] + A[r * 3 + 1] * f[1] + A[r * 3 + 2] * f[2]) / det;
    }
    if (p->line_search) {
        /* backtracking from x_i + dx towards x_i on G_i (Algorithm 1) */
        double *xw = (double *)x; /* evaluated in place, restored below */
        double x0[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        double G0 = orc_local_energy(m, p, h, i, x, y);
        double alpha = 1.0;
        int ok = 0;
        for (int k = 0; k < 8 && !ok; ++k, alpha *= 0.5) {
            for (int r = 0; r < 3; ++r) xw[3 * i + r] = x0[r] + alpha * dx[r];
            if (orc_local_energy(m, p, h, i, x, y) <= G0) ok = 1;
        }
        for (int r = 0; r < 3; ++r) xw[3 * i + r] = x0[r];
        if (!ok) alpha = 0.0;
        else alpha *= 2.0; /* undo the increment of the accepting pass */
        for (int r = 0; r < 3; ++r) dx[r] *= alpha;
    }
    return 0;
}

/* One colour pass (Algorithm 1 inner loop).  Vertices of one colour share
 * no tet, so updating them in place, in any order, equals writing x^new and
 * copying back after the pass (ground contact couples no two vertices). */
void orc_sweep_color(const orc_model *m, const orc_params *p, double h, const int *colors,
                     int color, double *x, const double *y, const double *xt,
                     unsigned char *colliding, orc_stats *st) {
    /* with self-contacts two vertices of one colour may be coupled: solve all
     * against the pass-start positions (x^new), then copy back */
    size_t n3 = 3 * (size_t)m->n_verts;
    double *xs = x;
    if (p->self_collision) {
        xs = (double *)malloc(sizeof(double) * n3 + 1);
        memcpy(xs, x, sizeof(double) * n3);
    }
    /* Sec. 3.9: the vertices of one colour share no force element, so each
     * solve reads only other colours' positions (or the pass-start copy) and
     * the order does not matter; the OpenMP build of this file (timed
     * multi-core baseline) splits this loop over threads and gives the same
     * numbers bit for bit. */
    long long solves = 0, skips = 0, contacts = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : solves, skips, contacts)
#endif
    for (int i = 0; i < m->n_verts; ++i) {
        if (colors[i] != color || m->pinned[i]) continue;
        double dx[3];
        int contact;
        int skipped = orc_vertex_solve(m, p, h, i, xs, y, xt, dx, &contact);
        solves++;
        skips += skipped;
        contacts += contact;
        if (contact && colliding) colliding[i] = 1;
        for (int r = 0; r < 3; ++r) x[3 * i + r] = xs[3 * i + r] + dx[r];
    }
    if (st) {
        st->vertex_solves += solves;
        st->det_skips += skips;
        st->contacts += contacts;
    }
    if (xs != x) free(xs);
}

/* Eq. 19: omega_1 = 1, omega_2 = 2/(2 - rho^2), omega_n = 4/(4 - rho^2 omega_{n-1}) */
double orc_cheby_omega(int n, double rho, double omega_prev) {
    if (n <= 1) return 1.0;
    if (n == 2) return 2.0 / (2.0 - rho * rho);
    return 4.0 / (4.0 - rho * rho * omega_prev);
}

/* Algorithm 1 for one time step.  In: x = x^t, v = v^t, vprev = v^{t-1}.
 * Out: x = x^{t+1}, v = v^{t+1}, vprev = v^t.  Returns 0. */
int orc_step(const orc_model *m, const orc_params *p, const int *colors, int n_colors,
             double h, int iters, double *x, double *v, double *vprev, orc_stats *st) {
    size_t n3 = 3 * (size_t)m->n_verts;
    double *xt = (double *)malloc(sizeof(double) * n3 + 1);
    double *y = (double *)malloc(sizeof(double) * n3 + 1);
    double *p1 = (double *)malloc(sizeof(double) * n3 + 1);
    double *p2 = (double *)malloc(sizeof(double) * n3 + 1);
    unsigned char *coll = (unsigned char *)calloc((size_t)m->n_verts + 1, 1);
    memcpy(xt, x, sizeof(double) * n3);
    if (p->self_collision) orc_dcd((orc_model *)m, p, xt);  /* initial DCD using x^t */
    orc_inertia_target(m, p, h, xt, v, y);            /* Eq. 3 */
    orc_initial_guess(m, p, h, xt, v, vprev, x);      /* Sec. 3.7 */
    memcpy(p1, x, sizeof(double) * n3);               /* x^(0) */
    double omega = 1.0;
    double *xj = p->jacobi ? (double *)malloc(sizeof(double) * n3 + 1) : NULL;
    for (int n = 1; n <= iters; ++n) {
        /* CCD along x^t -> x^(n-1) before every ccd_interval-th iteration (Sec. 3.5) */
        if (p->self_collision && p->ccd_interval > 0 && (n - 1) % p->ccd_interval == 0) {
            orc_ccd((orc_model *)m, xt, x);
            if (p->ccd_edges) orc_ccd_edges((orc_model *)m, xt, x);
        }
        if (p->jacobi) {
            /* block Jacobi: solve every free vertex against the previous iterate */
            memcpy(xj, x, sizeof(double) * n3);
            long long solves = 0, skips = 0, contacts = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : solves, skips, contacts)
#endif
            for (int i = 0; i < m->n_verts; ++i) {
                if (m->pinned[i]) continue;
                double dx[3];
                int contact;
                int skipped = orc_vertex_solve(m, p, h, i, x, y, xt, dx, &contact);
                solves++;
                skips += skipped;
                contacts += contact;
                if (contact) coll[i] = 1;
                for (int r = 0; r < 3; ++r) xj[3 * i + r] = x[3 * i + r] + dx[r];
            }
            if (st) {
                st->vertex_solves += solves;
                st->det_skips += skips;
                st->contacts += contacts;
            }
            memcpy(x, xj, sizeof(double) * n3);
        } else {
            for (int c = 0; c < n_colors; ++c) orc_sweep_color(m, p, h, colors, c, x, y, xt, coll, st);
        }
        if (p->cheby_rho > 0.0) {
            omega = orc_cheby_omega(n, p->cheby_rho, omega);   /* Eq. 19 */
            for (int i = 0; i < m->n_verts; ++i) {
                for (int r = 0; r < 3; ++r) {
                    size_t q = 3 * (size_t)i + r;
                    double xbar = x[q];
                    double xn = xbar;
                    if (n >= 2 && !m->pinned[i] && !coll[i]) xn = omega * (xbar - p2[q]) + p2[q]; /* Eq. 18 */
                    p2[q] = p1[q];
                    p1[q] = xn;
                    x[q] = xn;
                }
            }
        }
    }
    for (size_t q = 0; q < n3; ++q) {                  /* Eq. 6 */
        double vn = (x[q] - xt[q]) / h;
        vprev[q] = v[q];
        v[q] = vn;
    }
    free(xt); free(y); free(p1); free(p2); free(coll); free(xj);
    return 0;
}

/* ------------------------------------------------------------------ */
/* diagnostics and assembly                                             */
/* ------------------------------------------------------------------ */

/* Eq. 2 variational energy G(x) = 1/(2h^2) |x - y|_M^2 + E(x) over the free
 * vertices, with the ground and wall penalties of Eq. 12 when enabled. */
double orc_energy_G(const orc_model *m, const orc_params *p, double h,
                    const double *x, const double *y) {
    double G = 0.0;
    double nh[1 + ORC_MAX_WALLS][3], c[1 + ORC_MAX_WALLS];
    int np = contact_planes(p, nh, c);
    for (int i = 0; i < m->n_verts; ++i) {
        if (m->pinned[i]) continue;
        double d2 = 0.0;
        for (int r = 0; r < 3; ++r) d2 += (x[3 * i + r] - y[3 * i + r]) * (x[3 * i + r] - y[3 * i + r]);
        G += m->mass[i] / (2.0 * h * h) * d2;
        for (int k = 0; k < np; ++k) {
            double d = c[k] - dot3(x + 3 * i, nh[k]);
            if (d > 0.0) G += 0.5 * p->k_c * d * d;
        }
    }
    for (int j = 0; j < m->n_tets; ++j) {
        double xs[12];
        gather_tet(m, j, x, xs);
        G += orc_tet_energy(xs, m->B + 9 * (size_t)j, m->V[j], m->mu[j], m->lam[j]);
    }
    if (p->self_collision) {
        for (int a = 0; a < m->n_verts; ++a)
            if (m->contact[a] >= 0) {
                double nn[3], w[3];
                double d = contact_depth(m, a, x, nn, w);
                if (d > 0.0) G += 0.5 * p->k_c * d * d;
            }
        for (int e = 0; e < m->n_edges; ++e) {
            if (m->ee_partner[e] < 0) continue;
            int v[4];
            double cw[4];
            double d = ee_depth(m, e, x, v, cw);
            if (d > 0.0) G += 0.5 * p->k_c * d * d;
        }
    }
    return G;
}

int orc_model_n_edges(const orc_model *m) { return m->n_edges; }

void orc_model_edges(const orc_model *m, int *edges) {
    memcpy(edges, m->edges, sizeof(int) * 2 * (size_t)m->n_edges);
}

/* the current edge-edge pairs, by holding edge: partner (or -1), carried
 * flag, (s, u) and the normal per edge; returns the number of pairs */
int orc_model_ee_pairs(const orc_model *m, int *partner, unsigned char *carried, double *su, double *n) {
    int k = 0;
    for (int e = 0; e < m->n_edges; ++e) k += m->ee_partner[e] >= 0;
    if (partner) memcpy(partner, m->ee_partner, sizeof(int) * (size_t)m->n_edges);
    if (carried) memcpy(carried, m->ee_carried, (size_t)m->n_edges);
    if (su) memcpy(su, m->ee_su, sizeof(double) * 2 * (size_t)m->n_edges);
    if (n) memcpy(n, m->ee_n, sizeof(double) * 3 * (size_t)m->n_edges);
    return k;
}

void orc_elastic_grad(const orc_model *m, const double *x, double *grad) {
    memset(grad, 0, sizeof(double) * 3 * (size_t)m->n_verts);
    for (int j = 0; j < m->n_tets; ++j) {
        double xs[12], g[12];
        gather_tet(m, j, x, xs);
        orc_tet_grad(xs, m->B + 9 * (size_t)j, m->V[j], m->mu[j], m->lam[j], g);
        for (int a = 0; a < 4; ++a)
            for (int r = 0; r < 3; ++r) grad[3 * m->tets[4 * j + a] + r] += g[3 * a + r];
    }
}

/* 144 (row, col, value) triplets per tet, global DoF indices 3*i + r. */
void orc_elastic_hess_triplets(const orc_model *m, const double *x,
                               int *rows, int *cols, double *vals) {
    for (int j = 0; j < m->n_tets; ++j) {
        double xs[12], H[144];
        gather_tet(m, j, x, xs);
        orc_tet_hess(xs, m->B + 9 * (size_t)j, m->V[j], m->mu[j], m->lam[j], H);
        for (int a = 0; a < 12; ++a)
            for (int b = 0; b < 12; ++b) {
                size_t q = 144 * (size_t)j + 12 * a + b;
                rows[q] = 3 * m->tets[4 * j + a / 3] + a % 3;
                cols[q] = 3 * m->tets[4 * j + b / 3] + b % 3;
                vals[q] = H[a * 12 + b];
            }
    }
}

void orc_tet_grads(const orc_model *m, const double *x, double *g12) {
    for (int j = 0; j < m->n_tets; ++j) {
        double xs[12];
        gather_tet(m, j, x, xs);
        orc_tet_grad(xs, m->B + 9 * (size_t)j, m->V[j], m->mu[j], m->lam[j], g12 + 12 * (size_t)j);
    }
}

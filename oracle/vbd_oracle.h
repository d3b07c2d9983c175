/*
 * vbd_oracle.h -- serial FP64 CPU oracle for Vertex Block Descent
 * (Chen, Liu, Yang, Yuksel, "Vertex Block Descent", ACM TOG 43(4), 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes,
 * links or calls this code; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no header, helper or table
 * with the CUDA path.
 *
 * Every routine is a direct transcription of the paper's definitions
 * (Sec. 3.1 Eqs. 1-6, Sec. 3.2 Eqs. 7-9, Sec. 3.3 Eqs. 10-11, Sec. 3.5
 * Eq. 12, Sec. 3.7 options (a)-(d) and Eq. 17, Sec. 3.8 Eqs. 18-19,
 * Algorithm 1), in FP64,
 * with plain loops and no blocking or reordering.  Where the paper is
 * silent (material formula, Lame mapping, lumped mass, det threshold,
 * colouring algorithm) the readings are stated next to the code.
 *
 * Pins: every function is checked by tests against finite differences,
 * invariances, closed forms or brute force (tests/test_oracle_*.py).
 */
#ifndef VBD_ORACLE_H
#define VBD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_model orc_model;

typedef struct {
    double gravity[3];      /* a_ext of Eq. 3 */
    int ground_on;          /* ground half-space penalty of Eq. 12 */
    double ground_height;   /* plane {x : x.n = ground_height} */
    double ground_normal[3];
    double k_c;             /* collision stiffness, Eq. 12 */
    double cheby_rho;       /* Eqs. 18-19 spectral radius; 0 = no acceleration */
    int init_mode;          /* Sec. 3.7: 0 previous, 1 inertia, 2 inertia+acc, 3 adaptive */
    double det_eps;         /* relative threshold of the Sec. 3.2 singular-Hessian skip */
    double k_d;             /* Rayleigh damping coefficient, Eqs. 10-11 (0 = off) */
    double mu_c;            /* ground friction coefficient, Eqs. 13-16 (0 = off) */
    double eps_v;           /* friction velocity threshold of Eq. 15 [m/s] */
    int line_search;        /* 1: backtracking on G_i after each local step (Sec. 3.2) */
    int jacobi;             /* 1: block Jacobi: all vertices from the previous iterate */
    int self_collision;     /* 1: vertex-triangle penalty contacts from a DCD at x^t (Sec. 3.5) */
    double dcd_radius;      /* DCD search radius */
    int ccd_interval;       /* > 0: vertex-triangle CCD before every ccd_interval-th iteration (Sec. 3.5) */
    int ccd_edges;          /* 1: the CCD also pairs crossing boundary edges (Sec. 3.5) */
    int n_walls;            /* world-box walls (Sec. 3.4), 0..ORC_MAX_WALLS */
    double walls[4 * 6];    /* wall k: normal walls[4k..4k+2] (any length), offset walls[4k+3];
                               the allowed side is x.n/|n| >= offset */
} orc_params;

#define ORC_MAX_WALLS 6

typedef struct {
    long long vertex_solves;   /* local solves performed */
    long long det_skips;       /* solves skipped by the |det H| test */
    long long contacts;        /* solves that saw a ground, wall or self-contact penetration */
} orc_stats;

/* ---- materials and element (Sec. 5: stable neo-Hookean without log term) -- */
void orc_lame(double E, double nu, double *mu, double *lam);
int orc_rest_tet(const double X[12], double B[9], double *V);
void orc_tet_F(const double x[12], const double B[9], double F[9]);
double orc_nh_psi(const double F[9], double mu, double lam);
void orc_nh_pk1(const double F[9], double mu, double lam, double P[9]);
void orc_cofactor(const double F[9], double C[9]);
double orc_tet_energy(const double x[12], const double B[9], double V, double mu, double lam);
void orc_tet_grad(const double x[12], const double B[9], double V, double mu, double lam,
                  double grad[12]);
void orc_tet_hess_block(const double x[12], const double B[9], double V, double mu, double lam,
                        int k, int l, double Hkl[9]);
void orc_tet_hess(const double x[12], const double B[9], double V, double mu, double lam,
                  double H[144]);

/* ---- colouring (Sec. 3.9) --------------------------------------------- */
int orc_color_greedy(int n_verts, int n_tets, const int *tets, int *colors);
int orc_color_valid(int n_verts, int n_tets, const int *tets, const int *colors);

/* ---- model -------------------------------------------------------------- */
orc_model *orc_model_new(int n_verts, int n_tets, const double *rest, const int *tets,
                         const double *young, const double *poisson, const double *density,
                         const unsigned char *pinned, int *status);
void orc_model_free(orc_model *m);
int orc_model_n_verts(const orc_model *m);
int orc_model_n_tets(const orc_model *m);
void orc_model_mass(const orc_model *m, double *mass);
void orc_model_tet_data(const orc_model *m, double *B, double *V, double *mu, double *lam);
void orc_model_set_log_young(orc_model *m, const double *log_young);

/* ---- self-collision (Sec. 3.5: vertex-triangle, DCD at the step start) -- */
int orc_model_n_tris(const orc_model *m);
void orc_model_tris(const orc_model *m, int *tris);
void orc_closest_point_tri(const double p[3], const double a[3], const double b[3], const double c[3],
                           double q[3], double w[3]);
int orc_point_in_tet(const double *x, const int *tet, const double q[3]);
int orc_dcd_vertex(const orc_model *m, const orc_params *p, const double *x, int a);
void orc_dcd(orc_model *m, const orc_params *p, const double *x);
/* Vertex-triangle CCD along x(tau) = (1 - tau) x0 + tau x1, tau in [0, 1]
 * (Sec. 3.5): earliest impact of boundary vertex a with a boundary triangle
 * that shares no tet with it; returns the triangle (or -1) with its time of
 * impact and the barycentric weights of the impact point. */
int orc_ccd_vertex(const orc_model *m, const double *x0, const double *x1, int a, double *toi, double w[3]);
/* CCD of every boundary vertex without a step-start (DCD) pair; replaces the
 * previous CCD pairs.  Returns the number of CCD pairs. */
int orc_ccd(orc_model *m, const double *x0, const double *x1);
/* the edge-edge part of the CCD alone (pairs held by the edges) */
void orc_ccd_edges(orc_model *m, const double *x0, const double *x1);
/* Sec. 3.5, one edge of the edge-edge CCD: the boundary edge that edge e
 * (an index of orc_model_edges) hits first along the straight paths x0 -> x1
 * (ties within 1e-5 in time: the lowest index), among the edges none of
 * whose vertices shares a tet with one of e's; -1 if none, else the impact
 * parameters on e and on the partner in s_out, u_out. */
int orc_ee_first_hit(const orc_model *m, const double *x0, const double *x1, int e, double *s_out,
                     double *u_out);
/* Earliest root in [0, 1] of c0 + c1 t + c2 t^2 + c3 t^3 at or after t_min
 * whose point passes `accept`; -1 if none (exposed for the pins). */
double orc_cubic_first_root(const double c[4], double t_min);
void orc_model_contact_weights(const orc_model *m, double *w, unsigned char *is_ccd);
/* edge-edge CCD of one edge pair; returns the time of impact or -1 */
double orc_ee_impact(const double *x0, const double *x1, int p0, int p1, int q0, int q1, double *s, double *u);
int orc_model_n_edges(const orc_model *m);
void orc_model_edges(const orc_model *m, int *edges);
int orc_model_ee_pairs(const orc_model *m, int *partner, unsigned char *carried, double *su, double *n);
void orc_model_contacts(const orc_model *m, int *contact);
int orc_self_contact(const orc_model *m, const orc_params *p, double h, int i, const double *x,
                     const double *xt, double f[3], double H[9]);

/* Subspace constraint of Sec. 3.4 on vertex i: L = 1 line (dir = direction),
 * 2 plane (dir = normal), 3 = none.  Returns 0, or 1 for a bad argument. */
int orc_model_set_subspace(orc_model *m, int i, int L, const double dir[3]);

/* ---- one time step (Algorithm 1) --------------------------------------- */
void orc_inertia_target(const orc_model *m, const orc_params *p, double h,
                        const double *xt, const double *vt, double *y);
void orc_initial_guess(const orc_model *m, const orc_params *p, double h,
                       const double *xt, const double *vt, const double *vprev, double *x);
void orc_ground_friction(const orc_params *p, double h, const double xi[3], const double xti[3],
                         double lambda_n, double f[3], double H[9]);
int orc_vertex_solve(const orc_model *m, const orc_params *p, double h, int i,
                     const double *x, const double *y, const double *xt,
                     double dx[3], int *in_contact);
void orc_sweep_color(const orc_model *m, const orc_params *p, double h, const int *colors,
                     int color, double *x, const double *y, const double *xt,
                     unsigned char *colliding, orc_stats *st);
double orc_cheby_omega(int n, double rho, double omega_prev);
double orc_local_energy(const orc_model *m, const orc_params *p, double h, int i,
                        const double *x, const double *y);
int orc_step(const orc_model *m, const orc_params *p, const int *colors, int n_colors,
             double h, int iters, double *x, double *v, double *vprev, orc_stats *st);

/* ---- diagnostics, assembly for the dense Newton / adjoint pins ---------- */
double orc_energy_G(const orc_model *m, const orc_params *p, double h,
                    const double *x, const double *y);
void orc_elastic_grad(const orc_model *m, const double *x, double *grad);
void orc_elastic_hess_triplets(const orc_model *m, const double *x,
                               int *rows, int *cols, double *vals);
void orc_tet_grads(const orc_model *m, const double *x, double *g12);

#ifdef __cplusplus
}
#endif
#endif

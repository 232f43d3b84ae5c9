/*
 * lhe_oracle.h -- plain, slow FP64 CPU oracle for the fourth-order BGK lattice
 * Boltzmann model of the d-dimensional linear hyperbolic equation
 * (Chen, Chai & Shi, arXiv:2410.13165).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference arm may load this library. It shares no code, header,
 * table or constant with the CUDA library in paper_2410_13165_gb300/.
 *
 * Conventions (the paper's own formulation, not the GPU library's):
 *   - the state is the PRE-collision population f_k(x, t_n);
 *   - one step collides at every node, then PUSHES f*_k(x) to x + e_k
 *     (Eq. BGK-LB-Evolution: the left-hand side is f_k(x + c_k dt, t + dt));
 *   - populations are stored k-major: f[k*S + site], site = i_1 + n_1*(i_2 + n_2*(...));
 *   - unit lattice vectors e_k (entries in {-1,0,1}); physical velocity c_k = c e_k,
 *     c = dx/dt (acoustic scaling, Sec. 2.2).
 * Every function is pinned by a `-m "not gpu"` test against what the paper or the
 * mathematics fixes (see tests/test_oracle_*.py).
 */
#ifndef LHE_ORACLE_H
#define LHE_ORACLE_H
#include <stdint.h>

#define ORC_MAXD 5
#define ORC_MAXQ 51
#define ORC_MAXMODES 16

/* Model description filled by the Python wrapper from the functions below. */
typedef struct {
  int d, Q;
  int64_t n[ORC_MAXD];        /* nodes per dimension */
  double x0[ORC_MAXD];        /* physical coordinate of node 0 along each axis */
  double dx, dt;              /* lattice spacing and time step; c = dx/dt */
  double u[ORC_MAXD];         /* transport velocity (physical units) */
  double s;                   /* relaxation parameter s = 1/tau */
  double R;                   /* constant source term */
  int e[ORC_MAXQ * ORC_MAXD]; /* unit lattice vectors, e[k*d + i] */
  double omega[ORC_MAXQ];     /* EDF weights, f^eq_k = omega_k phi */
  int bc;                     /* 0 periodic, 1 full-way Dirichlet, 2 half-way Dirichlet */
  int bc_order;               /* full-way 1|3|4, half-way 1..4 */
} orc_model;

/* Exact solution family of the L-HE with constant R (initial and Dirichlet data):
 * phi(x,t) = b + R t + sum_i g_i (x_i - u_i t) + sum_m a_m sin(kappa_m . (x - u t) + theta_m). */
typedef struct {
  int nmodes;
  double b;
  double g[ORC_MAXD];
  double a[ORC_MAXMODES];
  double kappa[ORC_MAXMODES * ORC_MAXD];
  double theta[ORC_MAXMODES];
} orc_wave;

/* ---- lattice and equilibrium (Sec. 2.3, Sec. 4.1) ---- */
int orc_velocities(int d, int *e);                      /* returns Q, fills e[Q*d] */
int orc_moment_matrix(int d, const int *e, double *M);  /* natural-moment matrix, row-major Q x Q */
int orc_eps(int d, const double *sigma, const double *m4pairs, double *eps); /* Eq. (meq) */
double orc_m4_rule(int d, const double *sigma, double g); /* Eq. (meq-4rd) */
int orc_weights_closed(int d, const double *sigma, const double *m4pairs, double *omega); /* Eq. (omega_k-2) */
int orc_solve(int n, double *A, double *b);             /* Gaussian elimination, A x = b, b <- x */

/* ---- the scheme ---- */
void orc_set_threads(int nthreads);
void orc_init(const orc_model *m, int order, const double *phi0, const double *grad, double *f);
void orc_fd_grad(const orc_model *m, const double *phi, double *grad);
void orc_step(const orc_model *m, const orc_wave *w, int64_t n, const double *Rfield,
              const double *f, double *fstar, double *fnew);
void orc_phi(const orc_model *m, const double *f, double *phi);
double orc_exact(const orc_model *m, const orc_wave *w, const double *x, double t);
double orc_dir_deriv(const orc_model *m, const orc_wave *w, const double *x, double t,
                     const double *c, int p, int q);
void orc_node_coord(const orc_model *m, int64_t site, double *x);
/* the exact solution at every node (out[S]) and its spatial gradient (out[d*S]) at time t */
void orc_exact_field(const orc_model *m, const orc_wave *w, double t, double *out);
void orc_exact_grad_field(const orc_model *m, const orc_wave *w, double t, double *out);

/* ---- diagnostics ---- */
double orc_entropy(const orc_model *m, const double *f); /* sum_x sum_k f_k^2/(2 omega_k), Eq. (skfk) */

/* ---- discrete adjoint (periodic and Dirichlet boxes; see orc_adjoint_step) ---- */
void orc_adjoint_step(const orc_model *m, const double *lam_next, double *lam, double *gR);
void orc_adjoint_init(const orc_model *m, int order, int grad_is_fd, const double *lam0,
                      double *gphi0, double *ggrad);
#endif

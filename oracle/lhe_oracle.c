/*
 * lhe_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see lhe_oracle.h).
 *
 * Written from the paper (arXiv:2410.13165) in its order and notation:
 *   velocity set           Sec. 2.3, Eq. (DdQ-M) with the J_1/J_2 blocks of the d>3 case
 *   natural moments        Eq. (DdQ-M) rows, moment vector Eq. (meq), Eq. (third-condition-2)
 *   4th-order moments      Eq. (meq-4rd) (Remark 5), equal for every pair i<j
 *   EDF weights            Eq. (omega_k-2); cross-checked by solving M omega = eps
 *   evolution              Eq. (BGK-LB-Evolution), general s (s = 2: Eq. BGK-LB-Evolution-seq2)
 *   initialisation         Eq. (ini-simp) (third order) and f = f^eq (first order)
 *   full-way Dirichlet     Eq. (bun1), orders 1, 3, 4
 *   half-way Dirichlet     Eq. (bun2), orders 1..4 (the unknown is f_k(x_f, t+dt); the sum
 *                          f_k(x_f,t+dt) + f*_kbar(x_f,t) is what the appendix construction fixes)
 *   kinetic entropy        Eq. (skfk)
 * Build with -O2 -ffp-contract=off so no multiply-add is fused behind the source's back.
 */
#include "lhe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void orc_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

/* ------------------------------------------------------------------ lattice */

/* Eq. (DdQ-M): rest velocity; +e_1..+e_d (the Q_p blocks' +1 entries); -e_1..-e_d;
 * then for every pair i<j, four velocities with component i from J_1 = (1,-1,-1,1)
 * and component j from J_2 = (1,1,-1,-1). */
int orc_velocities(int d, int *e) {
  static const int J1[4] = {1, -1, -1, 1}, J2[4] = {1, 1, -1, -1};
  if (d < 1 || d > ORC_MAXD) return -1;
  const int Q = 2 * d * d + 1;
  memset(e, 0, sizeof(int) * (size_t)Q * d);
  int k = 1;
  for (int i = 0; i < d; ++i) e[(k++) * d + i] = 1;
  for (int i = 0; i < d; ++i) e[(k++) * d + i] = -1;
  for (int i = 0; i < d; ++i)
    for (int j = i + 1; j < d; ++j)
      for (int r = 0; r < 4; ++r) {
        e[k * d + i] = J1[r];
        e[k * d + j] = J2[r];
        ++k;
      }
  return Q;
}

/* Rows of M in the paper's order: 1; c^{x_i}; (c^{x_i})^2; c^{x_i}c^{x_j} (i<j);
 * (c^{x_i})^2 c^{x_j} (i = 1..d, j != i); (c^{x_i})^2 (c^{x_j})^2 (i<j). Unit lattice (c = 1). */
int orc_moment_matrix(int d, const int *e, double *M) {
  const int Q = 2 * d * d + 1;
  for (int k = 0; k < Q; ++k) {
    const int *ck = e + k * d;
    int r = 0;
    M[(r++) * Q + k] = 1.0;
    for (int i = 0; i < d; ++i) M[(r++) * Q + k] = ck[i];
    for (int i = 0; i < d; ++i) M[(r++) * Q + k] = ck[i] * ck[i];
    for (int i = 0; i < d; ++i)
      for (int j = i + 1; j < d; ++j) M[(r++) * Q + k] = ck[i] * ck[j];
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        if (j != i) M[(r++) * Q + k] = ck[i] * ck[i] * ck[j];
    for (int i = 0; i < d; ++i)
      for (int j = i + 1; j < d; ++j) M[(r++) * Q + k] = ck[i] * ck[i] * ck[j] * ck[j];
    if (r != Q) return -1;
  }
  return Q;
}

/* Eq. (meq) in lattice units (sigma = u/c): [1, sigma, (1+2 sigma_i^2)/3, 2 sigma_i sigma_j/3,
 * sigma_j/3 for the row (x_i^2 x_j), m4_ij]; m4pairs lists pairs i<j lexicographically. */
int orc_eps(int d, const double *sigma, const double *m4pairs, double *eps) {
  int r = 0;
  eps[r++] = 1.0;
  for (int i = 0; i < d; ++i) eps[r++] = sigma[i];
  for (int i = 0; i < d; ++i) eps[r++] = (1.0 + 2.0 * sigma[i] * sigma[i]) / 3.0;
  for (int i = 0; i < d; ++i)
    for (int j = i + 1; j < d; ++j) eps[r++] = 2.0 * sigma[i] * sigma[j] / 3.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (j != i) eps[r++] = sigma[j] / 3.0;
  int p = 0;
  for (int i = 0; i < d; ++i)
    for (int j = i + 1; j < d; ++j) eps[r++] = m4pairs[p++];
  return r;
}

/* Eq. (meq-4rd): m4 = g * max{lower bounds} + (1 - g) * min{upper bounds}, lattice units. */
double orc_m4_rule(int d, const double *sigma, double g) {
  if (d < 2) return 0.0;
  double sum2 = 0.0;
  for (int i = 0; i < d; ++i) sum2 += sigma[i] * sigma[i];
  double lo = (-6.0 + 2.0 * d + 4.0 * sum2) / (3.0 * d * (d - 1));
  for (int i = 0; i < d; ++i)
    for (int j = i + 1; j < d; ++j) {
      const double a = (fabs(sigma[i] + sigma[j]) - 2.0 * sigma[i] * sigma[j]) / 3.0;
      const double b = (fabs(sigma[i] - sigma[j]) + 2.0 * sigma[i] * sigma[j]) / 3.0;
      if (a > lo) lo = a;
      if (b > lo) lo = b;
    }
  double hi = 1e300;
  for (int i = 0; i < d; ++i) {
    const double v = (1.0 + 2.0 * sigma[i] * sigma[i] - fabs((4.0 - d) * sigma[i])) / (3.0 * (d - 1));
    if (v < hi) hi = v;
  }
  return g * lo + (1.0 - g) * hi;
}

static int pair_index(int d, int i, int j) { /* lexicographic index of pair i<j */
  int p = 0;
  for (int a = 0; a < d; ++a)
    for (int b = a + 1; b < d; ++b) {
      if (a == i && b == j) return p;
      ++p;
    }
  return -1;
}

/* Eq. (omega_k-2) with c = 1 (lattice units) and per-pair fourth moments m4_ij. */
int orc_weights_closed(int d, const double *sigma, const double *m4pairs, double *omega) {
  int e[ORC_MAXQ * ORC_MAXD];
  const int Q = orc_velocities(d, e);
  if (Q < 0) return -1;
  double sum2 = 0.0, m4all = 0.0;
  for (int i = 0; i < d; ++i) sum2 += sigma[i] * sigma[i];
  for (int p = 0; p < d * (d - 1) / 2; ++p) m4all += m4pairs[p];
  for (int k = 0; k < Q; ++k) {
    const int *ck = e + k * d;
    int nz = 0, ia = -1, ib = -1;
    for (int i = 0; i < d; ++i)
      if (ck[i] != 0) {
        if (nz == 0) ia = i; else ib = i;
        ++nz;
      }
    if (nz == 0) {
      omega[k] = (3.0 - d - 2.0 * sum2 + 3.0 * m4all) / 3.0;
    } else if (nz == 1) {
      double m4row = 0.0;
      for (int j = 0; j < d; ++j)
        if (j != ia) m4row += m4pairs[ia < j ? pair_index(d, ia, j) : pair_index(d, j, ia)];
      omega[k] = (ck[ia] * (4.0 - d) * sigma[ia] + 1.0 + 2.0 * sigma[ia] * sigma[ia] - 3.0 * m4row) / 6.0;
    } else {
      const double m4 = m4pairs[pair_index(d, ia, ib)];
      const double si = ck[ia], sj = ck[ib];
      omega[k] = (3.0 * m4 + 2.0 * si * sj * sigma[ia] * sigma[ib] + si * sigma[ia] + sj * sigma[ib]) / 12.0;
    }
  }
  return Q;
}

/* Gaussian elimination with partial pivoting; returns 0 on success, -1 if singular. */
int orc_solve(int n, double *A, double *b) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(A[r * n + col]) > fabs(A[piv * n + col])) piv = r;
    if (fabs(A[piv * n + col]) < 1e-300) return -1;
    if (piv != col) {
      for (int c = 0; c < n; ++c) {
        const double t = A[col * n + c];
        A[col * n + c] = A[piv * n + c];
        A[piv * n + c] = t;
      }
      const double t = b[col];
      b[col] = b[piv];
      b[piv] = t;
    }
    for (int r = col + 1; r < n; ++r) {
      const double f = A[r * n + col] / A[col * n + col];
      for (int c = col; c < n; ++c) A[r * n + c] -= f * A[col * n + c];
      b[r] -= f * b[col];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double acc = b[r];
    for (int c = r + 1; c < n; ++c) acc -= A[r * n + c] * b[c];
    b[r] = acc / A[r * n + r];
  }
  return 0;
}

/* ------------------------------------------------------------------ geometry */

static int64_t n_sites(const orc_model *m) {
  int64_t S = 1;
  for (int i = 0; i < m->d; ++i) S *= m->n[i];
  return S;
}

static void site_to_idx(const orc_model *m, int64_t site, int64_t *idx) {
  for (int i = 0; i < m->d; ++i) {
    idx[i] = site % m->n[i];
    site /= m->n[i];
  }
}

static int64_t idx_to_site(const orc_model *m, const int64_t *idx) {
  int64_t s = 0;
  for (int i = m->d - 1; i >= 0; --i) s = s * m->n[i] + idx[i];
  return s;
}

void orc_node_coord(const orc_model *m, int64_t site, double *x) {
  int64_t idx[ORC_MAXD];
  site_to_idx(m, site, idx);
  for (int i = 0; i < m->d; ++i) x[i] = m->x0[i] + (double)idx[i] * m->dx;
}

static int opposite(const orc_model *m, int k) {
  for (int j = 0; j < m->Q; ++j) {
    int same = 1;
    for (int i = 0; i < m->d; ++i)
      if (m->e[j * m->d + i] != -m->e[k * m->d + i]) same = 0;
    if (same) return j;
  }
  return -1;
}

/* ------------------------------------------------------------------ exact solution */

static double sin_deriv(double xi, int j) { /* j-th derivative of sin at xi */
  switch (j & 3) {
    case 0: return sin(xi);
    case 1: return cos(xi);
    case 2: return -sin(xi);
    default: return -cos(xi);
  }
}

/* d_t^q (c . grad)^p phi(x, t) for the exact-solution family of lhe_oracle.h. */
double orc_dir_deriv(const orc_model *m, const orc_wave *w, const double *x, double t,
                     const double *c, int p, int q) {
  const int d = m->d;
  double r = 0.0;
  if (p == 0 && q == 0) {
    r += w->b + m->R * t;
    for (int i = 0; i < d; ++i) r += w->g[i] * (x[i] - m->u[i] * t);
  } else if (p == 0 && q == 1) {
    r += m->R;
    for (int i = 0; i < d; ++i) r -= w->g[i] * m->u[i];
  } else if (p == 1 && q == 0) {
    for (int i = 0; i < d; ++i) r += w->g[i] * c[i];
  }
  for (int mo = 0; mo < w->nmodes; ++mo) {
    const double *kap = w->kappa + mo * ORC_MAXD;
    double xi = w->theta[mo], kc = 0.0, ku = 0.0;
    for (int i = 0; i < d; ++i) {
      xi += kap[i] * (x[i] - m->u[i] * t);
      kc += kap[i] * c[i];
      ku += kap[i] * m->u[i];
    }
    double fac = w->a[mo];
    for (int a = 0; a < p; ++a) fac *= kc;
    for (int a = 0; a < q; ++a) fac *= -ku;
    r += fac * sin_deriv(xi, p + q);
  }
  return r;
}

double orc_exact(const orc_model *m, const orc_wave *w, const double *x, double t) {
  double zero[ORC_MAXD] = {0};
  return orc_dir_deriv(m, w, x, t, zero, 0, 0);
}

void orc_exact_field(const orc_model *m, const orc_wave *w, double t, double *out) {
  const int64_t S = n_sites(m);
#pragma omp parallel for schedule(static)
  for (int64_t site = 0; site < S; ++site) {
    double x[ORC_MAXD];
    orc_node_coord(m, site, x);
    out[site] = orc_exact(m, w, x, t);
  }
}

void orc_exact_grad_field(const orc_model *m, const orc_wave *w, double t, double *out) {
  const int64_t S = n_sites(m);
#pragma omp parallel for schedule(static)
  for (int64_t site = 0; site < S; ++site) {
    double x[ORC_MAXD];
    orc_node_coord(m, site, x);
    for (int i = 0; i < m->d; ++i) {
      double c[ORC_MAXD] = {0};
      c[i] = 1.0;
      out[(int64_t)i * S + site] = orc_dir_deriv(m, w, x, t, c, 1, 0);
    }
  }
}

/* ------------------------------------------------------------------ scheme */

/* Eq. (ini-simp): f_k(x,0) = omega_k [phi0 + (dt/2) (u - c_k) . grad phi0]  (order 3),
 * or f_k = f^eq_k = omega_k phi0 (order 1). grad is laid out grad[i*S + site]. */
void orc_init(const orc_model *m, int order, const double *phi0, const double *grad, double *f) {
  const int64_t S = n_sites(m);
  const double c = m->dx / m->dt;
  for (int64_t site = 0; site < S; ++site) {
    for (int k = 0; k < m->Q; ++k) {
      double val = phi0[site];
      if (order == 3) {
        double dot = 0.0;
        for (int i = 0; i < m->d; ++i) dot += (m->u[i] - c * m->e[k * m->d + i]) * grad[(int64_t)i * S + site];
        val = val + 0.5 * m->dt * dot;
      }
      f[(int64_t)k * S + site] = m->omega[k] * val;
    }
  }
}

/* Fourth-order central difference of a periodic field: d_i phi ~
 * (-phi(x+2e_i) + 8 phi(x+e_i) - 8 phi(x-e_i) + phi(x-2e_i)) / (12 dx). */
void orc_fd_grad(const orc_model *m, const double *phi, double *grad) {
  const int64_t S = n_sites(m);
  for (int64_t site = 0; site < S; ++site) {
    int64_t idx[ORC_MAXD], nb[ORC_MAXD];
    site_to_idx(m, site, idx);
    for (int i = 0; i < m->d; ++i) {
      double v[5];
      for (int o = -2; o <= 2; ++o) {
        memcpy(nb, idx, sizeof(nb));
        nb[i] = ((idx[i] + o) % m->n[i] + m->n[i]) % m->n[i];
        v[o + 2] = phi[idx_to_site(m, nb)];
      }
      grad[(int64_t)i * S + site] = (-v[4] + 8.0 * v[3] - 8.0 * v[1] + v[0]) / (12.0 * m->dx);
    }
  }
}

/* Boundary value of the unknown population k at node `site` for step n -> n+1; R: the source at the
 * node (the constant R, or the per-site field of the step). */
static double boundary_value(const orc_model *m, const orc_wave *w, int64_t n, int64_t site, int k,
                             const double *fstar, double R) {
  const int d = m->d;
  const int64_t S = n_sites(m);
  const double dt = m->dt, c = m->dx / m->dt;
  double x[ORC_MAXD], ck[ORC_MAXD];
  orc_node_coord(m, site, x);
  for (int i = 0; i < d; ++i) ck[i] = c * m->e[k * d + i];
  const double wk = m->omega[k];
  if (m->bc == 1) {
    /* Eq. (bun1) at the boundary node x_b = x, new time t + dt. */
    const double t1 = (double)(n + 1) * dt;
    const double phi = orc_dir_deriv(m, w, x, t1, ck, 0, 0);
    if (m->bc_order == 1) return wk * phi;
    const double feq = wk * phi;
    const double c_grad = wk * orc_dir_deriv(m, w, x, t1, ck, 1, 0);  /* c_k . grad f^eq */
    const double f_t = wk * orc_dir_deriv(m, w, x, t1, ck, 0, 1);     /* d_t f^eq */
    double val = feq - 0.5 * dt * c_grad - 0.5 * dt * f_t + 0.5 * dt * wk * R;
    if (m->bc_order == 3) return val;
    const double c_grad_tt = wk * orc_dir_deriv(m, w, x, t1, ck, 1, 2);   /* c . grad d_t^2 f^eq */
    const double cc_hess_t = wk * orc_dir_deriv(m, w, x, t1, ck, 2, 1);   /* c^2 : grad^2 d_t f^eq */
    const double f_ttt = wk * orc_dir_deriv(m, w, x, t1, ck, 0, 3);       /* d_t^3 f^eq */
    const double ccc_grad3 = wk * orc_dir_deriv(m, w, x, t1, ck, 3, 0);   /* c^3 : grad^3 f^eq */
    val += dt * dt * dt / 8.0 * c_grad_tt + dt * dt * dt / 8.0 * cc_hess_t + dt * dt * dt / 24.0 * f_ttt +
           dt * dt * dt / 24.0 * ccc_grad3;
    return val;
  }
  /* Eq. (bun2): f_k(x_f, t+dt) = -f*_kbar(x_f, t) + [scheme terms at x_b = x_f - c_k dt/2, time t]. */
  const int kb = opposite(m, k);
  const double t = (double)n * dt;
  double xb[ORC_MAXD];
  for (int i = 0; i < d; ++i) xb[i] = x[i] - 0.5 * dt * ck[i];
  const double wsum = wk + m->omega[kb];  /* f^eq_k + f^eq_kbar = (omega_k + omega_kbar) phi */
  const double wdif = wk - m->omega[kb];  /* f^eq_k - f^eq_kbar = (omega_k - omega_kbar) phi */
  double B = wsum * orc_dir_deriv(m, w, xb, t, ck, 0, 0);
  if (m->bc_order >= 2)
    B += 0.5 * dt * wsum * orc_dir_deriv(m, w, xb, t, ck, 0, 1) + 0.5 * dt * (wk * R + m->omega[kb] * R);
  if (m->bc_order >= 3)
    B += -dt * dt / 8.0 * wsum * orc_dir_deriv(m, w, xb, t, ck, 2, 0) -
         dt * dt / 4.0 * wdif * orc_dir_deriv(m, w, xb, t, ck, 1, 1);
  if (m->bc_order >= 4)
    B += -dt * dt * dt / 8.0 * wdif * orc_dir_deriv(m, w, xb, t, ck, 1, 2) -
         dt * dt * dt / 16.0 * wsum * orc_dir_deriv(m, w, xb, t, ck, 2, 1) -
         dt * dt * dt / 24.0 * wsum * orc_dir_deriv(m, w, xb, t, ck, 0, 3);
  return -fstar[(int64_t)kb * S + site] + B;
}

/* One step t_n -> t_{n+1} of Eq. (BGK-LB-Evolution):
 *   collide at every node: f*_k = f_k - s (f_k - omega_k phi) + dt omega_k R(x), phi = sum_k f_k;
 *   push f*_k(x) to x + e_k (periodic wrap, or dropped when it leaves a Dirichlet box);
 *   Dirichlet: every population whose source x - e_k lies outside the box is set by Eq. (bun1)/(bun2). */
void orc_step(const orc_model *m, const orc_wave *w, int64_t n, const double *Rfield,
              const double *f, double *fstar, double *fnew) {
  const int d = m->d, Q = m->Q;
  const int64_t S = n_sites(m);
#pragma omp parallel for schedule(static)
  for (int64_t site = 0; site < S; ++site) {
    double phi = 0.0;
    for (int k = 0; k < Q; ++k) phi += f[(int64_t)k * S + site];
    const double R = Rfield ? Rfield[site] : m->R;
    for (int k = 0; k < Q; ++k) {
      const double fk = f[(int64_t)k * S + site];
      const double feq = m->omega[k] * phi;
      fstar[(int64_t)k * S + site] = fk - m->s * (fk - feq) + m->dt * m->omega[k] * R;
    }
  }
  if (m->bc != 0) {
    for (int64_t i = 0; i < (int64_t)Q * S; ++i) fnew[i] = NAN;
  }
#pragma omp parallel for schedule(static)
  for (int64_t site = 0; site < S; ++site) {
    int64_t idx[ORC_MAXD], dst[ORC_MAXD];
    site_to_idx(m, site, idx);
    for (int k = 0; k < Q; ++k) {
      int inside = 1;
      for (int i = 0; i < d; ++i) {
        dst[i] = idx[i] + m->e[k * d + i];
        if (m->bc == 0) dst[i] = (dst[i] + m->n[i]) % m->n[i];
        else if (dst[i] < 0 || dst[i] >= m->n[i]) inside = 0;
      }
      if (inside) fnew[(int64_t)k * S + idx_to_site(m, dst)] = fstar[(int64_t)k * S + site];
    }
  }
  if (m->bc == 0) return;
#pragma omp parallel for schedule(static)
  for (int64_t site = 0; site < S; ++site) {
    int64_t idx[ORC_MAXD];
    site_to_idx(m, site, idx);
    for (int k = 0; k < Q; ++k) {
      int outside = 0;
      for (int i = 0; i < d; ++i) {
        const int64_t src = idx[i] - m->e[k * d + i];
        if (src < 0 || src >= m->n[i]) outside = 1;
      }
      if (outside) fnew[(int64_t)k * S + site] = boundary_value(m, w, n, site, k, fstar, Rfield ? Rfield[site] : m->R);
    }
  }
}

/* Zeroth moment, Eq. (0-1-meq): phi = sum_k f_k. */
void orc_phi(const orc_model *m, const double *f, double *phi) {
  const int64_t S = n_sites(m);
  for (int64_t site = 0; site < S; ++site) {
    double acc = 0.0;
    for (int k = 0; k < m->Q; ++k) acc += f[(int64_t)k * S + site];
    phi[site] = acc;
  }
}

double orc_entropy(const orc_model *m, const double *f) {
  const int64_t S = n_sites(m);
  double acc = 0.0;
  for (int64_t site = 0; site < S; ++site)
    for (int k = 0; k < m->Q; ++k) {
      const double fk = f[(int64_t)k * S + site];
      acc += fk * fk / (2.0 * m->omega[k]);
    }
  return acc;
}

/* ------------------------------------------------------------------ adjoint */

static int opposite_link(const orc_model *m, int k) {
  for (int j = 0; j < m->Q; ++j) {
    int same = 1;
    for (int i = 0; i < m->d; ++i)
      if (m->e[j * m->d + i] != -m->e[k * m->d + i]) same = 0;
    if (same) return j;
  }
  return -1;
}

/* Transpose of orc_step. With lam_next = dL/df(t_{n+1}) (pre-collision populations):
 *   mu_k(x) = dL/df*_k(x). The push sends f*_k(x) to x + e_k, so mu_k(x) = lam_next_k(x + e_k)
 *             when that node exists (periodic: always, with wrap). On a Dirichlet box a link that
 *             leaves the box feeds nothing in the full-way scheme (Eq. (bun1): the unknown
 *             population at the far side is set from the boundary data alone), while in the
 *             half-way scheme the unknown population of the opposite link at the same node is
 *             f_kbar(x) = -f*_k(x) + B (Eq. (bun2)), so mu_k(x) = -lam_next_kbar(x).
 *   gR(x)  += dt sum_k omega_k mu_k(x)                  (f*_k carries dt omega_k R(x))
 *   lam_j(x) = (1 - s) mu_j(x) + s sum_k omega_k mu_k(x)   (collision f* = f - s(f - omega phi))
 * The boundary data enter the step additively, so they do not appear in the transpose. */
void orc_adjoint_step(const orc_model *m, const double *lam_next, double *lam, double *gR) {
  const int d = m->d, Q = m->Q;
  const int64_t S = n_sites(m);
#pragma omp parallel for schedule(static)
  for (int64_t site = 0; site < S; ++site) {
    int64_t idx[ORC_MAXD], dst[ORC_MAXD];
    double mu[ORC_MAXQ];
    site_to_idx(m, site, idx);
    double wmu = 0.0;
    for (int k = 0; k < Q; ++k) {
      int inside = 1;
      for (int i = 0; i < d; ++i) {
        dst[i] = idx[i] + m->e[k * d + i];
        if (m->bc == 0) dst[i] = (dst[i] + m->n[i]) % m->n[i];
        else if (dst[i] < 0 || dst[i] >= m->n[i]) inside = 0;
      }
      if (inside) mu[k] = lam_next[(int64_t)k * S + idx_to_site(m, dst)];
      else if (m->bc == 2) mu[k] = -lam_next[(int64_t)opposite_link(m, k) * S + site];
      else mu[k] = 0.0;
      wmu += m->omega[k] * mu[k];
    }
    if (gR) gR[site] += m->dt * wmu;
    for (int j = 0; j < Q; ++j) lam[(int64_t)j * S + site] = (1.0 - m->s) * mu[j] + m->s * wmu;
  }
}

/* Transpose of orc_init (and of orc_fd_grad when grad_is_fd). lam0 = dL/df(0).
 *   gphi0(x) = sum_k omega_k lam0_k(x) [+ D^T applied to the gradient part]
 *   ggrad_i(x) = (dt/2) sum_k omega_k (u_i - c e_ki) lam0_k(x)   (order 3 only). */
void orc_adjoint_init(const orc_model *m, int order, int grad_is_fd, const double *lam0,
                      double *gphi0, double *ggrad) {
  const int d = m->d, Q = m->Q;
  const int64_t S = n_sites(m);
  const double c = m->dx / m->dt;
  if (S <= 0 || d <= 0) return;
  double *G = NULL;
  if (order == 3) G = (double *)calloc((size_t)d * (size_t)S, sizeof(double));
  for (int64_t site = 0; site < S; ++site) {
    double acc = 0.0;
    for (int k = 0; k < Q; ++k) acc += m->omega[k] * lam0[(int64_t)k * S + site];
    gphi0[site] = acc;
    if (order == 3) {
      for (int i = 0; i < d; ++i) {
        double gi = 0.0;
        for (int k = 0; k < Q; ++k)
          gi += m->omega[k] * (m->u[i] - c * m->e[k * d + i]) * lam0[(int64_t)k * S + site];
        G[(int64_t)i * S + site] = 0.5 * m->dt * gi;
      }
    }
  }
  if (order == 3) {
    if (!grad_is_fd) {
      memcpy(ggrad, G, sizeof(double) * (size_t)d * S);
    } else {
      /* Transpose of the periodic fourth-order central difference of orc_fd_grad:
       * (D_i^T v)(x) = (-v(x-2e_i) + 8 v(x-e_i) - 8 v(x+e_i) + v(x+2e_i)) / (12 dx). */
      for (int64_t site = 0; site < S; ++site) {
        int64_t idx[ORC_MAXD], nb[ORC_MAXD];
        site_to_idx(m, site, idx);
        for (int i = 0; i < d; ++i) {
          double v[5];
          for (int o = -2; o <= 2; ++o) {
            memcpy(nb, idx, sizeof(nb));
            nb[i] = ((idx[i] + o) % m->n[i] + m->n[i]) % m->n[i];
            v[o + 2] = G[(int64_t)i * S + idx_to_site(m, nb)];
          }
          gphi0[site] += (-v[0] + 8.0 * v[1] - 8.0 * v[3] + v[4]) / (12.0 * m->dx);
        }
      }
    }
  }
  free(G);
}

// lhe_bnode.cuh -- evaluation of the unknown populations at a node of a Dirichlet box (Eq. (bun1),
// Eq. (bun2)), shared by the boundary-node kernel and the FP64 interior-row kernel.
#pragma once

#include "lhe_internal.h"

namespace lhe {

// Per-node data of the boundary schemes: (sin, cos) of every mode's phase xi_m at the node and
// step time, the linear part of h and (full-way) h itself.
template <int D>
struct BNode {
  double sn[kMaxModes], cs[kMaxModes];
  double lin0, H;
};

template <int D, int KIND>
__device__ __forceinline__ void bnode_prepare(const BoundaryArgs &a, const int (&x)[D], BNode<D> &nd) {
  double X[D];
#pragma unroll
  for (int i = 0; i < D; ++i) X[i] = a.x0[i] + (double)x[i] * a.dx;
  const double te = a.t_eval;
  const int M = a.nmodes;
  // (cos, sin) of xi_m = theta_m - kappa_m . u t + sum_i kappa_mi X_i: the step's time factor times the
  // node's per-axis factors (tabulated on the host), with no transcendental call per node.
  for (int m = 0; m < M; ++m) {
    double c = a.ph_c[m], s = a.ph_s[m];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double *t = a.axis + 2 * ((size_t)m * a.axis_len + a.axis_off[i] + x[i]);
      const double ca = __ldg(t), sa = __ldg(t + 1);
      const double c2 = fma(c, ca, -s * sa);
      s = fma(c, sa, s * ca);
      c = c2;
    }
    nd.sn[m] = s;
    nd.cs[m] = c;
  }
  double lin0 = a.b + a.R * te;  // linear part of h at (x, t_eval)
#pragma unroll
  for (int i = 0; i < D; ++i) lin0 = fma(a.gl[i], X[i] - a.u[i] * te, lin0);
  nd.lin0 = lin0;
  double H = lin0;  // h(x, t_eval) (full-way)
  if (KIND == 1)
    for (int m = 0; m < M; ++m) H = fma(a.a[m], nd.sn[m], H);
  nd.H = H;
}

// The part of unknown population k that depends on the boundary data only: the population itself
// (full-way) or B_k of f_k = B_k - f*_kbar(x) (half-way).
template <int D, int KIND>
__device__ __forceinline__ double bnode_data(const BoundaryArgs &a, const BNode<D> &nd, int k) {
  constexpr int Q = Lattice<D>::Q;
  const int M = a.nmodes;
  const double *coef = a.table;                                 // [m][k][2]
  const double *kconst = a.table + (size_t)2 * a.nmodes * Q;    // [k][2]
  if (KIND == 1) {
    double acc = nd.H - __ldg(kconst + 2 * k);
    for (int m = 0; m < M; ++m) acc = fma(-__ldg(coef + 2 * (m * Q + k)), nd.cs[m], acc);
    return a.omega[k] * acc;
  }
  double acc = fma(__ldg(kconst + 2 * k), nd.lin0, __ldg(kconst + 2 * k + 1));
  for (int m = 0; m < M; ++m) {
    acc = fma(__ldg(coef + 2 * (m * Q + k)), nd.sn[m], acc);
    acc = fma(__ldg(coef + 2 * (m * Q + k) + 1), nd.cs[m], acc);
  }
  return acc;
}

// Half-way: f*_kbar(x, t) at the node itself, subtracted from B_k (Eq. (bun2)).
template <int D, bool DEV>
__device__ __forceinline__ double bnode_fkb(const BoundaryArgs &a, int k, int32_t site) {
  constexpr Lattice<D> L{};
  const int kb = L.opp[k];
  const int64_t S = a.g.S;
  return DEV ? fma(a.omega[kb], df_value(a.phi_src[site]), (double)static_cast<const float *>(a.src)[kb * S + site])
             : static_cast<const double *>(a.src)[kb * S + site];
}

// Pre-collision population k at `site` whose source lies outside the box.
template <int D, int KIND, bool DEV>
__device__ __forceinline__ double bnode_unknown(const BoundaryArgs &a, const BNode<D> &nd, int k, int32_t site) {
  const double acc = bnode_data<D, KIND>(a, nd, k);
  return KIND == 1 ? acc : acc - bnode_fkb<D, DEV>(a, k, site);
}

// Index j (0 .. 2D-2) of link k among the links whose first component is e_k,1 = sgn (the unknown
// links of a node on an x_1 face), in the order of k; -1 if e_k,1 != sgn.
template <int D>
__host__ __device__ constexpr int xface_link(int k, int sgn) {
  constexpr Lattice<D> L{};
  int j = 0;
  for (int q = 0; q < k; ++q)
    if (L.e[q][0] == sgn) ++j;
  return L.e[k][0] == sgn ? j : -1;
}

}  // namespace lhe

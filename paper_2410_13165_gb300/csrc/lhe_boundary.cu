// lhe_boundary.cu -- boundary-node kernels of a Dirichlet box (Sec. 3.2).
//
// One thread per boundary node x (some coordinate at 0 or n_i - 1). For every population k:
//   source x - e_k inside the box : f_k(x, t+dt) = f*_k(x - e_k, t)      (streamed)
//   source outside (unknown)      : full-way, Eq. (bun1), data at (x, t+dt):
//       order 1: omega_k phi
//       order 3: omega_k [phi - (dt/2)(c_k.grad phi + d_t phi)] + (dt/2) omega_k R
//       order 4: order 3 + omega_k (dt^3/24) (c_k.grad + d_t)^3 phi
//     (the four dt^3 terms of Eq. (bun1) are the binomial expansion of (c_k.grad + d_t)^3 / 24)
//                                   half-way, Eq. (bun2) at x_b = x - c_k dt/2, time t:
//       f_k(x, t+dt) = -f*_kbar(x, t) + (w_k + w_kbar)[phi + (dt/2)(phi_t + R) - (dt^2/8) c c:grad^2 phi
//                       - (dt^3/16) c c:grad^2 phi_t - (dt^3/24) phi_ttt]
//                       - (w_k - w_kbar)[(dt^2/4) c.grad phi_t + (dt^3/8) c.grad phi_tt]   (terms by order)
// then the node collides like the bulk. The Dirichlet data phi = h come from the exact-solution
// family h = b + R t + g.(x - u t) + sum_m a_m sin(xi_m), xi_m = kappa_m.(x - u t) + theta_m. Along
// c_k every derivative d_t^q (c_k.grad)^p of a mode is a_m A^p B^q sin^(p+q)(xi_m), A = kappa_m.c_k,
// B = -kappa_m.u, so each scheme is, per unknown k, a node value plus sum_m (U_mk sin xi_m + V_mk
// cos xi_m) with coefficients that depend only on (m, k), the order and the lattice; the host
// tabulates them (the half-way shift to x_b is the rotation of (sin, cos) by (dx/2) kappa_m.e_k,
// folded into U and V). Full-way: f_k = omega_k [h(x) - C_k - sum_m T_mk cos xi_m]; half-way:
// f_k = wp_k lin(x) + K_k + sum_m (U_mk sin xi_m + V_mk cos xi_m) - f*_kbar(x), lin = linear part of h.
// The phase xi_m at a node is assembled from tabulated per-axis factors; boundary nodes come
// grouped by face signature so that a warp shares one set of unknown populations. The per-node
// evaluation (lhe_bnode.cuh) is shared with the FP64 interior kernel of Dirichlet boxes, which treats
// the nodes of the two x_1 faces (whose other coordinates are interior) in the lanes of their rows.
#include "lhe_bnode.cuh"

namespace lhe {

template <int D, int KIND, bool DEV>
__global__ void __launch_bounds__(128) k_boundary(const BoundaryArgs a) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nsites) return;
  const int32_t site = a.sites[t];
  const int64_t S = a.g.S;
  int x[D];
  {
    uint32_t r = (uint32_t)site;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (i == D - 1) {
        x[i] = (int)r;
      } else {
        const uint32_t q = a.g.dv[i].div(r);
        x[i] = (int)(r - q * (uint32_t)a.g.n[i]);
        r = q;
      }
    }
  }
  BNode<D> nd;
  const bool jets = a.rec != nullptr;  // data from jet records (else from the exact-solution family)
  if (!jets) bnode_prepare<D, KIND>(a, x, nd);
  const double *__restrict__ rec = jets ? a.rec + a.roff[t] : nullptr;
  int ju = 0;

  const double *__restrict__ fsrc = static_cast<const double *>(a.src);
  const float *__restrict__ gsrc = static_cast<const float *>(a.src);
  double v[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    bool inside = true;
    int32_t o = site;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (L.e[k][i] != 0) {
        const int xs = x[i] - L.e[k][i];
        if (xs < 0 || xs >= a.g.n[i]) inside = false;
        o -= L.e[k][i] * a.g.stride[i];
      }
    }
    if (inside) {
      v[k] = DEV ? fma(a.omega[k], df_value(a.phi_src[o]), (double)gsrc[k * S + o]) : fsrc[k * S + o];
      continue;
    }
    if (jets) {
      const double b = a.rec_scale * __ldg(rec + ju++);
      v[k] = KIND == 1 ? b : b - bnode_fkb<D, DEV>(a, k, site);
    } else {
      v[k] = bnode_unknown<D, KIND, DEV>(a, nd, k, site);
    }
  }
  // collision, as in the bulk: phi = sum_k f_k (the split moment sum of the row kernels), f*_k = (1 - s) f_k +
  // omega_k (s phi + dt R)
  const double phi = split_moment_sum<Q, kBoxFixedTerms<Q>>(v);
  const double psi = fma(a.s, phi, a.dt * (a.Rfield ? __ldg(a.Rfield + site) : a.R));
  const bool s2 = a.s == 2.0;
  if (DEV) {
    float *gdst = static_cast<float *>(a.dst);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const double fs = s2 ? fma(a.omega[k], psi, -v[k]) : fma(a.omega[k], psi, a.oms * v[k]);
      gdst[k * S + site] = (float)fma(-a.omega[k], phi, fs);
    }
    a.phi_dst[site] = df_split(phi);
  } else {
    double *fdst = static_cast<double *>(a.dst);
#pragma unroll
    for (int k = 0; k < Q; ++k)
      fdst[k * S + site] = s2 ? fma(a.omega[k], psi, -v[k]) : fma(a.omega[k], psi, a.oms * v[k]);
  }
}

// Records of the boundary data from jets of phi (lhe_lbm_set_boundary_jet): for every boundary node
// and unknown link k (in the order of k), with c = c e_k,
//   full-way, jet at the node and t + dt (Eq. (bun1)):
//     order 1: omega_k phi;  order 3: omega_k [phi - (dt/2)(c.grad + d_t) phi] + (dt/2) omega_k R;
//     order 4: order 3 + omega_k (dt^3/24) (c.grad + d_t)^3 phi
//   half-way, jet at x_b = x - c dt/2 and t (Eq. (bun2) without -f*_kbar), w+- = omega_k +- omega_kbar:
//     w+ phi + [P >= 2] w+ (dt/2)(phi_t + R) - [P >= 3] (w+ (dt^2/8) cc:grad^2 phi + w- (dt^2/4) c.grad phi_t)
//     - [P >= 4] (w+ (dt^3/16) cc:grad^2 phi_t + w+ (dt^3/24) phi_ttt + w- (dt^3/8) c.grad phi_tt).
// R is the source at the node (the per-site field of the step, when there is one).
// A jet holds every derivative of order <= 3 in (t, x_1..x_d); J.i3[a*36 + b*6 + e] and
// J.i2[a*6 + b] give the position of the derivative in the variables a, b(, e) (0: t, i: x_i), in
// any order.
struct JetIndex {
  int16_t i3[216];
  int16_t i2[36];
};

template <int D, int KIND>
__global__ void __launch_bounds__(128) k_jet_records(const BoundaryArgs a, const double *__restrict__ jet,
                                                     const JetIndex J, double *__restrict__ rec) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  constexpr int JL = (D + 4) * (D + 3) * (D + 2) / 6;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nsites) return;
  const int32_t site = a.sites[t];
  int x[D];
  {
    uint32_t r = (uint32_t)site;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (i == D - 1) {
        x[i] = (int)r;
      } else {
        const uint32_t q = a.g.dv[i].div(r);
        x[i] = (int)(r - q * (uint32_t)a.g.n[i]);
        r = q;
      }
    }
  }
  const int32_t r0 = a.roff[t];
  const int P = a.order;
  const double dt = a.dt;
  const double R = a.Rfield ? a.Rfield[site] : a.R;  // the source at the node
  int ju = 0;
  for (int k = 0; k < Q; ++k) {
    bool inside = true;
    for (int i = 0; i < D; ++i) {
      const int xs = x[i] - L.e[k][i];
      if (xs < 0 || xs >= a.g.n[i]) inside = false;
    }
    if (inside) continue;
    const double *j = jet + (size_t)(KIND == 1 ? t : r0 + ju) * JL;
    double w[D + 1];  // weights of the variables in (d_t + c.grad): 1 for t, c_i for x_i
    w[0] = 1.0;
    for (int i = 0; i < D; ++i) w[i + 1] = a.c * L.e[k][i];
    double val;
    if (KIND == 1) {
      const double wk = a.omega[k];
      val = wk * j[0];
      if (P >= 3) {
        double d1 = 0.0;
        for (int v = 0; v <= D; ++v) d1 += w[v] * j[1 + v];
        val = wk * (j[0] - 0.5 * dt * d1) + 0.5 * dt * wk * R;
      }
      if (P >= 4) {
        double d3 = 0.0;
        for (int p0 = 0; p0 <= D; ++p0)
          for (int p1 = 0; p1 <= D; ++p1)
            for (int p2 = 0; p2 <= D; ++p2) {
              const double ww = w[p0] * w[p1] * w[p2];
              if (ww != 0.0) d3 += ww * j[J.i3[p0 * 36 + p1 * 6 + p2]];
            }
        val += wk * dt * dt * dt / 24.0 * d3;
      }
    } else {
      const int kb = L.opp[k];
      const double wp = a.omega[k] + a.omega[kb], wm = a.omega[k] - a.omega[kb];
      val = wp * j[0];
      if (P >= 2) val += 0.5 * dt * wp * (j[1] + R);
      if (P >= 3) {
        double cch = 0.0, cgt = 0.0;
        for (int p0 = 1; p0 <= D; ++p0) {
          cgt += w[p0] * j[J.i2[p0 * 6]];
          for (int p1 = 1; p1 <= D; ++p1) cch += w[p0] * w[p1] * j[J.i2[p0 * 6 + p1]];
        }
        val -= dt * dt / 8.0 * wp * cch + dt * dt / 4.0 * wm * cgt;
      }
      if (P >= 4) {
        double ccht = 0.0, cgtt = 0.0;
        for (int p0 = 1; p0 <= D; ++p0) {
          cgtt += w[p0] * j[J.i3[p0 * 36]];
          for (int p1 = 1; p1 <= D; ++p1) ccht += w[p0] * w[p1] * j[J.i3[p0 * 36 + p1 * 6]];
        }
        val -= dt * dt * dt / 16.0 * wp * ccht + dt * dt * dt / 24.0 * wp * j[J.i3[0]] + dt * dt * dt / 8.0 * wm * cgtt;
      }
    }
    rec[a.rmap ? a.rmap[r0 + ju] : r0 + ju] = val;  // node-major, or in the order of the dense entries
    ++ju;
  }
}

template <int D>
static cudaError_t jet_records_d(int kind, const BoundaryArgs &a, const double *jet, const JetIndex &J, double *rec,
                                 cudaStream_t st) {
  if (a.nsites <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((a.nsites + 127) / 128);
  if (kind == 1) k_jet_records<D, 1><<<blocks, 128, 0, st>>>(a, jet, J, rec);
  else k_jet_records<D, 2><<<blocks, 128, 0, st>>>(a, jet, J, rec);
  return cudaGetLastError();
}

cudaError_t launch_jet_records(int d, int kind, const BoundaryArgs &a, const double *jet, const int16_t *jidx,
                               double *rec, cudaStream_t st) {
  JetIndex J;
  for (int i = 0; i < 216; ++i) J.i3[i] = jidx[i];
  for (int i = 0; i < 36; ++i) J.i2[i] = jidx[216 + i];
  switch (d) {
    case 1: return jet_records_d<1>(kind, a, jet, J, rec, st);
    case 2: return jet_records_d<2>(kind, a, jet, J, rec, st);
    case 3: return jet_records_d<3>(kind, a, jet, J, rec, st);
    case 4: return jet_records_d<4>(kind, a, jet, J, rec, st);
    case 5: return jet_records_d<5>(kind, a, jet, J, rec, st);
    default: return cudaErrorInvalidValue;
  }
}

// Cotangent of the jets of one Dirichlet step (lhe_lbm_adjoint_jet_grad): the transpose of
// k_jet_records. a.src holds the adjoint state rho_k(x) = omega_k dL/df_k(x) of the pre-collision
// populations that the step produced, so the cotangent of an unknown population's value is
// rho_k / omega_k (the R terms and the half-way -f*_kbar do not depend on the jets). Full-way: one row
// per boundary node, summed over its unknown links (omega_k times the cotangent is rho_k); half-way:
// one row per unknown population, w+ and w- times rho_k / omega_k. Each thread owns the rows of its
// node and zeroes them first. FP32 deviations (DEV): rho_k = omega_k W + eps_k.
template <int D, int KIND, bool DEV>
__global__ void __launch_bounds__(128) k_jet_grad(const BoundaryArgs a, const JetIndex J, double *__restrict__ out) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  constexpr int JL = (D + 4) * (D + 3) * (D + 2) / 6;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nsites) return;
  const int32_t site = a.sites[t];
  int x[D];
  {
    uint32_t r = (uint32_t)site;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (i == D - 1) {
        x[i] = (int)r;
      } else {
        const uint32_t q = a.g.dv[i].div(r);
        x[i] = (int)(r - q * (uint32_t)a.g.n[i]);
        r = q;
      }
    }
  }
  const double *__restrict__ rho = static_cast<const double *>(a.src);
  const int64_t S = a.g.S;
  const int32_t r0 = a.roff[t];
  const int P = a.order;
  const double dt = a.dt;
  if (KIND == 1)
    for (int e = 0; e < JL; ++e) out[t * JL + e] = 0.0;
  int ju = 0;
  for (int k = 0; k < Q; ++k) {
    bool inside = true;
    for (int i = 0; i < D; ++i) {
      const int xs = x[i] - L.e[k][i];
      if (xs < 0 || xs >= a.g.n[i]) inside = false;
    }
    if (inside) continue;
    double *g = out + (size_t)(KIND == 1 ? t : r0 + ju) * JL;
    double w[D + 1];  // weights of the variables in (d_t + c.grad): 1 for t, c_i for x_i
    w[0] = 1.0;
    for (int i = 0; i < D; ++i) w[i + 1] = a.c * L.e[k][i];
    const double rk = DEV ? fma(a.omega[k], df_value(a.phi_src[site]), (double)static_cast<const float *>(a.src)[k * S + site])
                          : rho[k * S + site];
    if (KIND == 1) {
      g[0] += rk;
      if (P >= 3)
        for (int v = 0; v <= D; ++v) g[1 + v] -= 0.5 * dt * w[v] * rk;
      if (P >= 4) {
        const double c3 = dt * dt * dt / 24.0 * rk;
        for (int p0 = 0; p0 <= D; ++p0)
          for (int p1 = 0; p1 <= D; ++p1)
            for (int p2 = 0; p2 <= D; ++p2) {
              const double ww = w[p0] * w[p1] * w[p2];
              if (ww != 0.0) g[J.i3[p0 * 36 + p1 * 6 + p2]] += ww * c3;
            }
      }
    } else {
      for (int e = 0; e < JL; ++e) g[e] = 0.0;
      const int kb = L.opp[k];
      const double lam = rk / a.omega[k];
      const double wp = (a.omega[k] + a.omega[kb]) * lam, wm = (a.omega[k] - a.omega[kb]) * lam;
      g[0] = wp;
      if (P >= 2) g[1] += 0.5 * dt * wp;
      if (P >= 3)
        for (int p0 = 1; p0 <= D; ++p0) {
          g[J.i2[p0 * 6]] -= dt * dt / 4.0 * wm * w[p0];
          for (int p1 = 1; p1 <= D; ++p1) g[J.i2[p0 * 6 + p1]] -= dt * dt / 8.0 * wp * w[p0] * w[p1];
        }
      if (P >= 4) {
        g[J.i3[0]] -= dt * dt * dt / 24.0 * wp;
        for (int p0 = 1; p0 <= D; ++p0) {
          g[J.i3[p0 * 36]] -= dt * dt * dt / 8.0 * wm * w[p0];
          for (int p1 = 1; p1 <= D; ++p1) g[J.i3[p0 * 36 + p1 * 6]] -= dt * dt * dt / 16.0 * wp * w[p0] * w[p1];
        }
      }
    }
    ++ju;
  }
}

template <int D>
static cudaError_t jet_grad_d(int kind, bool dev, const BoundaryArgs &a, const JetIndex &J, double *out,
                              cudaStream_t st) {
  if (a.nsites <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((a.nsites + 127) / 128);
  if (kind == 1) {
    if (dev) k_jet_grad<D, 1, true><<<blocks, 128, 0, st>>>(a, J, out);
    else k_jet_grad<D, 1, false><<<blocks, 128, 0, st>>>(a, J, out);
  } else {
    if (dev) k_jet_grad<D, 2, true><<<blocks, 128, 0, st>>>(a, J, out);
    else k_jet_grad<D, 2, false><<<blocks, 128, 0, st>>>(a, J, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_jet_grad(int d, int kind, bool dev, const BoundaryArgs &a, const int16_t *jidx, double *out,
                            cudaStream_t st) {
  JetIndex J;
  for (int i = 0; i < 216; ++i) J.i3[i] = jidx[i];
  for (int i = 0; i < 36; ++i) J.i2[i] = jidx[216 + i];
  switch (d) {
    case 1: return jet_grad_d<1>(kind, dev, a, J, out, st);
    case 2: return jet_grad_d<2>(kind, dev, a, J, out, st);
    case 3: return jet_grad_d<3>(kind, dev, a, J, out, st);
    case 4: return jet_grad_d<4>(kind, dev, a, J, out, st);
    case 5: return jet_grad_d<5>(kind, dev, a, J, out, st);
    default: return cudaErrorInvalidValue;
  }
}

// Adjoint of a Dirichlet step at the boundary nodes (FP64), in the weighted variable
// rho_k(x) = omega_k dL/df_k(x) of the pre-collision populations (the interior nodes use the bulk
// adjoint kernel). Transposing the pull: mu_j(x) = omega_j dL/df*_j(x) = rho_j(x + e_j) where
// x + e_j is a node of the box. Where it is not, the post-collision population leaves the box: in
// the full-way scheme it feeds nothing (Eq. (bun1) sets the unknown population at the far side
// from the boundary data alone), in the half-way scheme it is the -f*_j(x) of the unknown
// f_jbar(x) = -f*_j(x) + B (Eq. (bun2)), so mu_j(x) = -(omega_j / omega_jbar) rho_jbar(x). Then
// rho_k <- (1 - s) mu_k + s omega_k sum_j mu_j, as in the bulk. FP32 deviations (DEV): the adjoint state
// is rho_k = omega_k W + eps_k (W a double-float pair, eps in FP32), formed in FP64 here, and the result
// is stored as the forward boundary kernel stores a state: W' = sum_j mu_j, eps'_k = rho'_k - omega_k W'.
template <int D, int KIND, bool DEV>
__global__ void __launch_bounds__(128) k_adj_boundary(const BoundaryArgs a) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nsites) return;
  const int32_t site = a.sites[t];
  const int64_t S = a.g.S;
  int x[D];
  {
    uint32_t r = (uint32_t)site;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (i == D - 1) {
        x[i] = (int)r;
      } else {
        const uint32_t q = a.g.dv[i].div(r);
        x[i] = (int)(r - q * (uint32_t)a.g.n[i]);
        r = q;
      }
    }
  }
  const double *__restrict__ src = static_cast<const double *>(a.src);
  const float *__restrict__ esrc = static_cast<const float *>(a.src);
  // the adjoint state rho_j at node o
  auto rho = [&](int j, int32_t o) {
    return DEV ? fma(a.omega[j], df_value(a.phi_src[o]), (double)esrc[j * S + o]) : src[j * S + o];
  };
  double mu[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    bool inside = true;
    int32_t o = site;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (L.e[k][i] != 0) {
        const int xs = x[i] + L.e[k][i];
        if (xs < 0 || xs >= a.g.n[i]) inside = false;
        o += L.e[k][i] * a.g.stride[i];
      }
    }
    if (inside) mu[k] = rho(k, o);
    else mu[k] = KIND == 2 ? -a.wratio[k] * rho(L.opp[k], site) : 0.0;
  }
  if (DEV) {
    const double M = fixed_moment_sum<Q, 0>(mu);
    const double psi = a.s * M;
    float *edst = static_cast<float *>(a.dst);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const double r = a.s == 2.0 ? fma(a.omega[k], psi, -mu[k]) : fma(a.omega[k], psi, a.oms * mu[k]);
      edst[k * S + site] = (float)fma(-a.omega[k], M, r);
    }
    a.phi_dst[site] = df_split(M);
    return;
  }
  double *__restrict__ dst = static_cast<double *>(a.dst);
  if (a.s == 2.0) {
    const double psi = fixed_moment_sum<Q, 1>(mu);  // 2 sum_j mu_j
#pragma unroll
    for (int k = 0; k < Q; ++k) dst[k * S + site] = fma(a.omega[k], psi, -mu[k]);
  } else {
    const double psi = a.s * fixed_moment_sum<Q, 0>(mu);
#pragma unroll
    for (int k = 0; k < Q; ++k) dst[k * S + site] = fma(a.omega[k], psi, a.oms * mu[k]);
  }
}

template <int D>
static cudaError_t adj_boundary_d(int kind, bool dev, const BoundaryArgs &a, cudaStream_t st) {
  if (a.nsites <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((a.nsites + 127) / 128);
  if (kind == 1) {
    if (dev) k_adj_boundary<D, 1, true><<<blocks, 128, 0, st>>>(a);
    else k_adj_boundary<D, 1, false><<<blocks, 128, 0, st>>>(a);
  } else {
    if (dev) k_adj_boundary<D, 2, true><<<blocks, 128, 0, st>>>(a);
    else k_adj_boundary<D, 2, false><<<blocks, 128, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_boundary(int d, int kind, bool dev, const BoundaryArgs &a, cudaStream_t st) {
  switch (d) {
    case 1: return adj_boundary_d<1>(kind, dev, a, st);
    case 2: return adj_boundary_d<2>(kind, dev, a, st);
    case 3: return adj_boundary_d<3>(kind, dev, a, st);
    case 4: return adj_boundary_d<4>(kind, dev, a, st);
    case 5: return adj_boundary_d<5>(kind, dev, a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int D>
static cudaError_t boundary_d(int kind, bool dev, const BoundaryArgs &a, cudaStream_t st) {
  if (a.nsites <= 0) return cudaSuccess;
  const int threads = 128;
  const unsigned blocks = (unsigned)((a.nsites + threads - 1) / threads);
  if (kind == 1) {
    if (dev) k_boundary<D, 1, true><<<blocks, threads, 0, st>>>(a);
    else k_boundary<D, 1, false><<<blocks, threads, 0, st>>>(a);
  } else {
    if (dev) k_boundary<D, 2, true><<<blocks, threads, 0, st>>>(a);
    else k_boundary<D, 2, false><<<blocks, threads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_boundary(int d, int kind, bool dev, const BoundaryArgs &a, cudaStream_t st) {
  switch (d) {
    case 1: return boundary_d<1>(kind, dev, a, st);
    case 2: return boundary_d<2>(kind, dev, a, st);
    case 3: return boundary_d<3>(kind, dev, a, st);
    case 4: return boundary_d<4>(kind, dev, a, st);
    case 5: return boundary_d<5>(kind, dev, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lhe

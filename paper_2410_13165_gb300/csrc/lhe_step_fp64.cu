// lhe_step_fp64.cu -- fused pull-stream + BGK collision on DdQ(2d^2+1), FP64 populations.
//
// Forward (Eq. (BGK-LB-Evolution)), stored state = post-collision populations f*:
//   f_k(x)  = f*_k(x - e_k)                      (pull; periodic wrap or interior of a Dirichlet box)
//   phi(x)  = sum_k f_k(x)                       (Eq. (0-1-meq))
//   f*_k(x) = (1 - s) f_k + omega_k (s phi + dt R(x))      (s = 2: omega_k (2 phi + dt R) - f_k)
// For s != 2 the stored array may hold the scaled populations G = K f* (K = (1 - s)^-j), updated by
// G*_k = G_k + omega_k (sig sum_k G_k + K' dt R) with sig ~ s/(1 - s) and K' = K/(1 - s): the factor
// (1 - s) of the pulled populations is carried by K instead of one multiply per population.
// Adjoint (transpose of the step, in the weighted variable zeta_k = omega_k nu_k):
//   mu_k(x) = zeta_k(x + e_k)                    (reverse pull)
//   w(x)    = sum_k mu_k(x),  gR(x) += dt w(x)
//   zeta_k  = (1 - s) mu_k + omega_k s w
// Both are one thread per site, x_1 fastest, SoA population arrays pop[k*S + site].
#include "lhe_bnode.cuh"
#include "lhe_internal.h"
#include "lhe_sites.cuh"

namespace lhe {

// Template collision forms: s = 2, general s (mu, sig, rho from StepArgs), scaled representation.
constexpr int kModeGeneral = 0, kModeS2 = 1, kModeScaled = 2;

template <int D, bool ADJ, bool INTERIOR, int MODE>
__global__ void __launch_bounds__(LHE_STEP_THREADS) k_step_fp64(const StepArgs a) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  pdl_trigger();
  pdl_wait();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nwork) return;
  int x[D];
  const int32_t site = decode_site<D, INTERIOR>(a.g, t, x);
  if (skip_site<D, INTERIOR>(a.g, x)) return;
  int32_t om[D], op[D];
  axis_offsets<D, INTERIOR>(a.g, x, om, op);
  const double *__restrict__ src = static_cast<const double *>(a.src);
  double *__restrict__ dst = static_cast<double *>(a.dst);
  const int64_t S = a.g.S;
  double f[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) f[k] = __ldg(src + k * S + source_site<D, ADJ>(L, k, site, om, op));
  double psi;
  if (ADJ) {
    if (MODE == kModeS2) {
      psi = fixed_moment_sum<Q, 1>(f);  // 2 w
      if (a.gR) a.gR[site] = fma(a.half_dt, psi, a.gR[site]);
    } else {
      const double w = fixed_moment_sum<Q, 0>(f);
      psi = a.sig * w;
      if (a.gR) a.gR[site] = fma(a.gsc, w, a.gR[site]);
    }
  } else if (MODE == kModeS2) {
    psi = fixed_moment_sum<Q, 1>(f) + (a.Rfield ? a.dt * __ldg(a.Rfield + site) : a.dtR);
  } else {
    psi = fma(a.sig, fixed_moment_sum<Q, 0>(f), a.Rfield ? a.rho_dt * __ldg(a.Rfield + site) : a.rho_dtR);
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const double out = MODE == kModeS2      ? fma(a.omega[k], psi, -f[k])
                       : MODE == kModeScaled ? fma(a.omega[k], psi, f[k])
                                             : fma(a.omega[k], psi, a.mu * f[k]);
    st_stream(dst + k * S + site, out);
  }
}

// Boundary data of the x_1-face nodes of a Dirichlet box (those whose other coordinates are
// interior), for k_step_box: for interior row r (x_2..x_D interior) and side h (0: x_1 = 0, 1:
// x_1 = n_1 - 1), the 2D - 1 values bnode_data of the unknown links (e_k,1 = +1 on the low side,
// -1 on the high side) at xb[(2 r + h)(2D - 1) + j]. They do not depend on the state.
template <int D, int KIND>
__global__ void __launch_bounds__(128) k_xface_data(const BoundaryArgs b, double *__restrict__ xb, int64_t nrows) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  constexpr int J = 2 * D - 1;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 2 * nrows) return;
  const int h = (int)(t & 1);
  uint32_t r = (uint32_t)(t >> 1);
  int x[D];
  x[0] = h ? b.g.n[0] - 1 : 0;
#pragma unroll
  for (int i = 1; i < D; ++i) {
    if (i == D - 1) {
      x[i] = (int)r + 1;
    } else {
      const uint32_t q = b.g.dvi[i].div(r);
      x[i] = (int)(r - q * (uint32_t)(b.g.n[i] - 2)) + 1;
      r = q;
    }
  }
  BNode<D> nd;
  bnode_prepare<D, KIND>(b, x, nd);
  const int sgn = h ? -1 : 1;
#pragma unroll
  for (int k = 0; k < Q; ++k)
    if (L.e[k][0] == sgn) xb[t * J + xface_link<D>(k, sgn)] = bnode_data<D, KIND>(b, nd, k);
}

// Forward step of a Dirichlet box (FP64, constant R), whole x-rows through the interior: the interior
// lanes are those of k_step_fp64; the two face lanes of a row (x_1 = 0 or n_1 - 1, the other
// coordinates interior) take each unknown population (e_k,1 = +1 on the low face, -1 on the high face)
// from the data of k_xface_data (half-way: minus f*_kbar at the node) in the same load instruction as
// the row's pulled populations, and collide with the row. The values are those of the boundary-node
// kernel, bit for bit. Keeping these nodes in their rows avoids the boundary kernel's accesses strided
// by n_1, which wasted most of a sector per population read and forced a fill of every partially
// written sector.
template <int D, int MODE, int KIND>
__global__ void __launch_bounds__(LHE_STEP_THREADS) k_step_box(const StepArgs a, const double *__restrict__ xb) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  constexpr int J = 2 * D - 1;
  pdl_trigger();
  pdl_wait();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nwork) return;
  int x[D];
  const int32_t site = decode_site<D, true>(a.g, t, x);
  // +1: low x_1 face (links with e_k,1 = +1 unknown); -1: high face; 0: interior node
  const int face = x[0] == 0 ? 1 : (x[0] == a.g.n[0] - 1 ? -1 : 0);
  int32_t om[D], op[D];
  axis_offsets<D, true>(a.g, x, om, op);
  const double *__restrict__ src = static_cast<const double *>(a.src);
  double *__restrict__ dst = static_cast<double *>(a.dst);
  const int64_t S = a.g.S;
  const double *rec = xb + (2 * (int64_t)a.g.dv[0].div((uint32_t)t) + (face < 0 ? 1 : 0)) * J;  // face node's data
  double f[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const bool unknown = face != 0 && L.e[k][0] == face;
    const int j = L.e[k][0] == 1 ? xface_link<D>(k, 1) : xface_link<D>(k, -1);
    f[k] = __ldg(unknown ? rec + j : src + k * S + source_site<D, false>(L, k, site, om, op));
    if (KIND == 2 && L.e[k][0] != 0 && unknown) f[k] = f[k] - __ldg(src + L.opp[k] * S + site);
  }
  const double psi = MODE == kModeS2 ? fixed_moment_sum<Q, 1>(f) + a.dtR
                                     : fma(a.sig, fixed_moment_sum<Q, 0>(f), a.rho_dtR);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const double out = MODE == kModeS2 ? fma(a.omega[k], psi, -f[k]) : fma(a.omega[k], psi, a.mu * f[k]);
    st_stream(dst + k * S + site, out);
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_macro_fp64(const StepArgs a, double *__restrict__ phi) {
  constexpr int Q = Lattice<D>::Q;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.g.S) return;
  const double *__restrict__ src = static_cast<const double *>(a.src);
  double f[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) f[k] = src[k * a.g.S + t];
  const double dtR = a.Rfield ? a.dt * a.Rfield[t] : a.dtR;
  // phi(t_n) = sum_k f*_k(x, t_n) - dt R(x): the collision keeps sum_k f_k and adds dt R. pscale
  // converts a scaled state back to f* (1 otherwise, exact).
  phi[t] = fma(fixed_moment_sum<Q, 0>(f), a.pscale, -dtR);
}

template <int D, bool ADJ, bool INTERIOR>
static cudaError_t launch_step_fp64_t(const StepArgs &a, cudaStream_t st) {
  if (a.nwork <= 0) return cudaSuccess;
  const int threads = LHE_STEP_THREADS;
  const unsigned blocks = (unsigned)((a.nwork + threads - 1) / threads);
  const bool pdl = a.pdl != 0;
  if (a.s == 2.0) return launch_kernel(k_step_fp64<D, ADJ, INTERIOR, kModeS2>, blocks, threads, 0, st, pdl, a);
  if (a.collide == kCollideScaled)
    return launch_kernel(k_step_fp64<D, ADJ, INTERIOR, kModeScaled>, blocks, threads, 0, st, pdl, a);
  return launch_kernel(k_step_fp64<D, ADJ, INTERIOR, kModeGeneral>, blocks, threads, 0, st, pdl, a);
}

template <int D>
static cudaError_t step_fp64_d(bool adjoint, bool interior, const StepArgs &a, cudaStream_t st) {
  if (adjoint) return interior ? launch_step_fp64_t<D, true, true>(a, st) : launch_step_fp64_t<D, true, false>(a, st);
  return interior ? launch_step_fp64_t<D, false, true>(a, st) : launch_step_fp64_t<D, false, false>(a, st);
}

cudaError_t launch_step_fp64(int d, bool adjoint, bool interior, const StepArgs &a, cudaStream_t st) {
  switch (d) {
    case 1: return step_fp64_d<1>(adjoint, interior, a, st);
    case 2: return step_fp64_d<2>(adjoint, interior, a, st);
    case 3: return step_fp64_d<3>(adjoint, interior, a, st);
    case 4: return step_fp64_d<4>(adjoint, interior, a, st);
    case 5: return step_fp64_d<5>(adjoint, interior, a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int D>
static cudaError_t step_box_d(int kind, const StepArgs &a, const BoundaryArgs &b, double *xb, int64_t nrows,
                              cudaStream_t st) {
  if (a.nwork <= 0) return cudaSuccess;
  const unsigned dblocks = (unsigned)((2 * nrows + 127) / 128);
  cudaError_t e;
  if (kind == 1) k_xface_data<D, 1><<<dblocks, 128, 0, st>>>(b, xb, nrows);
  else k_xface_data<D, 2><<<dblocks, 128, 0, st>>>(b, xb, nrows);
  if ((e = cudaGetLastError())) return e;
  const int threads = LHE_STEP_THREADS;
  const unsigned blocks = (unsigned)((a.nwork + threads - 1) / threads);
  const double *cxb = xb;
  if (a.s == 2.0)
    return kind == 1 ? launch_kernel(k_step_box<D, kModeS2, 1>, blocks, threads, 0, st, false, a, cxb)
                     : launch_kernel(k_step_box<D, kModeS2, 2>, blocks, threads, 0, st, false, a, cxb);
  return kind == 1 ? launch_kernel(k_step_box<D, kModeGeneral, 1>, blocks, threads, 0, st, false, a, cxb)
                   : launch_kernel(k_step_box<D, kModeGeneral, 2>, blocks, threads, 0, st, false, a, cxb);
}

cudaError_t launch_step_box_fp64(int d, int kind, const StepArgs &a, const BoundaryArgs &b, double *xb, int64_t nrows,
                                 cudaStream_t st) {
  switch (d) {
    case 1: return step_box_d<1>(kind, a, b, xb, nrows, st);
    case 2: return step_box_d<2>(kind, a, b, xb, nrows, st);
    case 3: return step_box_d<3>(kind, a, b, xb, nrows, st);
    case 4: return step_box_d<4>(kind, a, b, xb, nrows, st);
    case 5: return step_box_d<5>(kind, a, b, xb, nrows, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_macro_fp64(int d, const StepArgs &a, double *phi_out, cudaStream_t st) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((a.g.S + threads - 1) / threads);
  switch (d) {
    case 1: k_macro_fp64<1><<<blocks, threads, 0, st>>>(a, phi_out); break;
    case 2: k_macro_fp64<2><<<blocks, threads, 0, st>>>(a, phi_out); break;
    case 3: k_macro_fp64<3><<<blocks, threads, 0, st>>>(a, phi_out); break;
    case 4: k_macro_fp64<4><<<blocks, threads, 0, st>>>(a, phi_out); break;
    case 5: k_macro_fp64<5><<<blocks, threads, 0, st>>>(a, phi_out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lhe

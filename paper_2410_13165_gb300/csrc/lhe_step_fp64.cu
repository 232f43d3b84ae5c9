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
  if (kPeriodicFixedTerms<Q> < Q) {  // the split sum (lhe_device.cuh); 2 w and 2 phi are exact doublings
    const double w = split_moment_sum<Q, kPeriodicFixedTerms<Q>>(f);
    if (ADJ) {
      psi = MODE == kModeS2 ? 2.0 * w : a.sig * w;
      if (a.gR) a.gR[site] = MODE == kModeS2 ? fma(a.half_dt, psi, a.gR[site]) : fma(a.gsc, w, a.gR[site]);
    } else if (MODE == kModeS2) {
      psi = fma(2.0, w, a.Rfield ? a.dt * __ldg(a.Rfield + site) : a.dtR);
    } else {
      psi = fma(a.sig, w, a.Rfield ? a.rho_dt * __ldg(a.Rfield + site) : a.rho_dtR);
    }
  } else if (ADJ) {
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

// lhe_provider.cu -- Dirichlet data and source of the manufactured solution
// phi*(x, t) = A exp(-lambda t) prod_i sin(kappa_i x_i + theta_i) of Eq. (HE) with its own source
// R(x, t) = d_t phi* + u . grad phi* (lhe_lbm_set_boundary_sine_product).
//
// The solution separates: phi*(x, t) = exp(-lambda t) P(x), and so do all its derivatives and R. The
// records of the unknown populations (Eq. (bun1) with data and R at t_{n+1}, Eq. (bun2) with data and
// R at t_n) are therefore exp(-lambda t_data) times those at unit factor. These kernels form, once,
// the jets of P at the boundary points and the field R0(x) = R(x, t) exp(lambda t); the records follow
// from them through k_jet_records, and each step only scales them (the boundary kernel's record scale)
// and the source field (k_scale_field).
#include <algorithm>

#include "lhe_internal.h"

namespace lhe {

// d^q/dz^q sin(z) for q = 0..3 (mod 4): sin, cos, -sin, -cos
__device__ __forceinline__ double dsin(double s, double c, int q) {
  switch (q & 3) {
    case 0: return s;
    case 1: return c;
    case 2: return -s;
    default: return -c;
  }
}

// Jets of P(x) = A prod_i sin(kappa_i x_i + theta_i) with the time factor exp(-lambda t) at t = 0:
// the entry of tuple (v_1 <= .. <= v_q) is (-lambda)^{#t} A prod_i kappa_i^{a_i} sin^{(a_i)}(kappa_i x_i
// + theta_i), a_i the number of v = i. tup[e * 6 + v] holds the count of variable v (0: t) in entry e.
template <int D>
__global__ void __launch_bounds__(128) k_sp_jets(const SineProductArgs a, const double *__restrict__ pts, int64_t P,
                                                  const int8_t *__restrict__ tup, double *__restrict__ jet) {
  constexpr int JL = (D + 4) * (D + 3) * (D + 2) / 6;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  double s[D], c[D];
#pragma unroll
  for (int i = 0; i < D; ++i) sincos(fma(a.kappa[i], pts[p * D + i], a.theta[i]), &s[i], &c[i]);
  for (int e = 0; e < JL; ++e) {
    double v = a.A;
    for (int q = 0; q < tup[e * 6]; ++q) v *= -a.lambda;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const int ai = tup[e * 6 + 1 + i];
      double f = dsin(s[i], c[i], ai);
      for (int q = 0; q < ai; ++q) f *= a.kappa[i];
      v *= f;
    }
    jet[p * JL + e] = v;
  }
}

// R0(x) = -lambda P(x) + sum_i u_i d_i P(x) at every node x_i = x0_i + j_i dx.
template <int D>
__global__ void __launch_bounds__(128) k_sp_source(const SineProductArgs a, const Geom g, double *__restrict__ R0) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.S) return;
  double s[D], c[D];
  uint32_t r = (uint32_t)t;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    int j;
    if (i == D - 1) {
      j = (int)r;
    } else {
      const uint32_t q = g.dv[i].div(r);
      j = (int)(r - q * (uint32_t)g.n[i]);
      r = q;
    }
    sincos(fma(a.kappa[i], fma((double)j, a.dx, a.x0[i]), a.theta[i]), &s[i], &c[i]);
  }
  double prod = a.A, adv = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double di = a.A * a.kappa[i] * c[i];  // d_i P
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (j != i) di *= s[j];
    adv = fma(a.u[i], di, adv);
    prod *= s[i];
  }
  R0[t] = fma(-a.lambda, prod, adv);
}

__global__ void __launch_bounds__(256) k_scale_field(const double *__restrict__ in, double scale, int64_t n,
                                                     double *__restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += stride) out[t] = scale * in[t];
}

cudaError_t launch_sp_jets(int d, const SineProductArgs &a, const double *pts, int64_t P, const int8_t *tup,
                           double *jet, cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((P + 127) / 128);
  switch (d) {
    case 1: k_sp_jets<1><<<blocks, 128, 0, st>>>(a, pts, P, tup, jet); break;
    case 2: k_sp_jets<2><<<blocks, 128, 0, st>>>(a, pts, P, tup, jet); break;
    case 3: k_sp_jets<3><<<blocks, 128, 0, st>>>(a, pts, P, tup, jet); break;
    case 4: k_sp_jets<4><<<blocks, 128, 0, st>>>(a, pts, P, tup, jet); break;
    case 5: k_sp_jets<5><<<blocks, 128, 0, st>>>(a, pts, P, tup, jet); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sp_source(const SineProductArgs &a, const Geom &g, double *R0, cudaStream_t st) {
  if (g.S <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((g.S + 127) / 128);
  switch (g.d) {
    case 1: k_sp_source<1><<<blocks, 128, 0, st>>>(a, g, R0); break;
    case 2: k_sp_source<2><<<blocks, 128, 0, st>>>(a, g, R0); break;
    case 3: k_sp_source<3><<<blocks, 128, 0, st>>>(a, g, R0); break;
    case 4: k_sp_source<4><<<blocks, 128, 0, st>>>(a, g, R0); break;
    case 5: k_sp_source<5><<<blocks, 128, 0, st>>>(a, g, R0); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_scale_field(const double *in, double scale, int64_t n, double *out, int sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)std::min<int64_t>(want, (int64_t)std::max(sms, 1) * 8);
  k_scale_field<<<blocks, 256, 0, st>>>(in, scale, n, out);
  return cudaGetLastError();
}

}  // namespace lhe

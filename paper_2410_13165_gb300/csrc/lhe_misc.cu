// lhe_misc.cu -- initialisation, finite-difference gradient, diagnostics reduction and the
// adjoint seed / gradient kernels.
#include "lhe_diag.cuh"
#include "lhe_internal.h"
#include "lhe_sites.cuh"

namespace lhe {

// ------------------------------------------------------------------------------ initialisation
// Eq. (ini-simp): f_k(x,0) = omega_k [phi0 + (dt/2)(u - c e_k) . grad phi0] (order 3) or
// omega_k phi0 (order 1); the stored state is post-collision. With A = phi0 + dt R(x) and the first
// moment of the correction vanishing (sum_k omega_k (u - c e_k) = 0), the collision
// f*_k = (1 - s) f_k + omega_k (s phi0 + dt R) is
//   f*_k = omega_k A + (1 - s)(dt/2) omega_k [u . grad phi0 - c e_k . grad phi0]     (FP64)
//   g*_k = f*_k - omega_k phi0 = omega_k dt R + (same correction),  phi = phi0      (FP32_DEV)
// three FP64 operations per population (c1_k = (1 - s)(dt/2) omega_k, c2_k = c c1_k on the host).
template <int D, bool DEV>
__global__ void __launch_bounds__(256) k_init(const InitArgs a) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  const int64_t site = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t S = a.g.S;
  if (site >= S) return;
  const double phi0 = a.phi0[site];
  const double dtR = a.Rfield ? a.dt * a.Rfield[site] : a.dtR;
  double gr[D];
  double ug = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    gr[i] = (a.order == 3) ? a.grad[i * S + site] : 0.0;
    ug = fma(a.u[i], gr[i], ug);
  }
  const double A = DEV ? dtR : phi0 + dtR;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    double eg = 0.0;  // e_k . grad phi0 (components are 0 or +-1)
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (L.e[k][i] == 1) eg += gr[i];
      if (L.e[k][i] == -1) eg -= gr[i];
    }
    const double v = fma(a.omega[k], A, fma(-a.c2[k], eg, a.c1[k] * ug));
    if (DEV) static_cast<float *>(a.dst)[k * S + site] = (float)v;
    else static_cast<double *>(a.dst)[k * S + site] = v;
  }
  if (DEV) a.phi_dst[site] = df_split(phi0);
}

template <int D>
static cudaError_t init_d(bool dev, const InitArgs &a, cudaStream_t st) {
  const unsigned blocks = (unsigned)((a.g.S + 255) / 256);
  if (dev) k_init<D, true><<<blocks, 256, 0, st>>>(a);
  else k_init<D, false><<<blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_init(int d, bool dev, const InitArgs &a, cudaStream_t st) {
  switch (d) {
    case 1: return init_d<1>(dev, a, st);
    case 2: return init_d<2>(dev, a, st);
    case 3: return init_d<3>(dev, a, st);
    case 4: return init_d<4>(dev, a, st);
    case 5: return init_d<5>(dev, a, st);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------------------------ FD gradient
// Periodic fourth-order central difference: d_i phi ~ (-phi(x+2e_i) + 8 phi(x+e_i) - 8 phi(x-e_i)
// + phi(x-2e_i)) / (12 dx). TRANSPOSE adds D_i^T G_i = -D_i G_i to `out` instead.
__device__ __forceinline__ int32_t wrap_off(int xi, int o, int32_t n, int32_t stride) {
  int y = xi + o;
  if (y < 0) y += n;
  if (y >= n) y -= n;
  return (y - xi) * stride;
}

template <int D, bool TRANSPOSE>
__global__ void __launch_bounds__(256) k_fd(const Geom g, double inv12dx, const double *__restrict__ in,
                                            double *__restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.S) return;
  int x[D];
  const int32_t site = decode_site<D, false>(g, t, x);
  double acc = TRANSPOSE ? out[site] : 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const double *v = in + (TRANSPOSE ? (int64_t)i * g.S : 0);
    const double p2 = v[site + wrap_off(x[i], 2, g.n[i], g.stride[i])];
    const double p1 = v[site + wrap_off(x[i], 1, g.n[i], g.stride[i])];
    const double m1 = v[site + wrap_off(x[i], -1, g.n[i], g.stride[i])];
    const double m2 = v[site + wrap_off(x[i], -2, g.n[i], g.stride[i])];
    const double di = (-p2 + 8.0 * p1 - 8.0 * m1 + m2) * inv12dx;
    if (TRANSPOSE) acc -= di;
    else out[(int64_t)i * g.S + site] = di;
  }
  if (TRANSPOSE) out[site] = acc;
}

template <int D, bool T>
static cudaError_t fd_d(const Geom &g, double dx, const double *in, double *out, cudaStream_t st) {
  const unsigned blocks = (unsigned)((g.S + 255) / 256);
  k_fd<D, T><<<blocks, 256, 0, st>>>(g, 1.0 / (12.0 * dx), in, out);
  return cudaGetLastError();
}

template <bool T>
static cudaError_t fd_dispatch(int d, const Geom &g, double dx, const double *in, double *out, cudaStream_t st) {
  switch (d) {
    case 1: return fd_d<1, T>(g, dx, in, out, st);
    case 2: return fd_d<2, T>(g, dx, in, out, st);
    case 3: return fd_d<3, T>(g, dx, in, out, st);
    case 4: return fd_d<4, T>(g, dx, in, out, st);
    case 5: return fd_d<5, T>(g, dx, in, out, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fd_grad(int d, const Geom &g, double dx, const double *phi, double *grad, cudaStream_t st) {
  return fd_dispatch<false>(d, g, dx, phi, grad, st);
}

cudaError_t launch_fd_grad_transpose_add(int d, const Geom &g, double dx, const double *G, double *out,
                                         cudaStream_t st) {
  return fd_dispatch<true>(d, g, dx, G, out, st);
}

// ------------------------------------------------------------------------------ diagnostics
// Per site: phi (from the post-collision state: sum_k f*_k - dt R), the pre-collision populations
// recovered from f* = (1-s) f + omega (s phi + dt R) (s != 1; for s = 1 the post-collision values
// are used), the kinetic entropy sum_k f_k^2 / (2 omega_k) (Eq. (skfk)), |phi| and non-finite
// values. Block partials go to a scratch array; a second single-block pass adds them in a fixed
// order, so the result does not depend on scheduling.
template <int D, bool DEV>
__global__ void __launch_bounds__(256) k_reduce_partials(const ReduceArgs a) {
  constexpr int Q = Lattice<D>::Q;
  __shared__ double sh[8 * 4];
  const int64_t S = a.g.S;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const bool recover = a.s != 1.0;
  for (int64_t site = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; site < S;
       site += (int64_t)gridDim.x * blockDim.x) {
    const double dtR = a.Rfield ? a.dt * a.Rfield[site] : a.dtR;
    if (DEV) {
      double phi, ent = 0.0, bad = 0.0;
      const float *g = static_cast<const float *>(a.pop);
      phi = df_value(a.phi[site]);
      if (!isfinite(phi)) bad += 1.0;
      ent = 0.5 * phi * phi;  // sum_k f_k^2/(2 w_k) = phi^2/2 + sum_k g_k^2/(2 w_k) since sum_k g_k = 0
      for (int k = 0; k < Q; ++k) {
        const double gs = (double)g[k * S + site];
        if (!isfinite(gs)) bad += 1.0;
        const double gk = recover ? (gs - a.omega[k] * dtR) / (1.0 - a.s) : gs;
        ent += gk * gk / (2.0 * a.omega[k]);
      }
      v[0] += phi;
      v[1] += ent;
      v[2] = fmax(v[2], fabs(phi));
      v[3] += bad;
    } else {
      diag_site_fp64(static_cast<const double *>(a.pop), S, site, Q, a.omega, a.s, recover, dtR, v);
    }
  }
  block_reduce4(v, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) a.partials[blockIdx.x * 4 + j] = v[j];
}

__global__ void __launch_bounds__(256) k_reduce_final(const double *__restrict__ partials, int nblocks,
                                                      double *__restrict__ out) {
  __shared__ double sh[8 * 4];
  reduce_partials_final(partials, nblocks, out, sh);
}

template <int D>
static cudaError_t reduce_d(bool dev, const ReduceArgs &a, int nblocks, cudaStream_t st) {
  if (dev) k_reduce_partials<D, true><<<nblocks, 256, 0, st>>>(a);
  else k_reduce_partials<D, false><<<nblocks, 256, 0, st>>>(a);
  k_reduce_final<<<1, 256, 0, st>>>(a.partials, nblocks, a.out);
  return cudaGetLastError();
}

cudaError_t launch_reduce(int d, bool dev, const ReduceArgs &a, int nblocks, cudaStream_t st) {
  switch (d) {
    case 1: return reduce_d<1>(dev, a, nblocks, st);
    case 2: return reduce_d<2>(dev, a, nblocks, st);
    case 3: return reduce_d<3>(dev, a, nblocks, st);
    case 4: return reduce_d<4>(dev, a, nblocks, st);
    case 5: return reduce_d<5>(dev, a, nblocks, st);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------------------------ adjoint
// Seed: nu_k(x, T) = dL/dphi_T(x) for every k (phi_T = sum_k f*_k - dt R), stored as
// zeta_k = omega_k nu_k (FP64) or as W = dL/dphi_T, eps_k = 0 (FP32_DEV); dL/dR := 0.
template <int D, bool DEV>
__global__ void __launch_bounds__(256) k_adj_seed(const Geom g, const StepArgs w, const double *__restrict__ seed,
                                                  void *adj, float2 *adjW, double *gR) {
  constexpr int Q = Lattice<D>::Q;
  const int64_t site = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (site >= g.S) return;
  const double s0 = seed[site];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    if (DEV) static_cast<float *>(adj)[k * g.S + site] = 0.0f;
    else static_cast<double *>(adj)[k * g.S + site] = w.omega[k] * s0;
  }
  if (DEV) adjW[site] = df_split(s0);
  gR[site] = 0.0;
}

template <int D>
static cudaError_t seed_d(bool dev, const Geom &g, const StepArgs &w, const double *seed, void *adj, float2 *adjW,
                          double *gR, cudaStream_t st) {
  const unsigned blocks = (unsigned)((g.S + 255) / 256);
  if (dev) k_adj_seed<D, true><<<blocks, 256, 0, st>>>(g, w, seed, adj, adjW, gR);
  else k_adj_seed<D, false><<<blocks, 256, 0, st>>>(g, w, seed, adj, adjW, gR);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_seed(int d, bool dev, const Geom &g, const double *omega, const double *seed, void *adj,
                                float2 *adjW, double *gR, cudaStream_t st) {
  StepArgs w{};
  for (int k = 0; k < kMaxQ; ++k) w.omega[k] = omega[k];
  switch (d) {
    case 1: return seed_d<1>(dev, g, w, seed, adj, adjW, gR, st);
    case 2: return seed_d<2>(dev, g, w, seed, adj, adjW, gR, st);
    case 3: return seed_d<3>(dev, g, w, seed, adj, adjW, gR, st);
    case 4: return seed_d<4>(dev, g, w, seed, adj, adjW, gR, st);
    case 5: return seed_d<5>(dev, g, w, seed, adj, adjW, gR, st);
    default: return cudaErrorInvalidValue;
  }
}

// Transpose of the initialisation (with its collision) applied to zeta^0 = omega nu^0,
// nu^0 = dL/df(0):  dL/dphi0 = sum_k zeta_k;  G_i = (dt/2) sum_k (u_i - c e_ki) zeta_k
// (= dL/d(grad phi0)_i for order 3). FP32_DEV: zeta_k = omega_k W + eps_k, where the W part
// cancels in G because sum_k omega_k (u - c e_k) = 0.
template <int D, bool DEV>
__global__ void __launch_bounds__(256) k_adj_grads(const AdjGradArgs a) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  const int64_t site = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t S = a.g.S;
  if (site >= S) return;
  double zsum = DEV ? df_value(a.adjW[site]) : 0.0;
  double G[D];
#pragma unroll
  for (int i = 0; i < D; ++i) G[i] = 0.0;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const double z = DEV ? (double)static_cast<const float *>(a.adj)[k * S + site]
                         : static_cast<const double *>(a.adj)[k * S + site];
    zsum += z;
#pragma unroll
    for (int i = 0; i < D; ++i) G[i] = fma(a.u[i] - a.c * L.e[k][i], z, G[i]);
  }
  a.gphi0[site] = zsum;
  if (a.order == 3 && a.G)
#pragma unroll
    for (int i = 0; i < D; ++i) a.G[i * S + site] = 0.5 * a.dt * G[i];
}

template <int D>
static cudaError_t grads_d(bool dev, const AdjGradArgs &a, cudaStream_t st) {
  const unsigned blocks = (unsigned)((a.g.S + 255) / 256);
  if (dev) k_adj_grads<D, true><<<blocks, 256, 0, st>>>(a);
  else k_adj_grads<D, false><<<blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_grads(int d, bool dev, const AdjGradArgs &a, cudaStream_t st) {
  switch (d) {
    case 1: return grads_d<1>(dev, a, st);
    case 2: return grads_d<2>(dev, a, st);
    case 3: return grads_d<3>(dev, a, st);
    case 4: return grads_d<4>(dev, a, st);
    case 5: return grads_d<5>(dev, a, st);
    default: return cudaErrorInvalidValue;
  }
}

// phi of the FP32-deviation form: double-float pair -> double.
__global__ void __launch_bounds__(256) k_df_to_double(const float2 *__restrict__ src, double *__restrict__ dst, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = df_value(src[i]);
}

cudaError_t launch_df_to_double(const float2 *src, double *dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_df_to_double<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

// In-place multiplication of an FP64 population array by a constant (undoes the scaled
// representation of the state; see lhe_api.cu).
__global__ void __launch_bounds__(256) k_scale_fp64(double *__restrict__ p, int64_t n, double factor) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] *= factor;
}

cudaError_t launch_scale_fp64(double *p, int64_t n, double factor, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_scale_fp64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, n, factor);
  return cudaGetLastError();
}

}  // namespace lhe

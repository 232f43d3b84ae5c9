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
// family h = b + R t + g.(x - u t) + sum_m a_m sin(kappa_m.(x - u t) + theta_m); along c_k every
// derivative d_t^q (c_k.grad)^p of a mode is a_m A^p B^q sin^(p+q)(xi) with A = kappa_m.c_k,
// B = -kappa_m.u. The half-way evaluation point is reached by rotating (sin, cos) of the node's
// phase by alpha = (dx/2) kappa_m.e_k (tabulated on the host).
#include "lhe_internal.h"

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
  double X[D];
#pragma unroll
  for (int i = 0; i < D; ++i) X[i] = a.x0[i] + (double)x[i] * a.dx;
  const double te = a.t_eval;
  const int M = a.nmodes;
  double sn[kMaxModes], cs[kMaxModes];
  for (int m = 0; m < M; ++m) {
    double xi = a.theta[m];
#pragma unroll
    for (int i = 0; i < D; ++i) xi = fma(a.kappa[m * kMaxD + i], X[i] - a.u[i] * te, xi);
    sincos(xi, &sn[m], &cs[m]);
  }
  double lin0 = a.b + a.R * te, gu = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    lin0 = fma(a.gl[i], X[i] - a.u[i] * te, lin0);
    gu = fma(a.gl[i], a.u[i], gu);
  }
  const double *ku = a.table + (size_t)a.nmodes * Q * 3;
  const double dt = a.dt, dt2 = dt * dt, dt3 = dt2 * dt;

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
    double gc = 0.0;  // g . c_k
#pragma unroll
    for (int i = 0; i < D; ++i)
      if (L.e[k][i] != 0) gc += a.gl[i] * (a.c * L.e[k][i]);
    if (KIND == 1) {
      // full-way at the node, time t + dt
      double D00 = lin0, D1 = gc + (a.R - gu), D3 = 0.0;  // D1 = (c.grad + d_t) phi, D3 = (c.grad + d_t)^3 phi
      for (int m = 0; m < M; ++m) {
        const double A = a.table[(m * Q + k) * 3];
        const double AB = A - ku[m];
        D00 = fma(a.a[m], sn[m], D00);
        D1 = fma(a.a[m] * AB, cs[m], D1);
        D3 = fma(-a.a[m] * AB * AB * AB, cs[m], D3);
      }
      double val;
      if (a.order == 1) {
        val = a.omega[k] * D00;
      } else {
        val = a.omega[k] * (D00 - 0.5 * dt * D1) + 0.5 * dt * a.omega[k] * a.R;
        if (a.order >= 4) val = fma(a.omega[k] * dt3 / 24.0, D3, val);
      }
      v[k] = val;
    } else {
      // half-way at x_b = x - e_k dx/2, time t
      const int kb = L.opp[k];
      const double wp = a.omega[k] + a.omega[kb], wm = a.omega[k] - a.omega[kb];
      double D00 = lin0 - 0.5 * dt * gc, D01 = a.R - gu;
      double D20 = 0.0, D11 = 0.0, D12 = 0.0, D21 = 0.0, D03 = 0.0;
      for (int m = 0; m < M; ++m) {
        const double *tb = a.table + (m * Q + k) * 3;
        const double A = tb[0], B = -ku[m];
        const double sb = sn[m] * tb[1] - cs[m] * tb[2];  // sin(xi - alpha)
        const double cb = cs[m] * tb[1] + sn[m] * tb[2];  // cos(xi - alpha)
        const double am = a.a[m];
        D00 = fma(am, sb, D00);
        D01 = fma(am * B, cb, D01);
        D20 = fma(-am * A * A, sb, D20);
        D11 = fma(-am * A * B, sb, D11);
        D12 = fma(-am * A * B * B, cb, D12);
        D21 = fma(-am * A * A * B, cb, D21);
        D03 = fma(-am * B * B * B, cb, D03);
      }
      double Bk = wp * D00;
      if (a.order >= 2) Bk += 0.5 * dt * wp * D01 + 0.5 * dt * wp * a.R;
      if (a.order >= 3) Bk += -dt2 / 8.0 * wp * D20 - dt2 / 4.0 * wm * D11;
      if (a.order >= 4) Bk += -dt3 / 8.0 * wm * D12 - dt3 / 16.0 * wp * D21 - dt3 / 24.0 * wp * D03;
      const double fkb = DEV ? fma(a.omega[kb], df_value(a.phi_src[site]), (double)gsrc[kb * S + site])
                              : fsrc[kb * S + site];
      v[k] = Bk - fkb;
    }
  }
  double phi = 0.0;
#pragma unroll
  for (int k = 0; k < Q; ++k) phi += v[k];
  const double psi = a.s * phi + dt * a.R;
  if (DEV) {
    float *gdst = static_cast<float *>(a.dst);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const double fs = fma(a.omega[k], psi, a.oms * v[k]);
      gdst[k * S + site] = (float)(fs - a.omega[k] * phi);
    }
    a.phi_dst[site] = df_split(phi);
  } else {
    double *fdst = static_cast<double *>(a.dst);
#pragma unroll
    for (int k = 0; k < Q; ++k) fdst[k * S + site] = fma(a.omega[k], psi, a.oms * v[k]);
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

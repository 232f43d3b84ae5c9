// lhe_stability.cu -- stability maps (Sec. 4): for a batch of velocities sigma and a grid of Fourier
// variables xi, the spectral radius of the amplification matrix of one step on a Fourier mode,
// G(xi) = T(xi) ((1 - s) I + s omega 1^T), T = diag(exp(-i e_k . xi)), in population space (Eq. (G)
// is the same matrix in moment space, G_moment = M G M^{-1}). The von Neumann (L2) condition is
// rho(G(xi)) <= 1 for every xi; Proposition 1's microscopic entropy condition is min_k omega_k > 0.
//
// One thread per (sigma, xi): the Q x Q complex matrix is reduced to upper Hessenberg form by
// Householder reflections, then its eigenvalues are found by the shifted QR iteration (Givens
// rotations, Wilkinson shifts, deflation on negligible subdiagonals), all in FP64. The QR route
// is backward stable, so the (Q-1)-fold eigenvalue 1 - s of G(0) comes out to rounding, where the
// roots of the characteristic polynomial would spread by eps^(1/(Q-1)). The radius per sigma is the
// maximum over its xi, reduced with an integer atomic max on the (non-negative) double bits.
#include "lhe_internal.h"

namespace lhe {

namespace {

constexpr double kPi = 3.14159265358979323846;

struct cd {
  double re, im;
};
__device__ __forceinline__ cd mk(double r, double i) { return cd{r, i}; }
__device__ __forceinline__ cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cd operator*(cd a, cd b) { return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
__device__ __forceinline__ cd cj(cd a) { return cd{a.re, -a.im}; }
__device__ __forceinline__ double ab2(cd a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ double ab(cd a) { return hypot(a.re, a.im); }
__device__ __forceinline__ double ab1(cd a) { return fabs(a.re) + fabs(a.im); }
// principal square root
__device__ __forceinline__ cd csqrt_(cd z) {
  const double r = ab(z);
  if (r == 0.0) return cd{0.0, 0.0};
  const double t = sqrt(0.5 * (r + fabs(z.re)));
  if (z.re >= 0.0) return cd{t, z.im / (2.0 * t)};
  return cd{fabs(z.im) / (2.0 * t), z.im >= 0.0 ? t : -t};
}

// Largest eigenvalue modulus of the N x N complex matrix A (destroyed). Returns NaN when the QR
// iteration does not converge within its iteration budget (80 sweeps per eigenvalue) and the
// remaining window is not triangular to 1e-10.
template <int N>
__device__ double spectral_radius(cd (&A)[N][N]) {
  // 1. upper Hessenberg form: for each column k, a reflection I - 2 v v^H / (v^H v) zeroes A[k+2.., k]
  for (int k = 0; k < N - 2; ++k) {
    double tail = 0.0;
    for (int i = k + 2; i < N; ++i) tail += ab2(A[i][k]);
    if (tail == 0.0) continue;
    const cd x0 = A[k + 1][k];
    const double xn = sqrt(ab2(x0) + tail), a0 = ab(x0);
    const cd ph = a0 > 0.0 ? mk(x0.re / a0, x0.im / a0) : mk(1.0, 0.0);
    cd v[N];
    v[k + 1] = x0 + xn * ph;
    for (int i = k + 2; i < N; ++i) v[i] = A[i][k];
    const double vv = ab2(v[k + 1]) + tail;
    for (int j = k; j < N; ++j) {  // A <- H A on rows k+1..N-1
      cd dot = mk(0.0, 0.0);
      for (int i = k + 1; i < N; ++i) dot = dot + cj(v[i]) * A[i][j];
      const cd f = (2.0 / vv) * dot;
      for (int i = k + 1; i < N; ++i) A[i][j] = A[i][j] - v[i] * f;
    }
    for (int i = 0; i < N; ++i) {  // A <- A H on columns k+1..N-1
      cd dot = mk(0.0, 0.0);
      for (int j = k + 1; j < N; ++j) dot = dot + A[i][j] * v[j];
      const cd f = (2.0 / vv) * dot;
      for (int j = k + 1; j < N; ++j) A[i][j] = A[i][j] - f * cj(v[j]);
    }
    for (int i = k + 2; i < N; ++i) A[i][k] = mk(0.0, 0.0);
  }
  // 2. shifted QR on the active window [lo, hi]
  double rho = 0.0;
  int hi = N - 1, iter = 0;
  cd gs[N];
  double gc[N];
  while (hi >= 0) {
    if (hi == 0) {
      rho = fmax(rho, ab(A[0][0]));
      break;
    }
    int lo = hi;
    for (; lo > 0; --lo) {
      const double tst = ab1(A[lo - 1][lo - 1]) + ab1(A[lo][lo]);
      if (ab1(A[lo][lo - 1]) <= 4.440892098500626e-16 * (tst > 0.0 ? tst : 1.0)) {  // 2 ulp
        A[lo][lo - 1] = mk(0.0, 0.0);
        break;
      }
    }
    if (lo == hi) {
      rho = fmax(rho, ab(A[hi][hi]));
      --hi;
      iter = 0;
      continue;
    }
    if (++iter > 80) {
      // budget spent: a window whose subdiagonal is at rounding level is triangular for our purpose
      for (int i = lo + 1; i <= hi; ++i)
        if (ab1(A[i][i - 1]) > 1e-10 * (ab1(A[i - 1][i - 1]) + ab1(A[i][i])))
          return __longlong_as_double(0x7FF8000000000000ll);
      for (int i = lo; i <= hi; ++i) rho = fmax(rho, ab(A[i][i]));
      hi = lo - 1;
      iter = 0;
      continue;
    }
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer to its last entry
    const cd a = A[hi - 1][hi - 1], b = A[hi - 1][hi], c = A[hi][hi - 1], d = A[hi][hi];
    const cd half_tr = 0.5 * (a + d);
    const cd disc = csqrt_(half_tr * half_tr - (a * d - b * c));
    const cd m1 = half_tr + disc, m2 = half_tr - disc;
    cd mu = ab2(m1 - d) < ab2(m2 - d) ? m1 : m2;
    if (iter % 10 == 9) {  // exceptional shift, off the symmetric configurations that stall the iteration
      const double sc = ab1(c) + (hi - 1 > lo ? ab1(A[hi - 1][hi - 2]) : 0.0);
      mu = d + mk(0.75 * sc, 0.45 * sc);
    }
    for (int i = lo; i <= hi; ++i) A[i][i] = A[i][i] - mu;
    for (int k = lo; k < hi; ++k) {  // R = G_{hi-1} ... G_lo (H - mu I)
      const cd x = A[k][k], y = A[k + 1][k];
      double cc;
      cd ss;
      const double ax = ab(x), ay = ab(y);
      if (ay == 0.0) {
        cc = 1.0;
        ss = mk(0.0, 0.0);
      } else if (ax == 0.0) {
        cc = 0.0;
        ss = mk(y.re / ay, -y.im / ay);
      } else {
        const double r = hypot(ax, ay);
        cc = ax / r;
        ss = (1.0 / r) * (mk(x.re / ax, x.im / ax) * cj(y));
      }
      gc[k] = cc;
      gs[k] = ss;
      for (int j = k; j <= hi; ++j) {
        const cd p = A[k][j], q = A[k + 1][j];
        A[k][j] = cc * p + ss * q;
        A[k + 1][j] = cc * q - cj(ss) * p;
      }
    }
    for (int k = lo; k < hi; ++k) {  // R Q: apply each G_k^H from the right
      const double cc = gc[k];
      const cd ss = gs[k];
      const int top = min(k + 2, hi);
      for (int i = lo; i <= top; ++i) {
        const cd p = A[i][k], q = A[i][k + 1];
        A[i][k] = cc * p + cj(ss) * q;
        A[i][k + 1] = cc * q - ss * p;
      }
    }
    for (int i = lo; i <= hi; ++i) A[i][i] = A[i][i] + mu;
  }
  return rho;
}

template <int D>
__global__ void __launch_bounds__(128) k_stability(const double *__restrict__ omega, int64_t npoints, int32_t nxi,
                                                   int64_t nper, double s, unsigned long long *__restrict__ rho_bits) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npoints * nper) return;
  const int64_t p = t / nper;
  int64_t r = t - p * nper;
  double xi[D];
  for (int i = 0; i < D; ++i) {
    const int64_t j = r % nxi;
    r /= nxi;
    xi[i] = -kPi + 2.0 * kPi * (double)j / (double)nxi;
  }
  cd A[Q][Q];
  for (int k = 0; k < Q; ++k) {
    double ph = 0.0;
    for (int i = 0; i < D; ++i) ph -= L.e[k][i] * xi[i];
    double sn, cs;
    sincos(ph, &sn, &cs);
    const cd tk = mk(cs, sn);  // exp(-i e_k . xi)
    const double wk = s * omega[p * Q + k];
    for (int j = 0; j < Q; ++j) A[k][j] = (wk + (j == k ? 1.0 - s : 0.0)) * tk;
  }
  double rho = spectral_radius<Q>(A);
  if (rho != rho) rho = __longlong_as_double(0x7FF0000000000000ll);  // not converged: report +inf
  atomicMax(rho_bits + p, (unsigned long long)__double_as_longlong(rho));
}

}  // namespace

cudaError_t launch_stability(int d, const double *omega_dev, int64_t npoints, int32_t nxi, double s,
                             unsigned long long *rho_bits_dev, cudaStream_t st) {
  int64_t nper = 1;
  for (int i = 0; i < d; ++i) nper *= nxi;
  const int64_t total = npoints * nper;
  if (total <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((total + 127) / 128);
  switch (d) {
    case 1: k_stability<1><<<blocks, 128, 0, st>>>(omega_dev, npoints, nxi, nper, s, rho_bits_dev); break;
    case 2: k_stability<2><<<blocks, 128, 0, st>>>(omega_dev, npoints, nxi, nper, s, rho_bits_dev); break;
    case 3: k_stability<3><<<blocks, 128, 0, st>>>(omega_dev, npoints, nxi, nper, s, rho_bits_dev); break;
    case 4: k_stability<4><<<blocks, 128, 0, st>>>(omega_dev, npoints, nxi, nper, s, rho_bits_dev); break;
    case 5: k_stability<5><<<blocks, 128, 0, st>>>(omega_dev, npoints, nxi, nper, s, rho_bits_dev); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lhe

// lhe_step_box.cu -- forward FP64 step of a Dirichlet box: the interior-row kernel that also treats
// the nodes of the two x_1 faces, and the kernel of their boundary data (Sec. 3.2, Eq. (bun1),
// Eq. (bun2)). The other boundary nodes are treated by lhe_boundary.cu.
#include "lhe_bnode.cuh"
#include "lhe_internal.h"
#include "lhe_sites.cuh"

namespace lhe {

namespace {
constexpr int kModeGeneral = 0, kModeS2 = 1;  // collision forms, as in lhe_step_fp64.cu
}  // namespace

// The family's data for unknown link k at a node, separated in time: P at p[0], A_m at p[(1 + 2m) st],
// B_m at p[(2 + 2m) st]; G = b + g.x, sn/cs = sin/cos(kappa_m . x). Full-way (Eq. (bun1), tabulated):
// omega_k [h - C_k - sum_m T_mk cos xi_m] with h = G + (R - g.u) t + sum_m a_m sin xi_m; half-way
// (Eq. (bun2) without -f*_kbar): wp_k lin + K_k + sum_m (U_mk sin xi_m + V_mk cos xi_m), lin = G + (R - g.u) t;
// xi_m = kappa_m . x + psi_m, so sin xi = sin(k.x) cos psi + cos(k.x) sin psi, cos xi = cos(k.x) cos psi -
// sin(k.x) sin psi.
template <int D, int KIND>
__device__ __forceinline__ void family_sep_coefs(const BoundaryArgs &b, int k, double G, const double *sn,
                                                 const double *cs, double *p, int st) {
  constexpr int Q = Lattice<D>::Q;
  const int M = b.nmodes;
  const double *coef = b.table;                        // [m][k][2]
  const double *kconst = b.table + (size_t)2 * M * Q;  // [k][2]
  if (KIND == 1) {
    const double w = b.omega[k];
    p[0] = w * (G - kconst[2 * k]);
    for (int m = 0; m < M; ++m) {
      const double T = coef[2 * (m * Q + k)];
      p[(1 + 2 * m) * st] = w * (b.a[m] * sn[m] - T * cs[m]);
      p[(2 + 2 * m) * st] = w * (b.a[m] * cs[m] + T * sn[m]);
    }
  } else {
    p[0] = fma(kconst[2 * k], G, kconst[2 * k + 1]);
    for (int m = 0; m < M; ++m) {
      const double U = coef[2 * (m * Q + k)], V = coef[2 * (m * Q + k) + 1];
      p[(1 + 2 * m) * st] = U * sn[m] + V * cs[m];
      p[(2 + 2 * m) * st] = U * cs[m] - V * sn[m];
    }
  }
}

// G = b + g.x and sin/cos(kappa_m . x) at node x.
template <int D>
__device__ __forceinline__ double family_node_phases(const BoundaryArgs &b, const int (&x)[D], double *sn, double *cs) {
  double G = b.b;
#pragma unroll
  for (int i = 0; i < D; ++i) G = fma(b.gl[i], b.x0[i] + (double)x[i] * b.dx, G);
  for (int m = 0; m < b.nmodes; ++m) {
    double ph = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) ph = fma(b.kappa[m * kMaxD + i], b.x0[i] + (double)x[i] * b.dx, ph);
    sincos(ph, &sn[m], &cs[m]);
  }
  return G;
}

// The family's data from separable coefficients p (stride st) at this step: P + lt_k + sum_m (A_m cos psi_m
// + B_m sin psi_m).
__device__ __forceinline__ double family_sep_value(const BoundaryArgs &b, int k, const double *p, int st) {
  double v = __ldg(p) + b.lt[k];
  for (int m = 0; m < b.nmodes; ++m) {
    v = fma(__ldg(p + (1 + 2 * m) * st), b.ph_c[m], v);
    v = fma(__ldg(p + (2 + 2 * m) * st), b.ph_s[m], v);
  }
  return v;
}


// The unknown populations of the x_1-face nodes of a Dirichlet box (those whose other coordinates
// are interior), for k_step_box: for interior row r (x_2..x_D interior) and side h (0: x_1 = 0, 1:
// x_1 = n_1 - 1), the 2D - 1 unknown links (e_k,1 = +1 on the low side, -1 on the high side) at
// xb[(2 r + h)(2D - 1) + j], exactly as the boundary-node kernel forms them: the boundary data (from the
// exact-solution family, or from the records of jets: the x_1-face-only nodes lead the boundary-node
// list, low face then high face, each in row order), and for the half-way scheme minus f*_kbar at the
// node (the state at the start of the step).
template <int D, int KIND>
__global__ void __launch_bounds__(128) k_xface_data(const BoundaryArgs b, double *__restrict__ xb, int64_t nrows,
                                                    const double *__restrict__ xsep) {
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
  int32_t site = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) site += x[i] * b.g.stride[i];
  const int sgn = h ? -1 : 1;
  if (b.rec) {
    const double *rec = b.rec + b.roff[h ? nrows + (t >> 1) : (t >> 1)];
#pragma unroll
    for (int k = 0; k < Q; ++k)
      if (L.e[k][0] == sgn) {
        const int j = xface_link<D>(k, sgn);
        const double v = b.rec_scale * __ldg(rec + j);
        xb[t * J + j] = KIND == 1 ? v : v - bnode_fkb<D, false>(b, k, site);
      }
    return;
  }
  if (xsep) {  // the family's data from separable coefficients (with face rows, see k_xface_sep)
    const int C = 1 + 2 * b.nmodes;
#pragma unroll
    for (int k = 0; k < Q; ++k)
      if (L.e[k][0] == sgn) {
        const int j = xface_link<D>(k, sgn);
        const double v = family_sep_value(b, k, xsep + (t * J + j) * C, 1);
        xb[t * J + j] = KIND == 1 ? v : v - bnode_fkb<D, false>(b, k, site);
      }
    return;
  }
  BNode<D> nd;
  bnode_prepare<D, KIND>(b, x, nd);
#pragma unroll
  for (int k = 0; k < Q; ++k)
    if (L.e[k][0] == sgn) xb[t * J + xface_link<D>(k, sgn)] = bnode_unknown<D, KIND, false>(b, nd, k, site);
}

// Forward step of a Dirichlet box (FP64; constant R or a per-site source), whole x-rows through the interior: the interior
// lanes are those of k_step_fp64; the two face lanes of a row (x_1 = 0 or n_1 - 1, the other
// coordinates interior) take each unknown population (e_k,1 = +1 on the low face, -1 on the high face)
// from k_xface_data (which also subtracts the half-way scheme's f*_kbar) in the same load instruction as
// the row's pulled populations, and collide with the row. The values are those of the boundary-node
// kernel, bit for bit. Keeping these nodes in their rows avoids the boundary kernel's accesses strided
// by n_1, which wasted most of a sector per population read and forced a fill of every partially
// written sector.
template <int D, int MODE>
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
  // a per-site source is loaded ahead of the populations, so that its latency overlaps theirs
  const double Rs = a.Rfield ? __ldg(a.Rfield + site) : 0.0;
  double f[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const bool unknown = face != 0 && L.e[k][0] == face;
    const int j = L.e[k][0] == 1 ? xface_link<D>(k, 1) : xface_link<D>(k, -1);
    f[k] = __ldg(unknown ? rec + j : src + k * S + source_site<D, false>(L, k, site, om, op));
  }
  const double psi = MODE == kModeS2 ? fixed_moment_sum<Q, 1>(f) + (a.Rfield ? a.dt * Rs : a.dtR)
                                     : fma(a.sig, fixed_moment_sum<Q, 0>(f), a.Rfield ? a.rho_dt * Rs : a.rho_dtR);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const double out = MODE == kModeS2 ? fma(a.omega[k], psi, -f[k]) : fma(a.omega[k], psi, a.mu * f[k]);
    st_stream(dst + k * S + site, out);
  }
}

// ------------------------------------------------------------------------------ face rows
// The boundary nodes off the x_1 faces lie on whole rows (fixed x_2..x_d with some of them on a
// face). Their unknown populations at the middle nodes of a row are the same links for the whole row
// (FaceRow::mask), so a row kernel like k_step_box takes them in the same load instructions as the
// pulled ones, reading coalesced data; the two end nodes add the links of their x_1 face. This
// replaces the boundary-node kernel for these nodes in the FP64 forward step. Data:
//   records (jets, the manufactured solution): per node, in the order of k over its unknown links,
//     times rec_scale (the values of the boundary-node kernel, bit for bit);
//   the exact-solution family: separable coefficients formed once per data set (k_face_sep):
//     data_k(x, t) = P + lt_k + sum_m (A_m cos psi_m + B_m sin psi_m), psi_m = theta_m - kappa_m . u t,
//     with P, A_m, B_m per (node, unknown link) and lt_k = q_k t per link and step.
// Half-way: minus f*_kbar at the node (the state at the start of the step), as in k_boundary.
// Layout of the coefficients, C = 1 + 2M per (node, link): row slot j of face row r at
// ((slot_r + j) C + c) n_1 + x_1 (coalesced over x_1); the end nodes' x_1-face links at
// E + ((2 r + h) J + jx) C + c, E = nslots C n_1, J = 2d - 1, h = 0 (x_1 = 0) or 1, jx = xface_link.

template <int D>
__host__ __device__ constexpr uint64_t xface_mask(int sgn) {
  constexpr Lattice<D> L{};
  uint64_t m = 0;
  for (int k = 0; k < Lattice<D>::Q; ++k)
    if (L.e[k][0] == sgn) m |= 1ull << k;
  return m;
}

// Coefficient pointer and stride of unknown link k at node x_1 of face row r (see the layout above).
template <int D>
__device__ __forceinline__ const double *face_coef(const FaceRow &fr, uint32_t r, int x1, int face1, int k, int C,
                                                   int n1, int32_t nslots, const double *sep, int &cs) {
  if ((fr.mask >> k) & 1ull) {
    const int j = __popcll(fr.mask & ((1ull << k) - 1ull));
    cs = n1;
    return sep + ((int64_t)(fr.slot + j) * C) * n1 + x1;
  }
  constexpr int J = 2 * D - 1;
  const int h = face1 > 0 ? 0 : 1;
  cs = 1;
  return sep + (int64_t)nslots * C * n1 + ((int64_t)(2 * r + h) * J + xface_link<D>(k, face1)) * C;
}

// Separable coefficients of the family's boundary data on the face rows (once per data set).
template <int D, int KIND>
__global__ void __launch_bounds__(128) k_face_sep(const BoundaryArgs b, const FaceRow *__restrict__ rows, int64_t nwork,
                                                  int32_t nslots, double *__restrict__ sep) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const int n1 = b.g.n[0];
  const uint32_t r = b.g.dv[0].div((uint32_t)t);
  const int x1 = (int)((uint32_t)t - r * (uint32_t)n1);
  const FaceRow fr = rows[r];
  int x[D];
  x[0] = x1;
  {
    uint32_t q = (uint32_t)fr.row;
#pragma unroll
    for (int i = 1; i < D; ++i) {
      if (i == D - 1) {
        x[i] = (int)q;
      } else {
        const uint32_t q2 = b.g.dv[i].div(q);
        x[i] = (int)(q - q2 * (uint32_t)b.g.n[i]);
        q = q2;
      }
    }
  }
  const int face1 = x1 == 0 ? 1 : (x1 == n1 - 1 ? -1 : 0);
  const int C = 1 + 2 * b.nmodes;
  double sn[kMaxModes], cs[kMaxModes];
  const double G = family_node_phases<D>(b, x, sn, cs);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const bool row_link = (fr.mask >> k) & 1ull;
    if (!row_link && !(face1 != 0 && L.e[k][0] == face1)) continue;
    int st = 0;
    double *p = const_cast<double *>(face_coef<D>(fr, r, x1, face1, k, C, n1, nslots, sep, st));
    family_sep_coefs<D, KIND>(b, k, G, sn, cs, p, st);
  }
}

// Separable coefficients of the family's data for the x_1-face nodes of the interior rows (k_xface_data),
// at xsep + ((2 r + h) J + j) C: row r, side h, link j = xface_link (once per data set).
template <int D, int KIND>
__global__ void __launch_bounds__(128) k_xface_sep(const BoundaryArgs b, int64_t nrows, double *__restrict__ xsep) {
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
  const int sgn = h ? -1 : 1, C = 1 + 2 * b.nmodes;
  double sn[kMaxModes], cs[kMaxModes];
  const double G = family_node_phases<D>(b, x, sn, cs);
#pragma unroll
  for (int k = 0; k < Q; ++k)
    if (L.e[k][0] == sgn) family_sep_coefs<D, KIND>(b, k, G, sn, cs, xsep + (t * J + xface_link<D>(k, sgn)) * C, 1);
}

// FP64 forward step of the face rows (one lane per node, rows of n_1 lanes).
template <int D, int KIND, int MODE, bool SEP>
__global__ void __launch_bounds__(LHE_STEP_THREADS) k_step_face(const StepArgs a, const BoundaryArgs b,
                                                                const FaceRow *__restrict__ rows, int32_t nslots,
                                                                const double *__restrict__ sep) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  constexpr uint64_t xlo = xface_mask<D>(1), xhi = xface_mask<D>(-1);
  pdl_trigger();
  pdl_wait();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nwork) return;
  const int n1 = a.g.n[0];
  const uint32_t r = a.g.dv[0].div((uint32_t)t);
  const int x1 = (int)((uint32_t)t - r * (uint32_t)n1);
  const FaceRow fr = rows[r];
  const int32_t site = fr.row * n1 + x1;
  const int face1 = x1 == 0 ? 1 : (x1 == n1 - 1 ? -1 : 0);
  const uint64_t nmask = fr.mask | (face1 > 0 ? xlo : (face1 < 0 ? xhi : 0ull));  // this node's unknown links
  const double *__restrict__ src = static_cast<const double *>(a.src);
  double *__restrict__ dst = static_cast<double *>(a.dst);
  const int64_t S = a.g.S;
  const double Rs = a.Rfield ? __ldg(a.Rfield + site) : 0.0;
  const double *rec = nullptr;
  if (!SEP) rec = b.rec + b.roff[face1 > 0 ? fr.blo : (face1 < 0 ? fr.bhi : fr.bmid + x1 - 1)];
  const int C = 1 + 2 * b.nmodes;
  double f[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const bool unknown = (nmask >> k) & 1ull;
    int32_t o = site;  // pull source x - e_k (inside the box when the link is known)
#pragma unroll
    for (int i = 0; i < D; ++i) o -= L.e[k][i] * a.g.stride[i];
    if (!SEP) {
      const int j = __popcll(nmask & ((1ull << k) - 1ull));
      const double v = __ldg(unknown ? rec + j : src + k * S + o);
      if (unknown) {
        const double bv = b.rec_scale * v;
        f[k] = KIND == 1 ? bv : bv - bnode_fkb<D, false>(b, k, site);
      } else {
        f[k] = v;
      }
    } else if (unknown) {
      int cs = 0;
      const double v = family_sep_value(b, k, face_coef<D>(fr, r, x1, face1, k, C, n1, nslots, sep, cs), cs);
      f[k] = KIND == 1 ? v : v - bnode_fkb<D, false>(b, k, site);
    } else {
      f[k] = __ldg(src + k * S + o);
    }
  }
  const double psi = MODE == kModeS2 ? fixed_moment_sum<Q, 1>(f) + (a.Rfield ? a.dt * Rs : a.dtR)
                                     : fma(a.sig, fixed_moment_sum<Q, 0>(f), a.Rfield ? a.rho_dt * Rs : a.rho_dtR);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const double out = MODE == kModeS2 ? fma(a.omega[k], psi, -f[k]) : fma(a.omega[k], psi, a.mu * f[k]);
    st_stream(dst + k * S + site, out);
  }
}

template <int D>
static cudaError_t step_face_d(int kind, const StepArgs &a, const BoundaryArgs &b, const FaceRow *rows, int32_t nslots,
                               const double *sep, cudaStream_t st) {
  if (a.nwork <= 0) return cudaSuccess;
  const int threads = LHE_STEP_THREADS;
  const unsigned blocks = (unsigned)((a.nwork + threads - 1) / threads);
  const bool s2 = a.s == 2.0, fw = kind == 1;
#define LHE_FACE(K, M, SP) launch_kernel(k_step_face<D, K, M, SP>, blocks, threads, 0, st, false, a, b, rows, nslots, sep)
  if (sep) {
    if (fw) return s2 ? LHE_FACE(1, kModeS2, true) : LHE_FACE(1, kModeGeneral, true);
    return s2 ? LHE_FACE(2, kModeS2, true) : LHE_FACE(2, kModeGeneral, true);
  }
  if (fw) return s2 ? LHE_FACE(1, kModeS2, false) : LHE_FACE(1, kModeGeneral, false);
  return s2 ? LHE_FACE(2, kModeS2, false) : LHE_FACE(2, kModeGeneral, false);
#undef LHE_FACE
}

cudaError_t launch_step_face_fp64(int d, int kind, const StepArgs &a, const BoundaryArgs &b, const FaceRow *rows,
                                  int64_t nrows, int32_t nslots, const double *sep, cudaStream_t st) {
  StepArgs aa = a;
  aa.nwork = nrows * a.g.n[0];
  switch (d) {
    case 2: return step_face_d<2>(kind, aa, b, rows, nslots, sep, st);
    case 3: return step_face_d<3>(kind, aa, b, rows, nslots, sep, st);
    case 4: return step_face_d<4>(kind, aa, b, rows, nslots, sep, st);
    case 5: return step_face_d<5>(kind, aa, b, rows, nslots, sep, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_xface_sep(int d, int kind, const BoundaryArgs &b, int64_t nrows, double *xsep, cudaStream_t st) {
  if (nrows <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((2 * nrows + 127) / 128);
#define LHE_XSEP(DD)                                                              \
  do {                                                                            \
    if (kind == 1) k_xface_sep<DD, 1><<<blocks, 128, 0, st>>>(b, nrows, xsep);   \
    else k_xface_sep<DD, 2><<<blocks, 128, 0, st>>>(b, nrows, xsep);             \
  } while (0)
  switch (d) {
    case 1: LHE_XSEP(1); break;
    case 2: LHE_XSEP(2); break;
    case 3: LHE_XSEP(3); break;
    case 4: LHE_XSEP(4); break;
    case 5: LHE_XSEP(5); break;
    default: return cudaErrorInvalidValue;
  }
#undef LHE_XSEP
  return cudaGetLastError();
}

cudaError_t launch_face_sep(int d, int kind, const BoundaryArgs &b, const FaceRow *rows, int64_t nrows, int32_t nslots,
                            double *sep, cudaStream_t st) {
  const int64_t nwork = nrows * b.g.n[0];
  if (nwork <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nwork + 127) / 128);
#define LHE_SEP(DD)                                                                      \
  do {                                                                                    \
    if (kind == 1) k_face_sep<DD, 1><<<blocks, 128, 0, st>>>(b, rows, nwork, nslots, sep); \
    else k_face_sep<DD, 2><<<blocks, 128, 0, st>>>(b, rows, nwork, nslots, sep);           \
  } while (0)
  switch (d) {
    case 2: LHE_SEP(2); break;
    case 3: LHE_SEP(3); break;
    case 4: LHE_SEP(4); break;
    case 5: LHE_SEP(5); break;
    default: return cudaErrorInvalidValue;
  }
#undef LHE_SEP
  return cudaGetLastError();
}

template <int D>
static cudaError_t step_box_d(int kind, const StepArgs &a, const BoundaryArgs &b, double *xb, int64_t nrows,
                              const double *xsep, cudaStream_t st) {
  if (a.nwork <= 0) return cudaSuccess;
  const unsigned dblocks = (unsigned)((2 * nrows + 127) / 128);
  cudaError_t e;
  if (kind == 1) k_xface_data<D, 1><<<dblocks, 128, 0, st>>>(b, xb, nrows, xsep);
  else k_xface_data<D, 2><<<dblocks, 128, 0, st>>>(b, xb, nrows, xsep);
  if ((e = cudaGetLastError())) return e;
  const int threads = LHE_STEP_THREADS;
  const unsigned blocks = (unsigned)((a.nwork + threads - 1) / threads);
  const double *cxb = xb;
  if (a.s == 2.0) return launch_kernel(k_step_box<D, kModeS2>, blocks, threads, 0, st, false, a, cxb);
  return launch_kernel(k_step_box<D, kModeGeneral>, blocks, threads, 0, st, false, a, cxb);
}

cudaError_t launch_step_box_fp64(int d, int kind, const StepArgs &a, const BoundaryArgs &b, double *xb, int64_t nrows,
                                 const double *xsep, cudaStream_t st) {
  switch (d) {
    case 1: return step_box_d<1>(kind, a, b, xb, nrows, xsep, st);
    case 2: return step_box_d<2>(kind, a, b, xb, nrows, xsep, st);
    case 3: return step_box_d<3>(kind, a, b, xb, nrows, xsep, st);
    case 4: return step_box_d<4>(kind, a, b, xb, nrows, xsep, st);
    case 5: return step_box_d<5>(kind, a, b, xb, nrows, xsep, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lhe

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

// The unknown populations of the x_1-face nodes of a Dirichlet box (those whose other coordinates
// are interior), for k_step_box: for interior row r (x_2..x_D interior) and side h (0: x_1 = 0, 1:
// x_1 = n_1 - 1), the 2D - 1 unknown links (e_k,1 = +1 on the low side, -1 on the high side) at
// xb[(2 r + h)(2D - 1) + j], exactly as the boundary-node kernel forms them: the boundary data (from the
// exact-solution family, or from the records of jets: the x_1-face-only nodes lead the boundary-node
// list, low face then high face, each in row order), and for the half-way scheme minus f*_kbar at the
// node (the state at the start of the step).
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
  const double sum = split_moment_sum<Q, kBoxFixedTerms<Q>>(f);  // the split moment sum of the larger lattices (lhe_device.cuh)
  const double psi = MODE == kModeS2 ? fma(2.0, sum, a.Rfield ? a.dt * Rs : a.dtR)
                                     : fma(a.sig, sum, a.Rfield ? a.rho_dt * Rs : a.rho_dtR);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const double out = MODE == kModeS2 ? fma(a.omega[k], psi, -f[k]) : fma(a.omega[k], psi, a.mu * f[k]);
    st_stream(dst + k * S + site, out);
  }
}

// ------------------------------------------------------------------------------ dense boundary data
// The whole box in one row kernel. The boundary data of a step are kept in an array shaped like the
// populations, bdata[k S + x], set only where population k of node x is unknown (its pull source
// x - e_k lies outside the box): the step kernel then chooses, per link and lane, between that entry
// and the pulled population by address arithmetic alone, so every load of a lane is independent and
// coalesced, boundary nodes or not. The producers below fill the entries from the records of jets or
// the manufactured solution (copied in the order of k over each node's unknown links, bit for bit the
// values of the boundary-node kernel) or from the exact-solution family (its data separated in time,
// formed once per data set).

// Lattice coordinates of `site` (x_1 fastest).
template <int D>
__device__ __forceinline__ void site_coords(const Geom &g, int32_t site, int (&x)[D]) {
  uint32_t r = (uint32_t)site;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if (i == D - 1) {
      x[i] = (int)r;
    } else {
      const uint32_t q = g.dv[i].div(r);
      x[i] = (int)(r - q * (uint32_t)g.n[i]);
      r = q;
    }
  }
}

// The family's data for unknown link k at a node, separated in time: P at p[0], A_m at p[(1 + 2m) st],
// B_m at p[(2 + 2m) st]; G = b + g.x, sn/cs = sin/cos(kappa_m . x). Full-way (Eq. (bun1), tabulated):
// omega_k [h - C_k - sum_m T_mk cos xi_m] with h = G + (R - g.u) t + sum_m a_m sin xi_m; half-way
// (Eq. (bun2) without -f*_kbar): wp_k lin + K_k + sum_m (U_mk sin xi_m + V_mk cos xi_m), lin = G + (R - g.u) t;
// xi_m = kappa_m . x + psi_m, so sin xi = sin(k.x) cos psi + cos(k.x) sin psi, cos xi = cos(k.x) cos psi -
// sin(k.x) sin psi.
template <int D, int KIND>
__device__ __forceinline__ void family_sep_coefs(const BoundaryArgs &b, int k, double G, const double *sn,
                                                 const double *cs, double *p, int64_t st) {
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

// The family's data from separable coefficients p (stride st) at this step: P + lt_k + sum_m (A_m cos psi_m
// + B_m sin psi_m).
__device__ __forceinline__ double family_sep_value(const BoundaryArgs &b, int k, const double *p, int64_t st) {
  double v = __ldg(p) + b.lt[k];
  for (int m = 0; m < b.nmodes; ++m) {
    v = fma(__ldg(p + (1 + 2 * m) * st), b.ph_c[m], v);
    v = fma(__ldg(p + (2 + 2 * m) * st), b.ph_s[m], v);
  }
  return v;
}

// The entries that a step sets, one per (unknown link k, boundary node x), given as ent[e] = (k << 32) | x:
// first those whose pull source leaves the box through a face of x_2..x_d ("row links": for the whole
// row the same links), sorted by k and then by x, kept in the dense array bdata[k S + x], where they form
// runs of at least n_1 nodes; then the links through an x_1 face only, at the two end nodes of each row,
// kept after it at Q S + (2 row + h) J + jx (h = 0 at x_1 = 0, 1 at x_1 = n_1 - 1; J = 2d - 1;
// jx = xface_link), compact per row end. Both producers' writes and the step kernel's reads are then contiguous.

// Links with e_k,i = sgn (bit k): those unknown at a node on the low (sgn = 1) or high (-1) face of axis i.
template <int D>
__host__ __device__ constexpr uint64_t face_links(int i, int sgn) {
  constexpr Lattice<D> L{};
  uint64_t m = 0;
  for (int k = 0; k < Lattice<D>::Q; ++k)
    if (L.e[k][i] == sgn) m |= 1ull << k;
  return m;
}

// The links of node x that leave the box through a face of x_2..x_d (bit k).
template <int D>
__device__ __forceinline__ uint64_t row_links_out(const Geom &g, const int (&x)[D]) {
  uint64_t m = 0;
#pragma unroll
  for (int i = 1; i < D; ++i) {
    if (x[i] == 0) m |= face_links<D>(i, 1);
    if (x[i] == g.n[i] - 1) m |= face_links<D>(i, -1);
  }
  return m;
}

// Separable coefficients of the family's data per entry, sep[c nent + e] (c < 1 + 2M: each coefficient
// contiguous over the entries, so that the per-step producer's loads are coalesced). Once per data set.
template <int D, int KIND>
__global__ void __launch_bounds__(128) k_family_sep(const BoundaryArgs b, const long long *__restrict__ ent,
                                                    int64_t nent, double *__restrict__ sep) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nent) return;
  const long long tg = ent[e];
  const int k = (int)(tg >> 32);
  const int32_t site = (int32_t)(tg & 0xffffffffll);
  int x[D];
  site_coords<D>(b.g, site, x);
  double G = b.b;  // b + g.x
#pragma unroll
  for (int i = 0; i < D; ++i) G = fma(b.gl[i], b.x0[i] + (double)x[i] * b.dx, G);
  double sn[kMaxModes], cs[kMaxModes];  // sin and cos of kappa_m . x
  for (int m = 0; m < b.nmodes; ++m) {
    double ph = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) ph = fma(b.kappa[m * kMaxD + i], b.x0[i] + (double)x[i] * b.dx, ph);
    sincos(ph, &sn[m], &cs[m]);
  }
  family_sep_coefs<D, KIND>(b, k, G, sn, cs, sep + e, nent);
}

// The unknown populations of this step into the dense array, one thread per entry (k, x): the records
// (formed in the order of the entries) times rec_scale, or the family's data from its separable
// coefficients (lt, ph_c, ph_s of the step in b); half-way minus f*_kbar(x) of the state at the start
// of the step (b.src). The same operations, in the same order, as the boundary-node kernel.
// A row entry (e < nrow_ent) goes to k S + x of the dense array and its half-way partner is kbar S + x,
// both formed from the entry's (k, x) (two 8-byte index loads fewer per entry); dst[e] is the entry's
// place in the dense array (k S + x) or, for the row-end entries, after it (Q S + (2 row + h) J + jx),
// and opp[e] = kbar S + x.
template <int KIND, bool REC>
__global__ void __launch_bounds__(256) k_bdata_step(const BoundaryArgs b, const long long *__restrict__ ent,
                                                    const long long *__restrict__ dst, const long long *__restrict__ opp,
                                                    int64_t nent, const double *__restrict__ data,
                                                    double *__restrict__ bdata) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nent) return;
  // (full-way records need no (k, x): their dst[e] costs the same bytes as the entry)
  const bool row = (!REC || KIND == 2) && e < b.nrow_ent;
  const long long tg = (row || !REC) ? __ldg(ent + e) : 0ll;
  const int k = (int)(tg >> 32);
  const long long x = tg & 0xffffffffll;
  double v = REC ? b.rec_scale * __ldg(data + e) : family_sep_value(b, k, data + e, nent);
  if (KIND == 2)
    v = v - __ldg(static_cast<const double *>(b.src) + (row ? (long long)b.kbar[k] * b.g.S + x : __ldg(opp + e)));
  bdata[row ? (long long)k * b.g.S + x : __ldg(dst + e)] = v;
}

// FP64 step of every node of a Dirichlet box (whole rows, x_1 fastest): each population is the pulled
// one or, when unknown, the entry of the dense array that k_bdata_step set for this step; then the
// collision of the bulk. No arithmetic per link: on GB300 an FP64 operation per link costs as much as
// the collision (the FP64 pipe retires ~2 per clock per SM).
template <int D, int MODE>
__global__ void __launch_bounds__(LHE_STEP_THREADS) k_step_box_dense(const StepArgs a, const double *__restrict__ bdata) {
  constexpr Lattice<D> L{};
  constexpr int Q = Lattice<D>::Q;
  pdl_trigger();
  pdl_wait();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nwork) return;
  constexpr int J = 2 * D - 1;
  int x[D];
  const int32_t site = decode_site<D, false>(a.g, t, x);
  const int side1 = x[0] == 0 ? 1 : (x[0] == a.g.n[0] - 1 ? -1 : 0);
  // this row end's x_1-face entries, after the dense part
  const double *xrow = bdata + (int64_t)Q * a.g.S + ((int64_t)2 * a.g.dv[0].div((uint32_t)t) + (side1 < 0 ? 1 : 0)) * J;
  const double *__restrict__ src = static_cast<const double *>(a.src);
  double *__restrict__ dst = static_cast<double *>(a.dst);
  const int64_t S = a.g.S;
  const double Rs = a.Rfield ? __ldg(a.Rfield + site) : 0.0;
  double f[Q];
  const uint64_t row_out = row_links_out<D>(a.g, x);
  const uint64_t x_out = side1 > 0 ? face_links<D>(0, 1) : (side1 < 0 ? face_links<D>(0, -1) : 0ull);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const bool row_unknown = (row_out >> k) & 1ull;
    const bool x_unknown = (x_out >> k) & 1ull;
    const int jx = L.e[k][0] == 1 ? xface_link<D>(k, 1) : xface_link<D>(k, -1);
    int32_t o = site;  // pull source x - e_k (inside the box when the link is known)
#pragma unroll
    for (int i = 0; i < D; ++i) o -= L.e[k][i] * a.g.stride[i];
    f[k] = __ldg(row_unknown ? bdata + k * S + site : (x_unknown ? xrow + jx : src + k * S + o));
  }
  // the split moment sum of the larger lattices (lhe_device.cuh)
  const double sum = split_moment_sum<Q, kBoxFixedTerms<Q>>(f);
  const double psi = MODE == kModeS2 ? fma(2.0, sum, a.Rfield ? a.dt * Rs : a.dtR)
                                     : fma(a.sig, sum, a.Rfield ? a.rho_dt * Rs : a.rho_dtR);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const double out = MODE == kModeS2 ? fma(a.omega[k], psi, -f[k]) : fma(a.omega[k], psi, a.mu * f[k]);
    st_stream(dst + k * S + site, out);
  }
}

template <int D>
static cudaError_t step_box_dense_d(const StepArgs &a, const double *bdata, cudaStream_t st) {
  const int threads = LHE_STEP_THREADS;
  const unsigned blocks = (unsigned)((a.nwork + threads - 1) / threads);
  const bool pdl = a.pdl != 0;
  if (a.s == 2.0) return launch_kernel(k_step_box_dense<D, kModeS2>, blocks, threads, 0, st, pdl, a, bdata);
  return launch_kernel(k_step_box_dense<D, kModeGeneral>, blocks, threads, 0, st, pdl, a, bdata);
}

cudaError_t launch_step_box_dense(int d, const StepArgs &a, const double *bdata, cudaStream_t st) {
  StepArgs aa = a;
  aa.nwork = a.g.S;
  if (aa.nwork <= 0) return cudaSuccess;
  switch (d) {
    case 1: return step_box_dense_d<1>(aa, bdata, st);
    case 2: return step_box_dense_d<2>(aa, bdata, st);
    case 3: return step_box_dense_d<3>(aa, bdata, st);
    case 4: return step_box_dense_d<4>(aa, bdata, st);
    case 5: return step_box_dense_d<5>(aa, bdata, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_bdata_step(int kind, bool rec, const BoundaryArgs &b, const long long *ent, const long long *dst,
                              const long long *opp, int64_t nent, const double *data, double *bdata, cudaStream_t st) {
  if (nent <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nent + 255) / 256);
  if (kind == 1) {
    if (rec) k_bdata_step<1, true><<<blocks, 256, 0, st>>>(b, ent, dst, opp, nent, data, bdata);
    else k_bdata_step<1, false><<<blocks, 256, 0, st>>>(b, ent, dst, opp, nent, data, bdata);
  } else {
    if (rec) k_bdata_step<2, true><<<blocks, 256, 0, st>>>(b, ent, dst, opp, nent, data, bdata);
    else k_bdata_step<2, false><<<blocks, 256, 0, st>>>(b, ent, dst, opp, nent, data, bdata);
  }
  return cudaGetLastError();
}

cudaError_t launch_family_sep(int d, int kind, const BoundaryArgs &b, const long long *ent, int64_t nent, double *sep,
                              cudaStream_t st) {
  if (nent <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nent + 127) / 128);
  const bool fw = kind == 1;
#define LHE_FSEP(DD) \
  (fw ? k_family_sep<DD, 1><<<blocks, 128, 0, st>>>(b, ent, nent, sep) : k_family_sep<DD, 2><<<blocks, 128, 0, st>>>(b, ent, nent, sep))
  switch (d) {
    case 1: LHE_FSEP(1); break;
    case 2: LHE_FSEP(2); break;
    case 3: LHE_FSEP(3); break;
    case 4: LHE_FSEP(4); break;
    case 5: LHE_FSEP(5); break;
    default: return cudaErrorInvalidValue;
  }
#undef LHE_FSEP
  return cudaGetLastError();
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
  if (a.s == 2.0) return launch_kernel(k_step_box<D, kModeS2>, blocks, threads, 0, st, false, a, cxb);
  return launch_kernel(k_step_box<D, kModeGeneral>, blocks, threads, 0, st, false, a, cxb);
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

}  // namespace lhe

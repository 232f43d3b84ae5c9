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
  const double psi = MODE == kModeS2 ? fixed_moment_sum<Q, 1>(f) + (a.Rfield ? a.dt * Rs : a.dtR)
                                     : fma(a.sig, fixed_moment_sum<Q, 0>(f), a.Rfield ? a.rho_dt * Rs : a.rho_dtR);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const double out = MODE == kModeS2 ? fma(a.omega[k], psi, -f[k]) : fma(a.omega[k], psi, a.mu * f[k]);
    st_stream(dst + k * S + site, out);
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

// lhe_step_dev.cu -- fused pull-stream + BGK collision with populations stored as FP32 deviations
// from the local equilibrium and the macroscopic variable accumulated in FP64.
//
// State at t_n: phi(x) and g*_k(x) = f*_k(x) - omega_k phi(x) (FP32), f* post-collision; phi is
// stored as an exact double-float pair h + l (48-bit significand, 8 bytes).
// With delta_k = phi(x - e_k) - phi(x) (forward pull direction):
//   f_k(x)      = omega_k phi(x - e_k) + g*_k(x - e_k)
//   phi_new(x)  = sum_k f_k(x) = phi(x) + Delta,   Delta = sum_k omega_k delta_k + sum_k g*_k(x - e_k)
//   g_k         = f_k - omega_k phi_new = omega_k (delta_k - Delta) + g*_k(x - e_k)
//   g*_k(new)   = (1 - s) g_k + dt omega_k R(x)                 (Eq. (BGK-LB-Evolution))
// Delta and the deviations are O(dx) and carried in FP32; the neighbour differences are
// delta_k = (h_k - h) + (l_k - l) in FP32 (exact leading part by Sterbenz for nearby values), and
// the moment update phi_new = h + (l + Delta) is formed as an exact FP32 pair (df_add: TwoSum,
// leading part the exact sum truncated to 24 bits, residual rounded to nearest).
//
// The adjoint uses the same kernel with the reverse pull (x + e_k), no source, and the weighted
// adjoint variable zeta_k = omega_k W + eps_k (W a double-float pair, eps in FP32); W_new is
// accumulated into dL/dR(x) += dt W_new.
#include "lhe_internal.h"
#include "lhe_sites.cuh"

namespace lhe {

// Register caps for the large lattices: D4Q33 at 5 resident blocks per SM (96 registers, no spills)
// and D5Q51 at 3 (168 registers, no spills). More registers per thread keep more of a node's loads in
// flight, more resident warps hide more latency; measured on this kernel, in % of the HBM copy
// bandwidth: D4Q33 48^4 uncapped 71 %, cap of 5 blocks 88 % (of 3 or 4: 87.6 %); D5Q51 24^5 uncapped
// (146 registers) 66 %, 4 blocks (128 registers, spills) 74 %, 2 blocks (196 registers) 69 %, 3 blocks
// 84 %. (A two-pass form for D5Q51, which reads the pulled values again for the new deviations so that
// 126 registers suffice at 4 blocks, measured 77 %.) The FP64 kernel is not capped: there the spills
// cost more than the occupancy gains (D5Q51 76 -> 66 %).
template <int D>
constexpr int dev_min_blocks() { return D == 4 ? 5 : (D == 5 ? 3 : 1); }

template <int D, bool ADJ, bool INTERIOR, bool S2>
__global__ void __launch_bounds__(LHE_STEP_THREADS, dev_min_blocks<D>()) k_step_dev(const StepArgs a) {
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
  const float *__restrict__ src = static_cast<const float *>(a.src);
  float *__restrict__ dst = static_cast<float *>(a.dst);
  const float2 *__restrict__ phis = a.phi_src;
  const int64_t S = a.g.S;

  const float2 p0 = __ldg(phis + site);
  const bool field = !ADJ && a.Rfield != nullptr;
  const float oms = (float)a.oms;
  float dl[Q], gk[Q];
  float accw = 0.0f, accg = 0.0f;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int32_t o = source_site<D, ADJ>(L, k, site, om, op);
    gk[k] = __ldg(src + k * S + o);
    if (k == 0) {
      dl[k] = 0.0f;
    } else {
      const float2 pk = __ldg(phis + o);
      dl[k] = (pk.x - p0.x) + (pk.y - p0.y);
    }
    accw = fmaf(a.omega_f[k], dl[k], accw);
    accg += gk[k];
  }
  const float Delta = accw + accg;
  const float2 pn = df_add(p0.x, p0.y + Delta);
  a.phi_dst[site] = pn;
  if (ADJ && a.gR) a.gR[site] = fma(a.dt, df_value(pn), a.gR[site]);
  float dtR = 0.0f;
  if (field) dtR = (float)(a.dt * __ldg(a.Rfield + site));
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const float r = fmaf(a.omega_f[k], dl[k] - Delta, gk[k]);  // pre-collision deviation g_k
    const float src_k = ADJ ? 0.0f : (field ? a.omega_f[k] * dtR : a.dtwR_f[k]);
    const float out = S2 ? (src_k - r) : fmaf(oms, r, src_k);
    st_stream(dst + k * S + site, out);
  }
}

template <int D, bool ADJ, bool INTERIOR>
static cudaError_t launch_step_dev_t(const StepArgs &a, cudaStream_t st) {
  if (a.nwork <= 0) return cudaSuccess;
  const int threads = LHE_STEP_THREADS;
  const unsigned blocks = (unsigned)((a.nwork + threads - 1) / threads);
  if (a.s == 2.0) return launch_kernel(k_step_dev<D, ADJ, INTERIOR, true>, blocks, threads, 0, st, a.pdl != 0, a);
  return launch_kernel(k_step_dev<D, ADJ, INTERIOR, false>, blocks, threads, 0, st, a.pdl != 0, a);
}

template <int D>
static cudaError_t step_dev_d(bool adjoint, bool interior, const StepArgs &a, cudaStream_t st) {
  if (adjoint) return interior ? launch_step_dev_t<D, true, true>(a, st) : launch_step_dev_t<D, true, false>(a, st);
  return interior ? launch_step_dev_t<D, false, true>(a, st) : launch_step_dev_t<D, false, false>(a, st);
}

cudaError_t launch_step_dev(int d, bool adjoint, bool interior, const StepArgs &a, cudaStream_t st) {
  switch (d) {
    case 1: return step_dev_d<1>(adjoint, interior, a, st);
    case 2: return step_dev_d<2>(adjoint, interior, a, st);
    case 3: return step_dev_d<3>(adjoint, interior, a, st);
    case 4: return step_dev_d<4>(adjoint, interior, a, st);
    case 5: return step_dev_d<5>(adjoint, interior, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lhe

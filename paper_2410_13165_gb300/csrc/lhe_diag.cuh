// lhe_diag.cuh -- the per-node body and the block reduction of the diagnostics (mass, kinetic
// entropy of Eq. (skfk), max |phi|, non-finite count), shared by the handle's reduction kernels
// (lhe_misc.cu) and the allocation-free entry point (lhe_noalloc.cu), so that both compute the same
// formula in the same order.
#pragma once

#include <cstdint>

namespace lhe {

// One node of an FP64 post-collision state f* (k-major, Q*S): phi = sum_k f*_k - dt R; the
// pre-collision populations recovered from f* = (1 - s) f + omega (s phi + dt R) (for s = 1 the
// post-collision values are used: recover = false); the entropy sum_k f_k^2 / (2 omega_k) and the
// number of non-finite populations. Accumulates into v = {mass, entropy, max |phi|, non-finite}.
// QT is int (a run-time Q) or a compile-time constant, which lets the caller's loops unroll.
template <typename QT>
__device__ __forceinline__ void diag_site_fp64(const double *__restrict__ f, int64_t S, int64_t site, QT Q,
                                               const double *omega, double s, bool recover, double dtR,
                                               double (&v)[4]) {
  double sum = 0.0, ent = 0.0, bad = 0.0;
  for (int k = 0; k < Q; ++k) sum += f[k * S + site];
  const double phi = sum - dtR;
  const double psi = s * phi + dtR;
  for (int k = 0; k < Q; ++k) {
    const double fs = f[k * S + site];
    if (!isfinite(fs)) bad += 1.0;
    const double fk = recover ? (fs - omega[k] * psi) / (1.0 - s) : fs;
    ent += fk * fk / (2.0 * omega[k]);
  }
  v[0] += phi;
  v[1] += ent;
  v[2] = fmax(v[2], fabs(phi));
  v[3] += bad;
}

// Sum (max for v[2]) of v over the block: warp shuffles, then warp 0's lane 0 adds the warps'
// results in warp order. The block's total is valid in thread 0 only. sh: 4 doubles per warp.
__device__ __forceinline__ void block_reduce4(double (&v)[4], double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] += __shfl_down_sync(0xffffffffu, v[0], o);
    v[1] += __shfl_down_sync(0xffffffffu, v[1], o);
    v[2] = fmax(v[2], __shfl_down_sync(0xffffffffu, v[2], o));
    v[3] += __shfl_down_sync(0xffffffffu, v[3], o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int j = 0; j < 4; ++j) sh[wid * 4 + j] = v[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      v[0] += sh[w * 4 + 0];
      v[1] += sh[w * 4 + 1];
      v[2] = fmax(v[2], sh[w * 4 + 2]);
      v[3] += sh[w * 4 + 3];
    }
  }
}

// Second pass: one block adds the per-block partials (4 per block) in block order and writes the
// four totals to out.
__device__ __forceinline__ void reduce_partials_final(const double *__restrict__ partials, int nblocks,
                                                      double *__restrict__ out, double *sh) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    v[0] += partials[b * 4 + 0];
    v[1] += partials[b * 4 + 1];
    v[2] = fmax(v[2], partials[b * 4 + 2]);
    v[3] += partials[b * 4 + 3];
  }
  block_reduce4(v, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) out[j] = v[j];
}

}  // namespace lhe

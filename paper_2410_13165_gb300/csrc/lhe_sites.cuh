// lhe_sites.cuh -- site decoding and neighbour addressing shared by the step kernels.
#pragma once

#include "lhe_internal.h"

namespace lhe {

// Thread index t -> lattice coordinates x and linear site index. For INTERIOR, t enumerates the
// whole x-rows (x_1 in [0, n_1 - 1]) through the interior of a Dirichlet box (x_i in [1, n_i - 2]
// for i > 1), so that warps read aligned rows; the caller skips x_1 = 0 and x_1 = n_1 - 1.
template <int D, bool INTERIOR>
__device__ __forceinline__ int32_t decode_site(const Geom &g, int64_t t, int (&x)[D]) {
  uint32_t r = (uint32_t)t;
  int32_t site = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const bool inner = INTERIOR && i > 0;
    const int32_t ni = inner ? g.n[i] - 2 : g.n[i];
    if (i == D - 1) {
      x[i] = (int)r;
    } else {
      const uint32_t q = inner ? g.dvi[i].div(r) : g.dv[i].div(r);
      x[i] = (int)(r - q * (uint32_t)ni);
      r = q;
    }
    if (inner) x[i] += 1;
    site += x[i] * g.stride[i];
  }
  return site;
}

// Interior rows include the two face nodes of each row; their threads do nothing.
template <int D, bool INTERIOR>
__device__ __forceinline__ bool skip_site(const Geom &g, const int (&x)[D]) {
  return INTERIOR && (x[0] == 0 || x[0] == g.n[0] - 1);
}

// Offsets from `site` to the neighbours x - e_i and x + e_i along each axis (periodic wrap when
// the box is periodic; interior sites never wrap).
template <int D, bool INTERIOR>
__device__ __forceinline__ void axis_offsets(const Geom &g, const int (&x)[D], int32_t (&om)[D],
                                             int32_t (&op)[D]) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    om[i] = (!INTERIOR && x[i] == 0) ? (g.n[i] - 1) * g.stride[i] : -g.stride[i];
    op[i] = (!INTERIOR && x[i] == g.n[i] - 1) ? -(g.n[i] - 1) * g.stride[i] : g.stride[i];
  }
}

// Source site of population k: x - e_k (forward) or x + e_k (adjoint).
template <int D, bool ADJ>
__device__ __forceinline__ int32_t source_site(const Lattice<D> &L, int k, int32_t site, const int32_t (&om)[D],
                                               const int32_t (&op)[D]) {
  int32_t o = site;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if (L.e[k][i] == 1) o += ADJ ? op[i] : om[i];
    if (L.e[k][i] == -1) o += ADJ ? om[i] : op[i];
  }
  return o;
}

}  // namespace lhe

// lhe_device.cuh -- device-side building blocks shared by the kernels of the library:
// the DdQ(2d^2+1) lattice as compile-time tables, division by run-time invariant integers,
// the fixed-point moment sum and the integer double -> float-pair split.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lhe {

constexpr int kMaxD = 5;
constexpr int kMaxQ = 51;
constexpr int kMaxModes = 16;

// ----------------------------------------------------------------------------------------------
// Lattice (Sec. 2.3, Eq. (DdQ-M)): k = 0 rest; k = 1..d: +e_i; k = d+1..2d: -e_i; then for each
// pair i<j (lexicographic) four velocities with component i from J1 = (1,-1,-1,1) and component
// j from J2 = (1,1,-1,-1). Built at compile time so unrolled loops see constant components.
template <int D>
struct Lattice {
  static constexpr int Q = 2 * D * D + 1;
  int e[Q][D];
  int opp[Q];
  int nnz[Q];
  int ax[Q][2];  // indices of the nonzero components (-1 if absent)
  __host__ __device__ constexpr Lattice() : e{}, opp{}, nnz{}, ax{} {
    const int J1[4] = {1, -1, -1, 1}, J2[4] = {1, 1, -1, -1};
    for (int k = 0; k < Q; ++k)
      for (int i = 0; i < D; ++i) e[k][i] = 0;
    int k = 1;
    for (int i = 0; i < D; ++i) e[k++][i] = 1;
    for (int i = 0; i < D; ++i) e[k++][i] = -1;
    for (int i = 0; i < D; ++i)
      for (int j = i + 1; j < D; ++j)
        for (int r = 0; r < 4; ++r) {
          e[k][i] = J1[r];
          e[k][j] = J2[r];
          ++k;
        }
    for (int a = 0; a < Q; ++a) {
      opp[a] = -1;
      for (int b = 0; b < Q; ++b) {
        bool same = true;
        for (int i = 0; i < D; ++i)
          if (e[b][i] != -e[a][i]) same = false;
        if (same) opp[a] = b;
      }
      nnz[a] = 0;
      ax[a][0] = ax[a][1] = -1;
      for (int i = 0; i < D; ++i)
        if (e[a][i] != 0) ax[a][nnz[a]++] = i;
    }
  }
};

// ----------------------------------------------------------------------------------------------
// Division of a 32-bit unsigned by a run-time invariant divisor with one multiply-high
// (Granlund & Montgomery, "Division by invariant integers using multiplication", PLDI 1994):
// q = (umulhi(n, m) + n) >> l with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1.
struct FastDiv {
  uint32_t d = 1, m = 0;
  int32_t l = 0;
  FastDiv() = default;
  __host__ explicit FastDiv(uint32_t div) : d(div) {
    l = 0;
    while ((1ull << l) < div) ++l;
    m = (uint32_t)((((1ull << 32) * ((1ull << l) - div)) / div) + 1ull);
    if (div == 1) m = 0;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    return (uint32_t)(((uint64_t)__umulhi(n, m) + n) >> l);
  }
};

// ----------------------------------------------------------------------------------------------
// Powers of two built from their bit pattern (no FP64 arithmetic): valid for -1022 <= p <= 1023.
__device__ __forceinline__ double pow2_bits(int p) {
  return __hiloint2double((p + 1023) << 20, 0);
}

__host__ __device__ constexpr int ceil_log2(int q) {
  int l = 0;
  while ((1 << l) < q) ++l;
  return l;
}

// Moment sum sum_k f_k of Q doubles accumulated exactly in 64-bit fixed point, aligned to the
// largest exponent: each term's 53-bit significand is shifted into a common frame with G guard
// bits (G = 10 - ceil(log2 Q) keeps Q terms below 2^63) and rounded to nearest on the way. The
// result is mult * sum + add with one rounding of the integer total. The error is below one
// unit in the last place of the largest |f_k| (sequential FP64 addition: up to (Q-1)/2 units).
// GB300 executes FP64 arithmetic and FP32<->FP64 conversions at ~2 per clock per SM, integer
// arithmetic ~30x faster; this moves the Q-1 additions of the moment sum off the FP64 pipe.
// NaN or Inf inputs fall back to plain FP64 addition so they propagate.
template <int Q>
__device__ __forceinline__ double fixed_moment_sum(const double (&f)[Q], double mult, double add) {
  constexpr int G = 10 - ceil_log2(Q);
  static_assert(G >= 3, "too many terms for a 64-bit accumulator");
  int emax = 0;
#pragma unroll
  for (int k = 0; k < Q; ++k) emax = max(emax, (__double2hiint(f[k]) >> 20) & 0x7FF);
  if (emax == 0x7FF) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < Q; ++k) s += f[k];
    return fma(mult, s, add);
  }
  const int E = max(emax, 1);
  long long acc = 0;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const unsigned hi = (unsigned)__double2hiint(f[k]);
    const unsigned lo = (unsigned)__double2loint(f[k]);
    const int e = (int)((hi >> 20) & 0x7FFu);
    const unsigned mh = (hi & 0xFFFFFu) | (e ? 0x100000u : 0u);
    const unsigned long long mg = ((((unsigned long long)mh) << 32) | lo) << G;  // < 2^(53+G)
    const int sh = E - max(e, 1);
    unsigned long long v;
    if (sh == 0) v = mg;
    else if (sh <= 53 + G) v = (mg + (1ull << (sh - 1))) >> sh;  // round half up
    else v = 0ull;
    acc += (hi >> 31) ? -(long long)v : (long long)v;
  }
  const double a = __ll2double_rn(acc);
  const int p = E - 1075 - G;
  if (p >= -1022) return fma(a, mult * pow2_bits(p), add);
  return fma(a * pow2_bits(p + 600), mult * pow2_bits(-600), add);
}

// Split a double into an unevaluated float pair x ~ h + l without FP64 arithmetic: h is x with
// its significand truncated to 24 bits, l the next 23 bits of the residual (|x - h - l| < 2^-47 |x|).
// Values outside the normal float range take the (rare) FP64 conversion path.
__device__ __forceinline__ void split_pair(double x, float &h, float &l) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7FFu);
  const int ef = e - 896;  // float biased exponent of the leading part
  if (ef >= 1 && ef <= 254) {
    const unsigned sign = hi & 0x80000000u;
    h = __uint_as_float(sign | ((unsigned)ef << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
    const unsigned r23 = (lo & 0x1FFFFFFFu) >> 6;
    const float rf = __uint_as_float(0x4B000000u | r23) - 8388608.0f;  // exact: r23 < 2^23
    const int es = e - 942;                                              // 2^(e - 1075 + 6)
    const float lv = (es >= 1) ? rf * __uint_as_float((unsigned)es << 23) : 0.0f;
    l = __uint_as_float(__float_as_uint(lv) ^ sign);
  } else {
    h = __double2float_rn(x);
    l = 0.0f;
  }
}

// Streaming stores: the new state is not re-read by this kernel.
__device__ __forceinline__ void st_stream(double *p, double v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(float *p, float v) { __stcs(p, v); }

}  // namespace lhe

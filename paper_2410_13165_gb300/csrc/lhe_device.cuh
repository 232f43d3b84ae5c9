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

// Threads per block of the fused step kernels (one thread per lattice node).
#ifndef LHE_STEP_THREADS
#define LHE_STEP_THREADS 128
#endif

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

// Moment sum of Q doubles, accumulated exactly in 64-bit fixed point on the integer pipes.
// Each term's 53-bit significand is placed, with G guard bits (G = 10 - ceil(log2 Q) keeps Q terms
// below 2^63), in the frame of the largest exponent present, rounding to nearest (ties up) when it
// is shifted right; the integer total is converted back to a correctly rounded double (ties to even)
// with integer operations only, times 2^P2. The error is below one unit in the last place of the
// largest |f_k| (sequential FP64 addition: up to (Q-1)/2 units). GB300 runs FP64 arithmetic and
// FP32<->FP64 conversions at ~2 per clock per SM and integer arithmetic far faster, so this takes
// the Q-1 additions of the moment sum (and the conversion) off the FP64 pipe.
// Subnormal terms are placed as if their exponent were 0 instead of 1 (an error below 2^-1022 in
// absolute value); any NaN or infinite term makes the result NaN.
template <int Q, int P2, class Get>
__device__ __forceinline__ double fixed_moment_sum_impl(Get f) {
  constexpr int G = 10 - ceil_log2(Q);
  static_assert(G >= 3, "too many terms for a 64-bit accumulator");
  unsigned emf = 0u;  // largest exponent field, in place (bits 20..30 of the high word)
#pragma unroll
  for (int k = 0; k < Q; ++k) emf = max(emf, (unsigned)__double2hiint(f(k)) & 0x7FF00000u);
  if (emf == 0x7FF00000u) return __longlong_as_double(0x7FF8000000000000ll);
  emf = max(emf, 0x00100000u);
  long long acc = 0;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const double fk = f(k);
    const unsigned hi = (unsigned)__double2hiint(fk);
    const unsigned lo = (unsigned)__double2loint(fk);
    const unsigned ef = hi & 0x7FF00000u;
    const unsigned mh = (hi & 0x000FFFFFu) | min(ef, 0x00100000u);  // implicit bit unless zero/subnormal
    const unsigned sh = (emf - max(ef, 0x00100000u)) >> 20;
    const unsigned long long m = ((((unsigned long long)mh) << 32) | lo) << G;  // < 2^(53+G)
    unsigned long long v;
    if (sh < 32u) v = (m + ((1ull << sh) >> 1)) >> sh;
    else if (sh < 64u) v = (m + (1ull << (sh - 1))) >> sh;
    else v = 0ull;
    const long long sg = (long long)((int)hi >> 31);  // 0 or -1
    acc += ((long long)v ^ sg) - sg;
  }
  if (acc == 0) return 0.0;
  const unsigned long long sbit = acc < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long a = acc < 0 ? (unsigned long long)(-acc) : (unsigned long long)acc;
  const int lz = __clzll((long long)a);
  a <<= lz;                                  // leading one at bit 63
  unsigned long long mant = a >> 11;         // 53 bits with the leading one
  const unsigned rem = (unsigned)a & 0x7FFu; // dropped bits
  mant += (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  int ex = (63 - lz) + (int)(emf >> 20) - 1075 - G + 1023 + P2;
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  if (ex <= 0 || ex >= 2047) {  // result outside the normal range: convert and scale in two exact steps
    const int p = (int)(emf >> 20) - 1075 - G + P2;
    const int p1 = p / 2;
    return __ll2double_rn(acc) * pow2_bits(p1) * pow2_bits(p - p1);
  }
  return __longlong_as_double((long long)(sbit | ((unsigned long long)ex << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

template <int Q, int P2>
__device__ __forceinline__ double fixed_moment_sum(const double (&f)[Q]) {
  return fixed_moment_sum_impl<Q, P2>([&](int k) { return f[k]; });
}

// Moment sum of the FP64 step kernels of the larger lattices. The fixed-point sum's integer work grows
// with Q while the FP64 pipe, which the collision keeps about half busy, has room: the first NFX terms
// are summed in fixed point and the rest added on the FP64 pipe. The split is chosen per kernel from
// scans on GB300 (number of fixed-point terms): the periodic step splits D5Q51 only (38 of 51: 24^5
// 1.269 -> 1.148 ms; a D4Q33 split made the 48^4 step slower, 0.444 -> 0.467 ms), the row kernels of
// Dirichlet boxes split D4Q33 as well (29 of 33: 64^4 1.711 -> 1.672 ms). The error is within
// (Q - NFX + 1) / 2 units in the last place of the sum (the oracle's sequential FP64 sum: up to
// (Q - 1) / 2).
template <int Q>
constexpr int kPeriodicFixedTerms = Q == 51 ? 38 : Q;
template <int Q>
constexpr int kBoxFixedTerms = Q == 51 ? 38 : (Q == 33 ? 29 : Q);

template <int Q, int NFX>
__device__ __forceinline__ double split_moment_sum(const double (&f)[Q]) {
  double s = fixed_moment_sum_impl<NFX, 0>([&](int k) { return f[k]; });
#pragma unroll
  for (int k = NFX; k < Q; ++k) s += f[k];
  return s;
}

// Double-float storage of the macroscopic variable of the FP32-deviation form: phi = h + l with h
// the value truncated to 24 significant bits and l the rounded residual (a 48-bit significand,
// relative spacing 2^-48). Neighbour differences are then plain FP32 arithmetic.
__device__ __forceinline__ double df_value(float2 p) { return (double)p.x + (double)p.y; }

__device__ __forceinline__ float2 df_split(double x) {
  const double hd = __hiloint2double(__double2hiint(x), __double2loint(x) & (int)0xE0000000);
  return make_float2((float)hd, (float)(x - hd));
}

// New pair for h + t, with h the leading part of a pair and t an FP32 increment: h' is the exact sum
// rounded toward zero to 24 significant bits, l' = (h + t) - h' rounded to nearest. TwoSum gives
// s + e = h + t exactly (s the rounded-to-nearest sum); when s was rounded away from zero it is moved
// one step toward zero, and s - h' (0 or one ulp) is exact. FP32 arithmetic only (the intrinsics
// keep the compiler from contracting or reordering the error terms).
__device__ __forceinline__ float2 df_add(float h, float t) {
  const float s = __fadd_rn(h, t);
  const float bp = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(t, bp));
  const bool away = (s > 0.0f && e < 0.0f) || (s < 0.0f && e > 0.0f);
  const float hn = away ? __int_as_float(__float_as_int(s) - 1) : s;
  return make_float2(hn, __fadd_rn(__fsub_rn(s, hn), e));
}

// Stores of the new state with the default cache policy. The evict-first hint (st.global.cs) was
// measured 0.6-1.7 % slower on every step kernel (D3Q19 256^3 FP64 744.6 vs 739.8 us, D4Q33 48^4 FP32
// deviations 252.9 vs 248.6 us), bitwise the same results.
__device__ __forceinline__ void st_stream(double *p, double v) { *p = v; }
__device__ __forceinline__ void st_stream(float *p, float v) { *p = v; }

// Programmatic dependent launch. A step kernel lets the next kernel of its stream be scheduled as
// soon as every CTA of this one is running (pdl_trigger), and waits for the kernel before it to
// complete, with its memory visible, before it touches global memory (pdl_wait). When the kernel was
// launched without the programmatic-serialization attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace lhe

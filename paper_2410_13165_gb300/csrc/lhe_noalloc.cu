// lhe_noalloc.cu -- diagnostics of a caller-owned FP64 state with no device allocation.
//
// Some callers cannot allocate device memory at the point where they want to inspect a state:
// code whose device memory is handed out by a framework's own allocator or capped by a fixed
// budget, or code running where the CUDA runtime refuses a cudaMalloc. lhe_lbm_diagnostics
// needs a handle, and handles allocate; this entry point needs neither. Its only scratch memory
// (the per-block partial sums of the reduction) lives in the file-scope device array below, which
// exists from the moment the library is loaded on a device until the process exits.
#include <mutex>
#include <string>

#include "lhe_internal.h"

namespace lhe {
constexpr int kNoAllocMaxBlocks = 4096;  // capacity of the scratch array below, in reduction blocks
}

// Four partial sums per block (mass, entropy, max |phi|, non-finite count): 128 KiB per device.
static __device__ __align__(256) double g_noalloc_partials[lhe::kNoAllocMaxBlocks * 4];

namespace lhe {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int64_t kNoAllocSitesPerBlock = 65536;  // each block reduces one contiguous chunk of nodes
constexpr int64_t kNoAllocMaxSites = kNoAllocSitesPerBlock * kNoAllocMaxBlocks;  // 268,435,456 nodes

struct NoAllocArgs {
  int64_t S;
  int32_t Q;
  const double *pop;
  const double *Rfield;
  double omega[kMaxQ];
  double s, dt, dtR;
};

__device__ __forceinline__ void reduce4(double (&v)[4], double *sh) {
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
  if (threadIdx.x == 0)
    for (int w = 1; w < nw; ++w) {
      v[0] += sh[w * 4 + 0];
      v[1] += sh[w * 4 + 1];
      v[2] = fmax(v[2], sh[w * 4 + 2]);
      v[3] += sh[w * 4 + 3];
    }
}

// Block b reduces nodes [b * kNoAllocSitesPerBlock, min(S, (b + 1) * kNoAllocSitesPerBlock)) and
// overwrites its own four partials, so nothing in the scratch array has to be cleared first.
// Per node: phi = sum_k f*_k - dt R, the pre-collision populations recovered from
// f* = (1 - s) f + omega (s phi + dt R) (post-collision values when s = 1), and the kinetic entropy
// sum_k f_k^2 / (2 omega_k).
__global__ void __launch_bounds__(kNoAllocThreads) k_noalloc_partials(const NoAllocArgs a, double *partials) {
  __shared__ double sh[(kNoAllocThreads / 32) * 4];
  const int64_t begin = (int64_t)blockIdx.x * kNoAllocSitesPerBlock;
  const int64_t end = min(a.S, begin + kNoAllocSitesPerBlock);
  const bool recover = a.s != 1.0;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t site = begin + threadIdx.x; site < end; site += kNoAllocThreads) {
    const double dtR = a.Rfield ? a.dt * a.Rfield[site] : a.dtR;
    double sum = 0.0, ent = 0.0, bad = 0.0;
    for (int k = 0; k < a.Q; ++k) sum += a.pop[k * a.S + site];
    const double phi = sum - dtR;
    const double psi = a.s * phi + dtR;
    for (int k = 0; k < a.Q; ++k) {
      const double fs = a.pop[k * a.S + site];
      if (!isfinite(fs)) bad += 1.0;
      const double fk = recover ? (fs - a.omega[k] * psi) / (1.0 - a.s) : fs;
      ent += fk * fk / (2.0 * a.omega[k]);
    }
    v[0] += phi;
    v[1] += ent;
    v[2] = fmax(v[2], fabs(phi));
    v[3] += bad;
  }
  reduce4(v, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) partials[blockIdx.x * 4 + j] = v[j];
}

__global__ void __launch_bounds__(kNoAllocThreads) k_noalloc_final(const double *partials, int nblocks, double *out) {
  __shared__ double sh[(kNoAllocThreads / 32) * 4];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += kNoAllocThreads) {
    v[0] += partials[b * 4 + 0];
    v[1] += partials[b * 4 + 1];
    v[2] = fmax(v[2], partials[b * 4 + 2]);
    v[3] += partials[b * 4 + 3];
  }
  reduce4(v, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) out[j] = v[j];
}

// Device address of the scratch array, resolved once per device (the host-side symbol is only a
// stand-in and must never be handed to a kernel).
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace lhe

extern "C" LHE_API lhe_status lhe_lbm_diagnostics_noalloc(const lhe_lbm_params *p, const double *pop_dev,
                                                          const double *R_dev, double *out_dev) {
  using namespace lhe;
  if (!p || !pop_dev || !out_dev) return record_error(LHE_ERR_ARG, "params, pop_dev and out_dev must not be NULL");
  if (p->precision != LHE_FP64)
    return record_error(LHE_ERR_ARG, "lhe_lbm_diagnostics_noalloc reads FP64 populations (precision LHE_FP64)");
  double omega[kMaxQ];
  int32_t Q = 0;
  const lhe_status st = lhe_lbm_model(p, omega, nullptr, nullptr, &Q);
  if (st != LHE_OK && st != LHE_ERR_UNSTABLE) return st;
  int64_t S = 1;
  for (int i = 0; i < p->d; ++i) {
    S *= p->n[i];
    if (S > kNoAllocMaxSites)
      return record_error(LHE_ERR_ARG, "lhe_lbm_diagnostics_noalloc handles at most 268435456 lattice nodes "
                                       "(4096 blocks of 65536 nodes in its fixed scratch array)");
  }
  double *scratch = nullptr;
  const cudaError_t se = scratch_for_current_device(&scratch);
  if (se != cudaSuccess)
    return record_error(LHE_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(se));
  NoAllocArgs a{};
  a.S = S;
  a.Q = Q;
  a.pop = pop_dev;
  a.Rfield = R_dev;
  for (int k = 0; k < Q; ++k) a.omega[k] = omega[k];
  a.s = 1.0 / p->tau;
  // dt = dx / c with dx from the first dimension (lhe_lbm_model has checked that dx agrees in all).
  const double span = (p->bc == LHE_BC_FULLWAY) ? (double)(p->n[0] - 1) : (double)p->n[0];
  a.dt = (p->hi[0] - p->lo[0]) / span / p->c;
  a.dtR = a.dt * p->R;
  const int nblocks = (int)((S + kNoAllocSitesPerBlock - 1) / kNoAllocSitesPerBlock);
  cudaStream_t stream = static_cast<cudaStream_t>(p->stream);
  k_noalloc_partials<<<nblocks, kNoAllocThreads, 0, stream>>>(a, scratch);
  k_noalloc_final<<<1, kNoAllocThreads, 0, stream>>>(scratch, nblocks, out_dev);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return record_error(LHE_ERR_CUDA, std::string("diagnostics launch: ") + cudaGetErrorString(le));
  return LHE_OK;
}

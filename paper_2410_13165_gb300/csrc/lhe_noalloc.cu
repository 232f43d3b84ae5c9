// lhe_noalloc.cu -- diagnostics of a caller-owned FP64 state with no device allocation.
//
// Some callers cannot allocate device memory at the point where they want to inspect a state:
// code whose device memory is handed out by a framework's own allocator or capped by a fixed
// budget, or code running where the CUDA runtime refuses a cudaMalloc. lhe_lbm_diagnostics
// needs a handle, and handles allocate; this entry point needs neither. Its only scratch memory
// (the per-block partial sums of the reduction) lives in the file-scope device array below, which
// exists from the moment the library is loaded on a device until the process exits.
#include <cuda.h>  // CUcontext / CUresult types only; the driver call is reached through the runtime

#include <algorithm>
#include <mutex>
#include <string>

#include "lhe_diag.cuh"
#include "lhe_internal.h"

namespace lhe {
constexpr int kNoAllocMaxBlocks = 4096;  // capacity of the scratch array below, in reduction blocks
}

// Four partial sums per block (mass, entropy, max |phi|, non-finite count): 128 KiB per device.
static __device__ __align__(256) double g_noalloc_partials[lhe::kNoAllocMaxBlocks * 4];

namespace lhe {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocBlocksPerSM = 4;
constexpr int64_t kNoAllocMaxSites = int64_t(1) << 28;  // 268,435,456 nodes: the stated maximum

struct NoAllocArgs {
  int64_t S;
  int32_t Q;
  const double *pop;
  const double *Rfield;
  double omega[kMaxQ];
  double s, dt, dtR;
};

// Grid-stride over the nodes; block b overwrites its own four partials, so nothing in the scratch
// array has to be cleared first. The per-node formula is diag_site_fp64, as in the handle's kernel.
__global__ void __launch_bounds__(kNoAllocThreads) k_noalloc_partials(const NoAllocArgs a, double *partials) {
  __shared__ double sh[(kNoAllocThreads / 32) * 4];
  const bool recover = a.s != 1.0;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t site = (int64_t)blockIdx.x * kNoAllocThreads + threadIdx.x; site < a.S;
       site += (int64_t)gridDim.x * kNoAllocThreads) {
    const double dtR = a.Rfield ? a.dt * a.Rfield[site] : a.dtR;
    diag_site_fp64(a.pop, a.S, site, a.Q, a.omega, a.s, recover, dtR, v);
  }
  block_reduce4(v, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) partials[blockIdx.x * 4 + j] = v[j];
}

__global__ void __launch_bounds__(kNoAllocThreads) k_noalloc_final(const double *partials, int nblocks, double *out) {
  __shared__ double sh[(kNoAllocThreads / 32) * 4];
  reduce_partials_final(partials, nblocks, out, sh);
}

// The scratch array's device address, per device. The host-side symbol g_noalloc_partials is only
// a stand-in and must never be handed to a kernel. The address belongs to the context in which the
// module was loaded: after cudaDeviceReset, or when the primary context is destroyed and created
// again, the module is loaded anew and the array may sit elsewhere. So each entry remembers the
// context it was resolved in (cuCtxGetId: unique for the life of the process) and is resolved
// again whenever the current context differs.
constexpr int kMaxDevices = 64;
struct ScratchEntry {
  unsigned long long ctx_id = 0;
  double *ptr = nullptr;
  int sms = 0;
};
std::mutex g_scratch_mu;
ScratchEntry g_scratch[kMaxDevices];

using CtxGetIdFn = CUresult(CUDAAPI *)(CUcontext, unsigned long long *);

CtxGetIdFn ctx_get_id_fn() {
  static CtxGetIdFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<CtxGetIdFn>(p);
  }();
  return fn;
}

// Id of the current context, or 0 if none is current on this thread (yet).
unsigned long long current_ctx_id() {
  const CtxGetIdFn fn = ctx_get_id_fn();
  unsigned long long id = 0;
  if (!fn || fn(nullptr, &id) != CUDA_SUCCESS) return 0;
  return id;
}

cudaError_t scratch_for_current_device(double **out, int *sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!ctx_get_id_fn()) return cudaErrorNotSupported;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchEntry &ent = g_scratch[dev];
  unsigned long long id = current_ctx_id();
  if (id == 0 || id != ent.ctx_id || !ent.ptr) {
    // cudaGetSymbolAddress also makes the device's primary context current on this thread when
    // no context is, so the id is read (again) after it.
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    id = current_ctx_id();
    if (id == 0) return cudaErrorDeviceUninitialized;  // "invalid device context"
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    ent.ctx_id = id;
    ent.ptr = static_cast<double *>(p);
    ent.sms = n;
  }
  *out = ent.ptr;
  *sms = ent.sms;
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
  const std::string prev_error = lhe_lbm_last_error(nullptr);
  double omega[kMaxQ];
  int32_t Q = 0;
  const lhe_status st = lhe_lbm_model(p, omega, nullptr, nullptr, &Q);
  if (st == LHE_ERR_UNSTABLE && !p->allow_unstable) return st;  // as lhe_lbm_create: some omega_k <= 0
  if (st != LHE_OK && st != LHE_ERR_UNSTABLE) return st;
  if (st == LHE_ERR_UNSTABLE) record_error(LHE_OK, prev_error);  // accepted: keep the caller's last error
  int64_t S = 1;
  for (int i = 0; i < p->d; ++i) {
    S *= p->n[i];
    if (S > kNoAllocMaxSites)
      return record_error(LHE_ERR_ARG, "lhe_lbm_diagnostics_noalloc handles at most 268435456 lattice nodes");
  }
  double *scratch = nullptr;
  int sms = 0;
  const cudaError_t se = scratch_for_current_device(&scratch, &sms);
  if (se != cudaSuccess)
    return record_error(LHE_ERR_CUDA, std::string("scratch address (cudaGetSymbolAddress / cuCtxGetId): ") +
                                          cudaGetErrorString(se));
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
  int64_t nb = (S + kNoAllocThreads - 1) / kNoAllocThreads;
  nb = std::min<int64_t>(nb, (int64_t)kNoAllocBlocksPerSM * std::max(sms, 1));
  nb = std::max<int64_t>(1, std::min<int64_t>(nb, kNoAllocMaxBlocks));
  const int nblocks = (int)nb;
  cudaStream_t stream = static_cast<cudaStream_t>(p->stream);
  k_noalloc_partials<<<nblocks, kNoAllocThreads, 0, stream>>>(a, scratch);
  k_noalloc_final<<<1, kNoAllocThreads, 0, stream>>>(scratch, nblocks, out_dev);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return record_error(LHE_ERR_CUDA, std::string("diagnostics launch: ") + cudaGetErrorString(le));
  return LHE_OK;
}

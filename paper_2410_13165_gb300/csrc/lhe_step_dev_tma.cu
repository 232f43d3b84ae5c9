// lhe_step_dev_tma.cu -- the FP32-deviation step on periodic D3Q19 boxes with the pulled rows staged
// in shared memory by bulk asynchronous copies (the TMA engine), several tiles in flight per SM.
//
// The arithmetic per node is that of k_step_dev (lhe_step_dev.cu), in the same order, so the two
// kernels give identical bits. What changes is how the populations reach the SM. The plain kernel
// keeps every load in flight in registers, which caps the bytes in flight per SM and leaves it
// latency bound at ~90 % of the copy bandwidth. Here a tile is R whole x-rows (y0..y0+R-1 at one z);
// for each tile a producer warp issues, per population k, the R source rows of g*_k (rows shifted
// by -e_k in y and z with periodic wrap; the x shift and its wrap are applied when reading shared
// memory), the 3(R+2) rows of phi that the tile's neighbourhood touches and, when used, the tile's
// rows of dL/dR (adjoint) or of the source field R(x) (forward). The copies of a tile
// complete on its stage's "full" mbarrier; the consumer warps compute the tile and release the
// stage on its "empty" mbarrier, after which the producer refills it. NS stages rotate, one
// persistent CTA per SM walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... and no block-wide
// barrier is taken inside the loop. Within one call of several steps, a step's kernel is scheduled
// while the previous one finishes and sets up its barriers before it waits for it (programmatic
// dependent launch).
//
// Every mbarrier wait is bounded in time; on expiry the kernel stops, records the failure in a
// host-visible flag, waits (bounded) for its copies in flight and returns. Each warp takes the decision
// to stop as a whole, so that no warp-wide operation runs with lanes missing.
#include "lhe_internal.h"

namespace lhe {

namespace {

#ifndef LHE_TMA_CONSUMER_WARPS
#define LHE_TMA_CONSUMER_WARPS 10
#endif
constexpr int kConsumerWarps = LHE_TMA_CONSUMER_WARPS;  // compute warps; one more warp issues the copies
constexpr int kTmaThreads = 32 * (kConsumerWarps + 1);
#ifndef LHE_TMA_TILE_NODES
#define LHE_TMA_TILE_NODES 512
#endif
constexpr int kTileNodes = LHE_TMA_TILE_NODES;  // nodes per tile (whole rows, at most this many)
#ifndef LHE_TMA_SMEM_BUDGET
#define LHE_TMA_SMEM_BUDGET (200u * 1024u)
#endif
#ifndef LHE_TMA_MIN_BLOCKS
#define LHE_TMA_MIN_BLOCKS 1
#endif
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s per wait (a tile takes microseconds)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Non-blocking test of the phase (try_wait may suspend the thread for a while before it answers).
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// true once the phase with the given parity has completed; false after limit_ns (or 2^30 polls), or
// as soon as *abort is set (abort may be null). limit_ns == 0 tests once without blocking (the test
// hook of LHE_FLAG_TEST_EXPIRE_WAIT).
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns, const volatile int *abort) {
  if (limit_ns == 0) return mbar_test_wait(bar, parity);
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort && *abort) return false;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// Global -> shared bulk copy completing on an mbarrier of the issuing CTA (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Tile number T of the launch (T = blockIdx.x + i gridDim.x): block ty of R rows in y of plane z.
struct TileRef {
  int ty, z;
};

__device__ __forceinline__ TileRef tile_ref(const DevTmaPlan &p, int T) {
  TileRef t;
  t.z = T / p.tiles_y;
  t.ty = T - t.z * p.tiles_y;
  return t;
}

// Issues the copies of tile t into stage s (the producer warp; lane 0 arms the barrier). Lane k < Q
// copies the R source rows of g*_k, lanes Q..Q+2 the R+2 phi rows of the planes z-1, z, z+1; rows
// that are consecutive in y are one copy (a run breaks only where y wraps).
template <bool ADJ>
__device__ __forceinline__ void issue_tile(const StepArgs &a, const DevTmaPlan &p, unsigned char *smem, uint32_t bar,
                                           TileRef t, int s, int lane) {
  constexpr int Q = Lattice<3>::Q;
  const int sgn = ADJ ? -1 : 1;
  const int z = t.z;
  const int y0 = t.ty * p.R;
  const uint32_t stage = smem_u32(smem) + (uint32_t)s * p.stage_bytes;
  if (lane == 0) mbar_arrive_expect_tx(bar, p.tx_bytes);
  __syncwarp();
  if (lane < Q) {
    const int k = lane;
    const int zz = wrap(z - sgn * p.ez[k], p.nz);
    const float *base = static_cast<const float *>(a.src) + (int64_t)k * a.g.S + (int64_t)p.ny * zz * p.nx;
    const uint32_t dst0 = stage + (uint32_t)(k * p.R * p.nx) * 4u;
    int r = 0;
    while (r < p.R) {
      const int y = wrap(y0 + r - sgn * p.ey[k], p.ny);
      int len = 1;
      while (r + len < p.R && y + len < p.ny) ++len;
      bulk_g2s(dst0 + (uint32_t)(r * p.nx) * 4u, base + (int64_t)y * p.nx, (uint32_t)(len * p.nx) * 4u, bar);
      r += len;
    }
  } else if (lane == Q + 3) {
    const double *xs = ADJ ? a.gR : a.Rfield;
    if (p.tx_bytes > p.g_bytes + p.phi_bytes && xs)
      bulk_g2s(stage + p.g_bytes + p.phi_bytes, xs + (int64_t)(y0 + p.ny * z) * p.nx, p.x_bytes, bar);
  } else if (lane < Q + 3) {
    const int dzi = lane - Q;
    const int zz = wrap(z + dzi - 1, p.nz);
    const float2 *base = a.phi_src + (int64_t)p.ny * zz * p.nx;
    const uint32_t dst0 = stage + p.g_bytes + (uint32_t)(dzi * (p.R + 2) * p.nx) * 8u;
    int j = 0;
    while (j < p.R + 2) {
      const int y = wrap(y0 - 1 + j, p.ny);
      int len = 1;
      while (j + len < p.R + 2 && y + len < p.ny) ++len;
      bulk_g2s(dst0 + (uint32_t)(j * p.nx) * 8u, base + (int64_t)y * p.nx, (uint32_t)(len * p.nx) * 8u, bar);
      j += len;
    }
  }
}

}  // namespace

// NXC: the row length n_1 when it is fixed at compile time (rows of 128 or 256 nodes, tiles of
// kTileNodes nodes: R = kTileNodes / NXC), so that the node index of a unit splits into row and x without a runtime
// division and the shared-memory offsets fold into constants; 0 for any other row length.
template <bool ADJ, bool S2, int NXC>
__global__ void __launch_bounds__(kTmaThreads, LHE_TMA_MIN_BLOCKS) k_step_dev3_tma(const StepArgs a, const DevTmaPlan p) {
  constexpr Lattice<3> L{};
  constexpr int Q = Lattice<3>::Q;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kTmaMaxStages];
  __shared__ __align__(8) uint64_t empty[kTmaMaxStages];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int my = p.ntiles > (int)blockIdx.x ? (p.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  pdl_trigger();
  if (tid == 0) {
    for (int s = 0; s < p.NS; ++s) {
      mbar_init(smem_u32(&full[s]), 1u);
      mbar_init(smem_u32(&empty[s]), (uint32_t)kConsumerWarps);
    }
    fence_mbar_init();
    fence_proxy_async();
    abort_flag = 0;
  }
  pdl_wait();  // the barriers are set up while the previous step finishes
  __syncthreads();

  const volatile int *abort_v = &abort_flag;
  if (warp == kConsumerWarps) {
    // producer warp: refill a stage as soon as every consumer warp has released it. Lane 0 waits and
    // decides; the decision is broadcast so that the warp leaves the loop as one.
    int i = 0;
    for (; i < my; ++i) {
      const int s = i % p.NS;
      const TileRef t = tile_ref(p, (int)blockIdx.x + i * (int)gridDim.x);
      if (i >= p.NS) {
        int stop = 0;
        if (lane == 0)
          stop = !mbar_wait(smem_u32(&empty[s]), (uint32_t)((i / p.NS - 1) & 1), kWaitLimitNs, abort_v) || *abort_v;
        if (__shfl_sync(0xffffffffu, stop, 0)) {
          if (lane == 0) *(volatile int *)&abort_flag = 1;
          break;
        }
      }
      issue_tile<ADJ>(a, p, smem, smem_u32(&full[s]), t, s, lane);
    }
    if (lane == 0) {
      bool aborted = *abort_v != 0;
      // leave only once the last stages have been consumed (bounded; given up if the consumers stop)
      for (int j = max(0, my - p.NS); j < my && !aborted; ++j)
        aborted = !mbar_wait(smem_u32(&empty[j % p.NS]), (uint32_t)((j / p.NS) & 1), kWaitLimitNs, abort_v);
      if (aborted) {
        *p.err = 1;
        // the latest copies issued into each stage, possibly not consumed: wait for them (bounded)
        // so that no copy into this CTA's shared memory is in flight when it exits
        for (int j = max(0, i - p.NS); j < i; ++j)
          mbar_wait(smem_u32(&full[j % p.NS]), (uint32_t)((j / p.NS) & 1), kWaitLimitNs, nullptr);
      }
    }
    __syncwarp();
    return;
  }

  // consumer warps
  // (the row length and tile height, constants where NXC fixes them, else read from the plan at each
  // use, so that the generic instantiation compiles as if NXC did not exist)
#define LHE_NX (NXC ? NXC : p.nx)
#define LHE_TILE_R (NXC ? kTileNodes / NXC : p.R)
  const int sgn = ADJ ? -1 : 1;
  const int64_t S = a.g.S;
  const float oms = (float)a.oms;
  const bool field = !ADJ && a.Rfield != nullptr;
  for (int i = 0; i < my; ++i) {
    const int s = i % p.NS;
    // every lane waits on the barrier itself (each observes the copies' completion); the warp stops as
    // one if any lane's wait gave up or another warp stopped
    const bool ok = mbar_wait(smem_u32(&full[s]), (uint32_t)((i / p.NS) & 1), p.consumer_wait_ns, abort_v);
    if (__any_sync(0xffffffffu, !ok || *abort_v)) {
      if (lane == 0) {
        *(volatile int *)&abort_flag = 1;
        *p.err = 1;
      }
      break;
    }
    const TileRef t = tile_ref(p, (int)blockIdx.x + i * (int)gridDim.x);
    float *__restrict__ dst = static_cast<float *>(a.dst);
    float2 *__restrict__ phi_dst = a.phi_dst;
    const int z = t.z;
    const int y0 = t.ty * LHE_TILE_R;
    const float *G = reinterpret_cast<const float *>(smem + (size_t)s * p.stage_bytes);
    const float2 *P = reinterpret_cast<const float2 *>(smem + (size_t)s * p.stage_bytes + p.g_bytes);
    const double *X = reinterpret_cast<const double *>(smem + (size_t)s * p.stage_bytes + p.g_bytes + p.phi_bytes);
    // 32-node units of the tile, dealt to the consumer warps round robin over the whole sequence of
    // units of this CTA, so that warps which drew fewer units in one tile draw more in the next
    const int units = (LHE_TILE_R * LHE_NX + 31) >> 5;
    const int u0 = (int)(((unsigned)warp + (unsigned)kConsumerWarps - (unsigned)((i * units) % kConsumerWarps)) %
                         (unsigned)kConsumerWarps);
    for (int u = u0; u < units; u += kConsumerWarps) {
      const int idx = u * 32 + lane;
      if (idx >= LHE_TILE_R * LHE_NX) break;
      const int r = NXC ? idx / NXC : (int)p.nx_div.div((uint32_t)idx), x = idx - r * LHE_NX;
      const int32_t site = x + LHE_NX * (y0 + r + p.ny * z);
      const int xm = x == 0 ? LHE_NX - 1 : x - 1, xp = x == LHE_NX - 1 ? 0 : x + 1;
      const float2 p0 = P[((LHE_TILE_R + 2) + r + 1) * LHE_NX + x];
      float dl[Q], gk[Q];
      float accw = 0.0f, accg = 0.0f;
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const int ex = sgn * L.e[k][0], ey = sgn * L.e[k][1], ez = sgn * L.e[k][2];
        const int sx = ex == 1 ? xm : (ex == -1 ? xp : x);
        gk[k] = G[(k * LHE_TILE_R + r) * LHE_NX + sx];
        if (k == 0) {
          dl[k] = 0.0f;
        } else {
          const float2 pk = P[((1 - ez) * (LHE_TILE_R + 2) + r + 1 - ey) * LHE_NX + sx];
          dl[k] = (pk.x - p0.x) + (pk.y - p0.y);
        }
        accw = fmaf(a.omega_f[k], dl[k], accw);
        accg += gk[k];
      }
      const float Delta = accw + accg;
      const float2 pn = df_add(p0.x, p0.y + Delta);
      phi_dst[site] = pn;
      if (ADJ && a.gR) a.gR[site] = fma(a.dt, df_value(pn), X[idx]);
      float dtR = 0.0f;
      if (field) dtR = (float)(a.dt * X[idx]);
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const float r = fmaf(a.omega_f[k], dl[k] - Delta, gk[k]);
        const float src_k = ADJ ? 0.0f : (field ? a.omega_f[k] * dtR : a.dtwR_f[k]);
        const float out = S2 ? (src_k - r) : fmaf(oms, r, src_k);
        st_stream(dst + k * S + site, out);
      }
    }
    // release the stage: order this warp's shared-memory reads before the producer's next copies
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
  }
}
#undef LHE_NX
#undef LHE_TILE_R

bool plan_dev3_tma(const Geom &g, int sms, DevTmaPlan &p) {
  if (g.d != 3) return false;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  if (nx % 4 != 0 || nx > 512) return false;
  int R = 1;
  for (int c = 1; c <= ny; ++c)
    if (ny % c == 0 && c * nx <= kTileNodes) R = c;
  const int Q = Lattice<3>::Q;
  const uint32_t g_bytes = (uint32_t)(Q * R * nx * 4);
  const uint32_t phi_bytes = (uint32_t)(3 * (R + 2) * nx * 8);
  const uint32_t x_bytes = (uint32_t)(R * nx * 8);
  const uint32_t stage = g_bytes + phi_bytes + x_bytes;
  const int NS = (int)std::min<uint32_t>((uint32_t)kTmaMaxStages, (uint32_t)(LHE_TMA_SMEM_BUDGET) / stage);
  if (NS < 2) return false;
  constexpr Lattice<3> L{};
  p = DevTmaPlan{};
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.R = R;
  p.NS = NS;
  p.tiles_y = ny / R;
  p.ntiles = p.tiles_y * nz;
  p.g_bytes = g_bytes;
  p.phi_bytes = phi_bytes;
  p.x_bytes = x_bytes;
  p.stage_bytes = stage;
  p.nx_div = FastDiv((uint32_t)nx);
  for (int k = 0; k < Q; ++k) {
    p.ey[k] = (int8_t)L.e[k][1];
    p.ez[k] = (int8_t)L.e[k][2];
  }
  p.grid = std::min(p.ntiles, sms);
  return true;
}

cudaError_t prepare_dev3_tma(const DevTmaPlan &p) {
  const int bytes = p.NS * (int)p.stage_bytes;
  cudaError_t e;
#define LHE_SMEM(kernel) \
  if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
  LHE_SMEM((k_step_dev3_tma<false, true, 0>)) LHE_SMEM((k_step_dev3_tma<false, false, 0>))
  LHE_SMEM((k_step_dev3_tma<true, true, 0>)) LHE_SMEM((k_step_dev3_tma<true, false, 0>))
  LHE_SMEM((k_step_dev3_tma<false, true, 128>)) LHE_SMEM((k_step_dev3_tma<false, false, 128>))
  LHE_SMEM((k_step_dev3_tma<true, true, 128>)) LHE_SMEM((k_step_dev3_tma<true, false, 128>))
  LHE_SMEM((k_step_dev3_tma<false, true, 256>)) LHE_SMEM((k_step_dev3_tma<false, false, 256>))
#undef LHE_SMEM
  return cudaSuccess;
}

template <int NXC>
static auto pick_dev3_tma(bool adjoint, bool s2) {
  return adjoint ? (s2 ? k_step_dev3_tma<true, true, NXC> : k_step_dev3_tma<true, false, NXC>)
                 : (s2 ? k_step_dev3_tma<false, true, NXC> : k_step_dev3_tma<false, false, NXC>);
}

cudaError_t launch_step_dev3_tma(bool adjoint, const StepArgs &a, const DevTmaPlan &plan, cudaStream_t st) {
  DevTmaPlan p = plan;
  const bool with_x = adjoint ? a.gR != nullptr : a.Rfield != nullptr;
  p.tx_bytes = p.g_bytes + p.phi_bytes + (with_x ? p.x_bytes : 0u);
  const size_t bytes = (size_t)p.NS * p.stage_bytes;
  const bool s2 = a.s == 2.0;
  // Constant row lengths where they were measured faster: forward 128 and 256, adjoint 128 (the
  // adjoint with constant rows of 256 was 6 % slower than with the runtime ones).
  auto kernel = (p.nx == 128 && p.R == kTileNodes / 128)              ? pick_dev3_tma<128>(adjoint, s2)
                : (!adjoint && p.nx == 256 && p.R == kTileNodes / 256) ? (s2 ? k_step_dev3_tma<false, true, 256>
                                                                              : k_step_dev3_tma<false, false, 256>)
                                                                       : pick_dev3_tma<0>(adjoint, s2);
  return launch_kernel(kernel, p.grid, kTmaThreads, bytes, st, a.pdl != 0, a, p);
}

}  // namespace lhe

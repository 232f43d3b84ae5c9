// lhe_internal.h -- host-side handle and kernel launch interfaces of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "lhe_device.cuh"
#include "lhe_lbm.h"

namespace lhe {

// Geometry of a box of n_i nodes (x_1 fastest).
struct Geom {
  int32_t d = 0;
  int32_t n[kMaxD] = {1, 1, 1, 1, 1};
  int32_t stride[kMaxD] = {0, 0, 0, 0, 0};
  FastDiv dv[kMaxD];   // divide by n_i (site -> coordinates)
  FastDiv dvi[kMaxD];  // divide by n_i - 2 (interior row index -> coordinates)
  int64_t S = 0;
  int64_t S_interior = 0;
  int64_t S_rows = 0;  // n_1 * prod_{i>1} (n_i - 2): the whole x-rows through interior nodes
};

// Arguments of the fused stream + collide kernels (forward and adjoint, both precisions).
struct StepArgs {
  Geom g;
  const void *src;         // populations at t_n (double or float, Q*S)
  void *dst;               // populations at t_{n+1}
  const float2 *phi_src;   // FP32_DEV: phi at t_n as a double-float pair (S)
  float2 *phi_dst;         // FP32_DEV: phi at t_{n+1}
  const double *Rfield;    // per-site source R(x) or nullptr (forward only)
  double *gR;              // adjoint: dL/dR(x) accumulator (S) or nullptr
  double omega[kMaxQ];
  float omega_f[kMaxQ];
  float dtwR_f[kMaxQ];     // FP32_DEV: dt * omega_k * R (constant source)
  double s, oms;           // s and 1 - s
  double dtR;              // dt * R (constant source)
  double dt, half_dt;
  // FP64 collision with s != 2 (see kCollide* in lhe_step_fp64.cu): f*_k = mu f_k + omega_k psi with
  // psi = sig sum_k f_k + rho_dt R(x) (or + rho_dtR); adjoint: gR += gsc w, psi = sig w.
  double mu, sig, rho_dt, rho_dtR, gsc;
  double pscale;           // macro: factor from the stored populations to f* (1 unless scaled)
  int32_t collide;         // kCollideGeneral / kCollideScaled (s != 2 only)
  int32_t pdl;             // launch with programmatic stream serialization (the kernel calls pdl_wait)
  int64_t nwork;           // number of sites processed (S, or the interior count)
};

// Launch `kernel` on `st`; with pdl set, with the programmatic-stream-serialization attribute, so
// that it may be scheduled while the previous kernel of the stream finishes (the kernel must call
// pdl_wait before it touches global memory).
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                          Args &&...args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1u : 0u;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Plan of the staged FP32-deviation step on periodic D3Q19 boxes (lhe_step_dev_tma.cu).
constexpr int kTmaMaxStages = 4;
struct DevTmaPlan {
  int32_t nx = 0, ny = 0, nz = 0;
  int32_t R = 0;           // x-rows per tile (R divides ny)
  int32_t NS = 0;          // pipeline stages
  int32_t tiles_y = 0, ntiles = 0, grid = 0;
  uint32_t g_bytes = 0;    // populations part of a stage: Q * R * nx floats
  uint32_t phi_bytes = 0;  // 3 (R + 2) nx float2 of phi
  uint32_t x_bytes = 0;    // R nx doubles: dL/dR (adjoint) or R(x) (forward) of the tile, when used
  uint32_t stage_bytes = 0;  // g_bytes + phi_bytes + room for x_bytes
  uint32_t tx_bytes = 0;   // bytes copied per tile in this launch (x part only when used)
  FastDiv nx_div;
  int8_t ey[kMaxQ] = {}, ez[kMaxQ] = {};  // y and z components of e_k
  int32_t *err = nullptr;  // host-mapped flag, set when a pipeline wait timed out
  uint64_t consumer_wait_ns = 1000000000ull;  // limit of the compute warps' waits (0: try once)
};

// FP64 collision forms for s != 2.
constexpr int kCollideGeneral = 0;  // two FP64 operations per population
constexpr int kCollideScaled = 1;   // scaled representation, one FMA per population

// The manufactured solution A exp(-lambda t) prod_i sin(kappa_i x_i + theta_i) and the node grid
// x_i = x0_i + j_i dx (lhe_provider.cu).
struct SineProductArgs {
  double A, lambda;
  double kappa[kMaxD], theta[kMaxD], u[kMaxD], x0[kMaxD];
  double dx;
};

// Arguments of the boundary-node kernels (Dirichlet boxes).
struct BoundaryArgs {
  Geom g;
  const int32_t *sites;    // boundary node indices
  int64_t nsites;
  // Boundary data given as jets (lhe_lbm_set_boundary_jet): per boundary node, one record entry per
  // unknown link in the order of k (rec + roff[node]) holding the population (full-way) or B_k
  // (half-way, Eq. (bun2) without -f*_kbar); rec == nullptr: data from the exact-solution family.
  const int32_t *roff;
  const double *rec;
  const int32_t *rmap = nullptr;  // k_jet_records: the position of each record (else node-major)
  double rec_scale = 1.0;  // factor on every record (a separable solution's time factor)
  const double *Rfield;    // per-site source R(x) of the step, or nullptr for the constant R
  const void *src;
  void *dst;
  const float2 *phi_src;
  float2 *phi_dst;
  const double *table;     // per (mode, k): [kc, cos alpha, sin alpha], then ku per mode
  const double *axis;      // per (mode, axis, node index): [cos, sin] of kappa_mi X_i
  int32_t axis_off[kMaxD]; // offset of axis i in the per-mode block of `axis`
  int32_t axis_len;        // sum_i n_i
  double ph_c[kMaxModes];  // cos and sin of theta_m - kappa_m . u t_eval
  double ph_s[kMaxModes];
  double omega[kMaxQ];
  double wratio[kMaxQ];    // omega_k / omega_kbar (adjoint of the half-way scheme)
  double s, oms, R, dt, dx, c;
  double x0[kMaxD];        // coordinate of node 0
  double u[kMaxD];
  double t_eval;           // time at which the boundary data are evaluated
  int32_t order;
  // exact-solution family (lhe_wave)
  int32_t nmodes;
  double b;
  double gl[kMaxD];
  double a[kMaxModes];
  double kappa[kMaxModes * kMaxD];
  double theta[kMaxModes];
  // the family's data in separable form (k_bdata_family): the unknown population's data is
  // P + lt_k + sum_m (A_m cos psi_m + B_m sin psi_m), psi_m = theta_m - kappa_m . u t_eval (ph_c, ph_s),
  // lt_k the part linear in t_eval (one value per link and step)
  double lt[kMaxQ];
  // the dense boundary data (k_bdata_step): entries [0, nrow_ent) are row links, whose places in the
  // dense array (k S + x) and half-way partners (kbar S + x) follow from the entry's (k, x)
  int64_t nrow_ent;
  int8_t kbar[kMaxQ];      // the link opposite to k
};

struct InitArgs {
  Geom g;
  const double *phi0;
  const double *grad;      // d*S (may be the library's FD buffer)
  const double *Rfield;
  void *dst;
  float2 *phi_dst;
  double omega[kMaxQ];
  double c1[kMaxQ];        // (1 - s)(dt/2) omega_k
  double c2[kMaxQ];        // c (1 - s)(dt/2) omega_k
  double s, oms, dt, dtR, c;
  double u[kMaxD];
  int32_t order;
};

struct ReduceArgs {
  Geom g;
  const void *pop;
  const float2 *phi;       // FP32_DEV
  const double *Rfield;
  double omega[kMaxQ];
  double s, dt, dtR;
  double *partials;        // gridDim.x * 4
  double *out;             // 4 (device)
};

struct AdjGradArgs {
  Geom g;
  const void *adj;         // adjoint populations zeta (FP64) or deviations (FP32_DEV)
  const float2 *adjW;      // FP32_DEV: adjoint macroscopic variable W
  double *gphi0;
  double *G;               // d*S: (dt/2) sum_k (u - c e_k) zeta_k
  double omega[kMaxQ];
  double dt, c;
  double u[kMaxD];
  int32_t order;
};

// Launchers (one per kernel family), implemented in the .cu files; return cudaGetLastError().
cudaError_t launch_step_fp64(int d, bool adjoint, bool interior, const StepArgs &a, cudaStream_t st);
cudaError_t launch_step_dev(int d, bool adjoint, bool interior, const StepArgs &a, cudaStream_t st);
cudaError_t launch_boundary(int d, int kind, bool dev, const BoundaryArgs &a, cudaStream_t st);
cudaError_t launch_jet_records(int d, int kind, const BoundaryArgs &a, const double *jet, const int16_t *jidx,
                               double *rec, cudaStream_t st);
cudaError_t launch_jet_grad(int d, int kind, bool dev, const BoundaryArgs &a, const int16_t *jidx, double *out,
                            cudaStream_t st);
cudaError_t launch_sp_jets(int d, const SineProductArgs &a, const double *pts, int64_t P, const int8_t *tup,
                           double *jet, cudaStream_t st);
cudaError_t launch_sp_source(const SineProductArgs &a, const Geom &g, double *R0, cudaStream_t st);
cudaError_t launch_scale_field(const double *in, double scale, int64_t n, double *out, int sms, cudaStream_t st);
cudaError_t launch_step_box_fp64(int d, int kind, const StepArgs &a, const BoundaryArgs &b, double *xb, int64_t nrows,
                                 cudaStream_t st);
cudaError_t launch_adjoint_boundary(int d, int kind, bool dev, const BoundaryArgs &a, cudaStream_t st);
// FP64 step of a whole Dirichlet box: each unknown population k of node x is read from bdata[k S + x],
// which launch_bdata_step fills for the step from the entries ent[e] = (k << 32) | x (sorted by k then
// x): records in the order of the entries (times b.rec_scale) or, rec = false, the family's separable
// coefficients (1 + 2M per entry, formed once per data set by family_sep); half-way minus f*_kbar(x)
// of b.src.
// The entries of links through a face of x_2..x_d are kept in the dense array; those of links through an
// x_1 face only, at the row ends, after it (Q S + (2 row + h) (2d - 1) + j); dst[e] / opp[e]: each entry's
// place there and the index of f*_kbar at its node (half-way).
cudaError_t launch_step_box_dense(int d, const StepArgs &a, const double *bdata, cudaStream_t st);
cudaError_t launch_bdata_step(int kind, bool rec, const BoundaryArgs &b, const long long *ent, const long long *dst,
                              const long long *opp, int64_t nent, const double *data, double *bdata, cudaStream_t st);
cudaError_t launch_family_sep(int d, int kind, const BoundaryArgs &b, const long long *ent, int64_t nent, double *sep,
                              cudaStream_t st);
cudaError_t launch_stability(int d, const double *omega_dev, int64_t npoints, int32_t nxi, double s,
                             unsigned long long *rho_bits_dev, cudaStream_t st);
cudaError_t launch_init(int d, bool dev, const InitArgs &a, cudaStream_t st);
cudaError_t launch_macro_fp64(int d, const StepArgs &a, double *phi_out, cudaStream_t st);
cudaError_t launch_fd_grad(int d, const Geom &g, double dx, const double *phi, double *grad, cudaStream_t st);
cudaError_t launch_fd_grad_transpose_add(int d, const Geom &g, double dx, const double *G, double *out,
                                         cudaStream_t st);
cudaError_t launch_reduce(int d, bool dev, const ReduceArgs &a, int nblocks, cudaStream_t st);
cudaError_t launch_adjoint_seed(int d, bool dev, const Geom &g, const double *omega, const double *seed,
                                void *adj, float2 *adjW, double *gR, cudaStream_t st);
cudaError_t launch_df_to_double(const float2 *src, double *dst, int64_t n, cudaStream_t st);
cudaError_t launch_scale_fp64(double *p, int64_t n, double factor, cudaStream_t st);
bool plan_dev3_tma(const Geom &g, int sms, DevTmaPlan &p);
cudaError_t prepare_dev3_tma(const DevTmaPlan &p);
cudaError_t launch_step_dev3_tma(bool adjoint, const StepArgs &a, const DevTmaPlan &p, cudaStream_t st);
cudaError_t launch_adjoint_grads(int d, bool dev, const AdjGradArgs &a, cudaStream_t st);

// Record the message lhe_lbm_last_error(NULL) returns on this thread; returns `status`.
lhe_status record_error(lhe_status status, const std::string &msg);

}  // namespace lhe

// The opaque handle of the C ABI.
struct lhe_lbm {
  lhe_lbm_params p{};
  lhe::Geom g;
  int Q = 0;
  double dx = 0, dt = 0, s = 2, R = 0;
  double omega[lhe::kMaxQ] = {};
  double m4[10] = {};
  int32_t e[lhe::kMaxQ * lhe::kMaxD] = {};
  double x0[lhe::kMaxD] = {};
  cudaStream_t stream = nullptr;
  int sms = 0;                  // multiprocessors of the device
  // forward state (ping-pong); FP64: double[Q*S]; FP32_DEV: float[Q*S] + phi float2[S]
  void *pop[2] = {nullptr, nullptr};
  float2 *phi[2] = {nullptr, nullptr};  // FP32_DEV: phi as a double-float pair
  int cur = 0;
  bool initialised = false;
  int64_t step = 0;
  double *Rfield = nullptr;     // owned copy of the per-site source of the last collision, or nullptr
  double *Rnext = nullptr;      // lhe_lbm_set_source: the source of the next step (buffer)
  int32_t Rnext_state = 0;      // 0: nothing pending; 1: the field in Rnext; 2: back to the constant R
  bool grad_was_fd = false;
  int init_order_used = 3;
  double *fdgrad = nullptr;     // d*S scratch for the finite-difference gradient
  // Dirichlet
  int32_t *bsites = nullptr;
  int64_t nb = 0;
  int64_t nb_xface = 0;         // leading entries of bsites on the x_1 faces only (other coordinates
                                // interior): the FP64 forward step treats them in the row kernel
  double *xface = nullptr;      // their boundary data per step (2 (2d - 1) doubles per interior row)
  // FP64 forward (unless LHE_FLAG_NODE_BOUNDARY): the boundary data of the step as a dense array
  // shaped like the populations (set at the unknown entries only), and the separable coefficients of
  // the family's data per record (1 + 2M doubles)
  double *bdata = nullptr;
  long long *bent = nullptr;    // its entries, (k << 32) | x: links through a face of x_2..x_d sorted by k then
                                // x, then those through an x_1 face only sorted by x then k
  long long *bdst = nullptr;    // each entry's place in bdata (the row-end part follows the Q S dense part)
  long long *bopp = nullptr;    // kbar S + x of each entry (half-way)
  int32_t *bmap = nullptr;      // the entry of each record (node-major index -> entry): records of jets and
                                // of the manufactured solution are formed in the order of the entries
  double *fsep = nullptr;
  size_t fsep_len = 0;
  bool have_wave = false;
  lhe_wave wave{};
  // boundary data as jets (lhe_lbm_set_boundary_jet), one step at a time
  bool jet_mode = false;        // the data come from jets (else from the wave)
  bool jet_ready = false;       // jets set for the next step
  std::vector<int32_t> bsites_host;  // boundary nodes in the library's order
  std::vector<int32_t> broff_host;   // per boundary node: first record (unknown links in the order of k)
  int64_t nrec = 0;             // records = (boundary node, unknown link) pairs
  int64_t nrow_ent = 0;         // dense boundary data: entries of row links (the first ones)
  int32_t *broff = nullptr;     // device copies, allocated by the first lhe_lbm_set_boundary_jet
  double *brec = nullptr;
  // lhe_lbm_set_boundary_sine_product: records and source at unit time factor, scaled every step
  bool sp_mode = false;
  double sp_lambda = 0.0;
  double *sp_rec0 = nullptr;
  double *sp_R0 = nullptr;
  double *bc_table = nullptr;
  double *bc_axis = nullptr;    // per-axis phase tables of the Dirichlet data
  // adjoint
  void *adj[2] = {nullptr, nullptr};
  float2 *adjW[2] = {nullptr, nullptr};
  double *gR = nullptr;
  int acur = 0;
  bool adj_ready = false;
  // Scaled representation of the FP64 state when s != 2 on periodic boxes: the stored populations
  // are K f* with K = (1 - s)^-j; j = 0 means the state is stored as f* itself. [0] forward, [1]
  // adjoint. acc accumulates the relative error of the rounded s/(1 - s) factors.
  // staged FP32-deviation step (periodic D3Q19)
  bool staged = false;
  lhe::DevTmaPlan tma{};
  int32_t *tma_err_host = nullptr;
  bool tma_expire_armed = false; // LHE_FLAG_TEST_EXPIRE_WAIT: the next staged launch gives up its waits
  int32_t scale_j[2] = {0, 0};
  double scale_acc[2] = {0.0, 0.0};
  // diagnostics
  double *red_partials = nullptr;
  double *red_out = nullptr;
  int red_blocks = 0;
  std::string err;
};

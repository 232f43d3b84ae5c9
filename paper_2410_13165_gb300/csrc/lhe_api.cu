// lhe_api.cu -- host implementation of the C ABI declared in include/lhe_lbm.h.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lhe_internal.h"

using namespace lhe;

namespace {

thread_local std::string g_last_error;

lhe_status fail(lhe_lbm *lbm, lhe_status st, const std::string &msg) {
  if (lbm) lbm->err = msg;
  else g_last_error = msg;
  return st;
}

lhe_status cuda_fail(lhe_lbm *lbm, cudaError_t e, const char *what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(lbm, e == cudaErrorMemoryAllocation ? LHE_ERR_OOM : LHE_ERR_CUDA, msg);
}

#define LHE_CK(lbm, call)                                    \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(lbm, e_, #call); \
  } while (0)

// Lattice vectors of the paper's DdQ(2d^2+1) ordering (same construction as the device tables).
int lattice_vectors(int d, int32_t *e) {
  switch (d) {
    case 1: { constexpr Lattice<1> L{}; for (int k = 0; k < L.Q; ++k) for (int i = 0; i < 1; ++i) e[k * d + i] = L.e[k][i]; return L.Q; }
    case 2: { constexpr Lattice<2> L{}; for (int k = 0; k < L.Q; ++k) for (int i = 0; i < 2; ++i) e[k * d + i] = L.e[k][i]; return L.Q; }
    case 3: { constexpr Lattice<3> L{}; for (int k = 0; k < L.Q; ++k) for (int i = 0; i < 3; ++i) e[k * d + i] = L.e[k][i]; return L.Q; }
    case 4: { constexpr Lattice<4> L{}; for (int k = 0; k < L.Q; ++k) for (int i = 0; i < 4; ++i) e[k * d + i] = L.e[k][i]; return L.Q; }
    case 5: { constexpr Lattice<5> L{}; for (int k = 0; k < L.Q; ++k) for (int i = 0; i < 5; ++i) e[k * d + i] = L.e[k][i]; return L.Q; }
    default: return -1;
  }
}

// Eq. (meq-4rd) in units of c^4 with sigma = u / c: g * max{lower bounds} + (1 - g) * min{upper bounds},
// the bounds being those of Eq. (psi-4-equal) (equal fourth moments for every pair).
double m4_rule(int d, const double *sig, double g) {
  if (d < 2) return 0.0;
  double ss = 0.0;
  for (int i = 0; i < d; ++i) ss += sig[i] * sig[i];
  double lower = (2.0 * d - 6.0 + 4.0 * ss) / (3.0 * d * (d - 1));
  for (int i = 0; i < d; ++i)
    for (int j = i + 1; j < d; ++j) {
      lower = std::fmax(lower, (std::fabs(sig[i] + sig[j]) - 2.0 * sig[i] * sig[j]) / 3.0);
      lower = std::fmax(lower, (std::fabs(sig[i] - sig[j]) + 2.0 * sig[i] * sig[j]) / 3.0);
    }
  double upper = INFINITY;
  for (int i = 0; i < d; ++i)
    upper = std::fmin(upper, (1.0 + 2.0 * sig[i] * sig[i] - std::fabs((4.0 - d) * sig[i])) / (3.0 * (d - 1)));
  return g * lower + (1.0 - g) * upper;
}

// Eq. (omega_k-2) (units c = 1, sigma = u/c) for per-pair fourth moments m4[p], p over i<j.
void weights(int d, const int32_t *e, int Q, const double *sig, const double *m4, double *omega) {
  int pidx[kMaxD][kMaxD] = {};
  int p = 0;
  double m4sum = 0.0, ss = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = i + 1; j < d; ++j) {
      pidx[i][j] = pidx[j][i] = p;
      m4sum += m4[p++];
    }
  for (int i = 0; i < d; ++i) ss += sig[i] * sig[i];
  for (int k = 0; k < Q; ++k) {
    int ax[2] = {-1, -1}, nz = 0;
    for (int i = 0; i < d; ++i)
      if (e[k * d + i]) ax[nz++] = i;
    if (nz == 0) {
      omega[k] = (3.0 - d - 2.0 * ss + 3.0 * m4sum) / 3.0;
    } else if (nz == 1) {
      const int i = ax[0];
      double row = 0.0;
      for (int j = 0; j < d; ++j)
        if (j != i) row += m4[pidx[i][j]];
      omega[k] = (e[k * d + i] * (4.0 - d) * sig[i] + 1.0 + 2.0 * sig[i] * sig[i] - 3.0 * row) / 6.0;
    } else {
      const int i = ax[0], j = ax[1];
      const double si = e[k * d + i], sj = e[k * d + j];
      omega[k] = (3.0 * m4[pidx[i][j]] + 2.0 * si * sj * sig[i] * sig[j] + si * sig[i] + sj * sig[j]) / 12.0;
    }
  }
}

struct Model {
  int Q = 0;
  double dx = 0, dt = 0, s = 0;
  double x0[kMaxD] = {};
  double m4[10] = {};
  double omega[kMaxQ] = {};
  int32_t e[kMaxQ * kMaxD] = {};
  bool stable = true;
};

lhe_status build_model(const lhe_lbm_params *p, Model &m, lhe_lbm *err_to) {
  if (!p) return fail(err_to, LHE_ERR_ARG, "params is NULL");
  const int d = p->d;
  if (d < 1 || d > kMaxD) return fail(err_to, LHE_ERR_ARG, "d must be in 1..5");
  if (p->bc < 0 || p->bc > 2) return fail(err_to, LHE_ERR_ARG, "bc must be LHE_BC_PERIODIC, LHE_BC_FULLWAY or LHE_BC_HALFWAY");
  if (p->precision != LHE_FP64 && p->precision != LHE_FP32_DEV) return fail(err_to, LHE_ERR_ARG, "unknown precision");
  if (p->init_order != 1 && p->init_order != 3) return fail(err_to, LHE_ERR_ARG, "init_order must be 1 or 3");
  if (p->bc == LHE_BC_FULLWAY && p->bc_order != 1 && p->bc_order != 3 && p->bc_order != 4)
    return fail(err_to, LHE_ERR_ARG, "full-way bc_order must be 1, 3 or 4");
  if (p->bc == LHE_BC_HALFWAY && (p->bc_order < 1 || p->bc_order > 4))
    return fail(err_to, LHE_ERR_ARG, "half-way bc_order must be 1..4");
  if (!(p->c > 0.0) || !std::isfinite(p->c)) return fail(err_to, LHE_ERR_ARG, "c must be positive");
  if (!(p->tau > 0.0) || !std::isfinite(p->tau)) return fail(err_to, LHE_ERR_ARG, "tau must be positive");
  if (p->flags & ~(LHE_FLAG_NO_STAGING | LHE_FLAG_NO_PDL | LHE_FLAG_TEST_EXPIRE_WAIT | LHE_FLAG_NODE_BOUNDARY))
    return fail(err_to, LHE_ERR_ARG, "unknown bits in flags");
  if (p->m4_mode != LHE_M4_RULE && p->m4_mode != LHE_M4_EXPLICIT) return fail(err_to, LHE_ERR_ARG, "unknown m4_mode");
  if (p->m4_mode == LHE_M4_RULE && !(p->g >= 0.0 && p->g <= 1.0)) return fail(err_to, LHE_ERR_ARG, "g must be in [0, 1]");
  double dxs[kMaxD];
  for (int i = 0; i < d; ++i) {
    if (p->n[i] < 3) return fail(err_to, LHE_ERR_ARG, "every n[i] must be >= 3");
    if (!(p->hi[i] > p->lo[i])) return fail(err_to, LHE_ERR_ARG, "every hi[i] must exceed lo[i]");
    if (!std::isfinite(p->u[i])) return fail(err_to, LHE_ERR_ARG, "u must be finite");
    const double span = (p->bc == LHE_BC_FULLWAY) ? (double)(p->n[i] - 1) : (double)p->n[i];
    dxs[i] = (p->hi[i] - p->lo[i]) / span;
  }
  for (int i = 1; i < d; ++i)
    if (std::fabs(dxs[i] - dxs[0]) > 1e-12 * dxs[0])
      return fail(err_to, LHE_ERR_ARG, "the lattice must be square: (hi-lo)/n (or /(n-1) for full-way) must agree in every dimension");
  if (!std::isfinite(p->R)) return fail(err_to, LHE_ERR_ARG, "R must be finite");
  m.dx = dxs[0];
  m.dt = m.dx / p->c;
  m.s = 1.0 / p->tau;
  for (int i = 0; i < d; ++i) m.x0[i] = p->lo[i] + (p->bc == LHE_BC_HALFWAY ? 0.5 * m.dx : 0.0);
  m.Q = lattice_vectors(d, m.e);
  double sig[kMaxD];
  for (int i = 0; i < d; ++i) sig[i] = p->u[i] / p->c;
  const int npairs = d * (d - 1) / 2;
  if (p->m4_mode == LHE_M4_RULE) {
    const double v = m4_rule(d, sig, p->g);
    for (int q = 0; q < npairs; ++q) m.m4[q] = v;
  } else {
    for (int q = 0; q < npairs; ++q) m.m4[q] = p->m4[q];
  }
  weights(d, m.e, m.Q, sig, m.m4, m.omega);
  m.stable = true;
  for (int k = 0; k < m.Q; ++k)
    if (!(m.omega[k] > 0.0)) m.stable = false;
  return LHE_OK;
}

Geom make_geom(int d, const int64_t *n) {
  Geom g;
  g.d = d;
  int64_t stride = 1, si = 1;
  for (int i = 0; i < d; ++i) {
    g.n[i] = (int32_t)n[i];
    g.stride[i] = (int32_t)stride;
    g.dv[i] = FastDiv((uint32_t)n[i]);
    g.dvi[i] = FastDiv((uint32_t)(n[i] - 2));
    stride *= n[i];
    si *= (n[i] - 2);
  }
  g.S = stride;
  g.S_interior = si;
  g.S_rows = d > 1 ? si / (n[0] - 2) * n[0] : n[0];
  return g;
}

size_t pop_bytes(const lhe_lbm *l) {
  return (size_t)l->Q * (size_t)l->g.S * (l->p.precision == LHE_FP64 ? sizeof(double) : sizeof(float));
}

StepArgs step_args(const lhe_lbm *l) {
  StepArgs a{};
  a.g = l->g;
  for (int k = 0; k < l->Q; ++k) {
    a.omega[k] = l->omega[k];
    a.omega_f[k] = (float)l->omega[k];
    a.dtwR_f[k] = (float)(l->dt * l->omega[k] * l->R);
  }
  a.s = l->s;
  a.oms = 1.0 - l->s;
  a.dtR = l->dt * l->R;
  a.dt = l->dt;
  a.half_dt = 0.5 * l->dt;
  a.Rfield = l->Rfield;
  a.collide = kCollideGeneral;
  a.mu = 1.0 - l->s;
  a.sig = l->s;
  a.rho_dt = a.dt;
  a.rho_dtR = a.dtR;
  a.gsc = a.dt;
  a.pscale = 1.0;
  a.pdl = 0;
  return a;
}

// ---- scaled representation of the FP64 state (s != 2, periodic boxes) ----
// With r = 1 - s the collision f*_k = r f_k + omega_k psi costs two FP64 operations per population,
// twice the s = 2 form. Storing G = K f* with K = r^-j after j consecutive scaled steps turns the
// step into
//   G*_k(x) = G_k(x - e_k) + omega_k Psi,   Psi = sig sum_k G_k + K' dt R,   sig = s/r, K' = K/r,
// one FMA per population and the same map up to rounding (the pulled term r f_k equals G_k / K').
// sig is one of the three doubles nearest to s/r, chosen every step so that the accumulated
// relative error of sig r against s stays within about one ulp (error feedback): a fixed rounded
// quotient would move the conserved mode by s times its rounding error on every step. Before K
// would pass 2^kScaleBits, one general step with mu = r^(j+1), sig = s r^j returns to K = 1.
constexpr double kScaleBits = 128.0;
constexpr double kMinScaledR = 1.0 / 64.0;

bool scaled_eligible(const lhe_lbm *l) {
  const double r = 1.0 - l->s;
  return l->p.bc == LHE_BC_PERIODIC && l->p.precision == LHE_FP64 && l->s != 2.0 && std::fabs(r) >= kMinScaledR &&
         std::fabs(r) <= 1.0 / kMinScaledR && std::fabs(r) != 1.0;
}

int scaled_run(const lhe_lbm *l) {  // longest run of scaled steps starting from K = 1
  const double b = std::fabs(std::log2(std::fabs(1.0 - l->s)));
  return b * 4096.0 <= kScaleBits ? 4096 : (int)std::floor(kScaleBits / b);
}

double pick_sig(double s, double r, double &acc) {
  const double c0 = s / r;
  const double cand[3] = {c0, std::nextafter(c0, -INFINITY), std::nextafter(c0, INFINITY)};
  double best = c0, best_err = std::fma(c0, r, -s) / s;
  for (double c : cand) {
    const double err = std::fma(c, r, -s) / s;  // relative error of c r against s
    if (std::fabs(acc + err) < std::fabs(acc + best_err)) {
      best = c;
      best_err = err;
    }
  }
  acc += best_err;
  return best;
}

// Collision constants of the next step of a scaled-eligible state ([0] forward, [1] adjoint).
void plan_scaled_step(lhe_lbm *l, int which, StepArgs &a) {
  const double s = l->s, r = 1.0 - s;
  int32_t &j = l->scale_j[which];
  const double rj = std::pow(r, (double)j);  // 1/K
  a.gsc = a.dt * rj;                          // adjoint: dt w = dt r^j sum_k Z_k
  if (j + 1 > scaled_run(l)) {
    a.collide = kCollideGeneral;
    a.mu = std::pow(r, (double)(j + 1));
    a.sig = s * rj;
    a.rho_dt = a.dt;
    a.rho_dtR = a.dtR;
    j = 0;
  } else {
    const double K1 = std::pow(r, -(double)(j + 1));
    a.collide = kCollideScaled;
    a.sig = pick_sig(s, r, l->scale_acc[which]);
    a.rho_dt = a.dt * K1;
    a.rho_dtR = a.dtR * K1;
    j += 1;
  }
}

// Returns a scaled state to f* in place (rounding once per population) and restarts the error
// feedback of sig.
lhe_status unscale(lhe_lbm *l, int which) {
  int32_t &j = l->scale_j[which];
  if (j == 0) return LHE_OK;
  double *p = static_cast<double *>(which == 0 ? l->pop[l->cur] : l->adj[l->acur]);
  LHE_CK(l, launch_scale_fp64(p, (int64_t)l->Q * l->g.S, std::pow(1.0 - l->s, (double)j), l->stream));
  j = 0;
  l->scale_acc[which] = 0.0;  // a state read out and set back continues exactly alike
  return LHE_OK;
}

// A staged step whose pipeline wait expired stops early and sets a host-mapped flag; the next step
// call reports it (the state is then incomplete).
lhe_status check_pipeline(lhe_lbm *l) {
  if (l->tma_err_host && *(volatile int32_t *)l->tma_err_host)
    return fail(l, LHE_ERR_CUDA, "a staged step kernel timed out waiting for its copies; the state is invalid "
                                 "(lhe_lbm_init or lhe_lbm_set_state starts a new one)");
  return LHE_OK;
}

// A new state (init, set_state) clears a reported pipeline failure: once the stream has drained the
// failed kernel, nothing can set the flag again.
lhe_status clear_pipeline(lhe_lbm *l) {
  if (l->tma_err_host && *(volatile int32_t *)l->tma_err_host) {
    LHE_CK(l, cudaStreamSynchronize(l->stream));
    *(volatile int32_t *)l->tma_err_host = 0;
  }
  return LHE_OK;
}

// The staged kernel's plan for the next launch; LHE_FLAG_TEST_EXPIRE_WAIT arms one launch whose compute
// warps give up their first unready wait.
DevTmaPlan staged_plan(lhe_lbm *l) {
  DevTmaPlan p = l->tma;
  if (l->tma_expire_armed) {
    p.consumer_wait_ns = 0;
    l->tma_expire_armed = false;
  }
  return p;
}

// Programmatic dependent launch between the consecutive step kernels of one step / adjoint_step call,
// and for the first step kernel of a call when the step kernels the library launched last (process-wide)
// were this handle's, on the same stream. The step kernels let their successor be scheduled as soon
// as all their CTAs run; a successor of another handle (another grid shape, another kernel) scheduled
// that early measured slower, so across calls only a handle's own step kernels chain this way. Work
// that the caller queued in between does not let the successor in early (it does not signal), and a
// successor always waits for its predecessor to complete, so the results are the same in every case.
bool pdl_ok(const lhe_lbm *l) { return !(l->p.flags & LHE_FLAG_NO_PDL); }

std::mutex g_last_steps_mu;
const lhe_lbm *g_last_steps_handle = nullptr;  // whose step kernels the library launched last
cudaStream_t g_last_steps_stream = nullptr;

bool continues_own_steps(const lhe_lbm *l) {
  std::lock_guard<std::mutex> lock(g_last_steps_mu);
  return g_last_steps_handle == l && g_last_steps_stream == l->stream;
}

void note_own_steps(const lhe_lbm *l) {
  std::lock_guard<std::mutex> lock(g_last_steps_mu);
  g_last_steps_handle = l;
  g_last_steps_stream = l->stream;
}

void forget_steps_of(const lhe_lbm *l) {
  std::lock_guard<std::mutex> lock(g_last_steps_mu);
  if (g_last_steps_handle == l) g_last_steps_handle = nullptr;
}

// The link k-bar with e_kbar = -e_k.
int opposite_link(const lhe_lbm *l, int k) {
  const int d = l->p.d;
  for (int j = 0; j < l->Q; ++j) {
    bool opp = true;
    for (int i = 0; i < d; ++i)
      if (l->e[j * d + i] != -l->e[k * d + i]) opp = false;
    if (opp) return j;
  }
  return -1;
}

lhe_status check_handle(lhe_lbm *l) {
  if (!l) return fail(nullptr, LHE_ERR_ARG, "handle is NULL");
  return LHE_OK;
}

}  // namespace

lhe_status lhe::record_error(lhe_status status, const std::string &msg) { return fail(nullptr, status, msg); }

extern "C" {

int32_t lhe_lbm_abi_version(void) { return LHE_ABI_VERSION; }
uint64_t lhe_lbm_params_size(void) { return sizeof(lhe_lbm_params); }

lhe_status lhe_lbm_default_params(lhe_lbm_params *p) {
  if (!p) return fail(nullptr, LHE_ERR_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->d = 3;
  p->bc = LHE_BC_PERIODIC;
  p->precision = LHE_FP64;
  p->init_order = 3;
  p->bc_order = 4;
  p->m4_mode = LHE_M4_RULE;
  for (int i = 0; i < LHE_MAX_DIM; ++i) {
    p->n[i] = 16;
    p->lo[i] = 0.0;
    p->hi[i] = 1.0;
  }
  p->c = 1.0;
  p->tau = 0.5;
  p->g = 0.5;
  return LHE_OK;
}

lhe_status lhe_lbm_model(const lhe_lbm_params *p, double *omega_host, double *m4_host, int32_t *e_host,
                         int32_t *Q_out) {
  Model m;
  const lhe_status st = build_model(p, m, nullptr);
  if (st != LHE_OK) return st;
  if (omega_host) std::memcpy(omega_host, m.omega, sizeof(double) * m.Q);
  if (m4_host) std::memcpy(m4_host, m.m4, sizeof(double) * (p->d * (p->d - 1) / 2));
  if (e_host) std::memcpy(e_host, m.e, sizeof(int32_t) * m.Q * p->d);
  if (Q_out) *Q_out = m.Q;
  if (!m.stable) return fail(nullptr, LHE_ERR_UNSTABLE, "some EDF weight omega_k <= 0: the fourth moments violate the entropy-stability conditions (Proposition 1)");
  return LHE_OK;
}

lhe_status lhe_lbm_create(const lhe_lbm_params *p, lhe_lbm **out) {
  if (!out) return fail(nullptr, LHE_ERR_ARG, "out is NULL");
  *out = nullptr;
  Model m;
  lhe_status st = build_model(p, m, nullptr);
  if (st != LHE_OK) return st;
  if (!m.stable && !p->allow_unstable)
    return fail(nullptr, LHE_ERR_UNSTABLE, "some EDF weight omega_k <= 0: not entropy stable (Proposition 1); set allow_unstable to proceed");
  int64_t S = 1;
  for (int i = 0; i < p->d; ++i) {
    if (p->n[i] > (int64_t)INT32_MAX) return fail(nullptr, LHE_ERR_ARG, "n[i] too large");
    S *= p->n[i];
    if (S > (int64_t)INT32_MAX) return fail(nullptr, LHE_ERR_ARG, "the lattice has more than 2^31-1 nodes");
  }
  lhe_lbm *l = new (std::nothrow) lhe_lbm();
  if (!l) return fail(nullptr, LHE_ERR_OOM, "host allocation failed");
  l->p = *p;
  l->Q = m.Q;
  l->dx = m.dx;
  l->dt = m.dt;
  l->s = m.s;
  l->R = p->R;
  std::memcpy(l->omega, m.omega, sizeof(m.omega));
  std::memcpy(l->m4, m.m4, sizeof(m.m4));
  std::memcpy(l->e, m.e, sizeof(m.e));
  std::memcpy(l->x0, m.x0, sizeof(m.x0));
  l->g = make_geom(p->d, p->n);
  l->stream = static_cast<cudaStream_t>(p->stream);
  auto bail = [&](lhe_status s2) {
    g_last_error = l->err;
    lhe_lbm_destroy(l);
    return s2;
  };
  const size_t pb = pop_bytes(l);
  for (int b = 0; b < 2; ++b) {
    cudaError_t e = cudaMalloc(&l->pop[b], pb);
    if (e != cudaSuccess) return bail(cuda_fail(l, e, "cudaMalloc(populations)"));
    if (p->precision == LHE_FP32_DEV) {
      e = cudaMalloc(&l->phi[b], sizeof(float2) * (size_t)S);
      if (e != cudaSuccess) return bail(cuda_fail(l, e, "cudaMalloc(phi)"));
    }
  }
  l->red_blocks = 152 * 4;
  cudaError_t e = cudaMalloc(&l->red_partials, sizeof(double) * 4 * (size_t)l->red_blocks + sizeof(double) * 4);
  if (e != cudaSuccess) return bail(cuda_fail(l, e, "cudaMalloc(reduction scratch)"));
  l->red_out = l->red_partials + 4 * (size_t)l->red_blocks;
  if (p->bc != LHE_BC_PERIODIC) {
    // Boundary nodes grouped by face signature (per dimension: interior, low face or high face), so
    // that the threads of a warp share one set of unknown populations; site order within a group.
    std::vector<std::pair<int32_t, int32_t>> keyed;
    keyed.reserve((size_t)(S - l->g.S_interior));
    for (int64_t s = 0; s < S; ++s) {
      int64_t r = s;
      int32_t sig = 0, w3 = 1;
      for (int i = 0; i < p->d; ++i) {
        const int64_t xi = r % p->n[i];
        r /= p->n[i];
        sig += w3 * (xi == 0 ? 1 : (xi == p->n[i] - 1 ? 2 : 0));
        w3 *= 3;
      }
      if (sig) keyed.emplace_back(sig, (int32_t)s);
    }
    std::sort(keyed.begin(), keyed.end());
    std::vector<int32_t> sites(keyed.size());
    l->nb_xface = 0;
    for (size_t j = 0; j < keyed.size(); ++j) {
      sites[j] = keyed[j].second;
      if (keyed[j].first <= 2) ++l->nb_xface;  // signatures 1 and 2 (x_1 face only) sort first
    }
    l->nb = (int64_t)sites.size();
    // records of boundary data given as jets: one per (boundary node, unknown link), in node order
    l->bsites_host = sites;
    l->broff_host.resize(sites.size());
    int64_t nrec = 0;
    for (size_t j = 0; j < sites.size(); ++j) {
      l->broff_host[j] = (int32_t)nrec;
      int32_t w = keyed[j].first;
      int unknown_links = 0;
      for (int k = 0; k < m.Q; ++k) {
        bool unknown = false;
        int32_t ws = w;
        for (int i = 0; i < p->d; ++i, ws /= 3) {
          const int e_ki = m.e[k * p->d + i];
          if ((ws % 3 == 1 && e_ki == 1) || (ws % 3 == 2 && e_ki == -1)) unknown = true;
        }
        unknown_links += unknown ? 1 : 0;
      }
      nrec += unknown_links;
      if (nrec > 0x7fffffff) return bail(fail(l, LHE_ERR_ARG, "too many boundary records"));
    }
    l->nrec = nrec;
    if (p->precision == LHE_FP64) {
      const int64_t nrows = l->g.S_rows / l->g.n[0];
      e = cudaMalloc(&l->xface, sizeof(double) * (size_t)(2 * nrows * (2 * p->d - 1)));
      if (e != cudaSuccess) return bail(cuda_fail(l, e, "cudaMalloc(x-face boundary data)"));
      if (!(p->flags & LHE_FLAG_NODE_BOUNDARY)) {
        // the step's boundary data: the entries (unknown link k of boundary node x) whose link leaves
        // through a face of x_2..x_d, sorted by k then x, in a dense array shaped like the populations;
        // then those through an x_1 face only, sorted by x then k, compact per row end; with the record
        // (node-major, as broff) that feeds each
        struct Ent {
          int cls;
          long long key1, key2;
          int32_t rec;
          bool operator<(const Ent &o) const {
            return cls != o.cls ? cls < o.cls : (key1 != o.key1 ? key1 < o.key1 : key2 < o.key2);
          }
        };
        std::vector<Ent> ent;
        ent.reserve((size_t)nrec);
        for (size_t j = 0; j < sites.size(); ++j) {
          int32_t r = l->broff_host[j];
          for (int k = 0; k < m.Q; ++k) {
            bool row = false, xo = false;
            int32_t ws = keyed[j].first;
            for (int i = 0; i < p->d; ++i, ws /= 3) {
              const int e_ki = m.e[k * p->d + i];
              const bool out = (ws % 3 == 1 && e_ki == 1) || (ws % 3 == 2 && e_ki == -1);
              if (out && i > 0) row = true;
              if (out && i == 0) xo = true;
            }
            if (row) ent.push_back(Ent{0, k, sites[j], r++});
            else if (xo) ent.push_back(Ent{1, sites[j], k, r++});
          }
        }
        std::sort(ent.begin(), ent.end());
        l->nrow_ent = 0;
        while (l->nrow_ent < (int64_t)ent.size() && ent[(size_t)l->nrow_ent].cls == 0) ++l->nrow_ent;
        std::vector<long long> ek(ent.size()), ed(ent.size()), eo(ent.size());
        std::vector<int32_t> er(ent.size());  // record (node-major) -> entry
        const int J = 2 * p->d - 1;
        const int64_t n1 = p->n[0];
        for (size_t i = 0; i < ent.size(); ++i) {
          const long long k = ent[i].cls == 0 ? ent[i].key1 : ent[i].key2;
          const long long x = ent[i].cls == 0 ? ent[i].key2 : ent[i].key1;
          ek[i] = (k << 32) | x;
          er[(size_t)ent[i].rec] = (int32_t)i;
          int kb = 0, jx = 0;
          const int side = (x % n1) == 0 ? 1 : -1;
          for (int q = 0; q < m.Q; ++q) {
            bool opp = true;
            for (int dd = 0; dd < p->d; ++dd)
              if (m.e[q * p->d + dd] != -m.e[k * p->d + dd]) opp = false;
            if (opp) kb = q;
            if (q < k && m.e[q * p->d] == side) ++jx;
          }
          ed[i] = ent[i].cls == 0 ? k * S + x : (long long)m.Q * S + (2 * (x / n1) + (side > 0 ? 0 : 1)) * J + jx;
          eo[i] = (long long)kb * S + x;
        }
        int64_t nrows_all = 1;
        for (int i = 1; i < p->d; ++i) nrows_all *= p->n[i];
        e = cudaMalloc(&l->bdata, pop_bytes(l) + sizeof(double) * (size_t)nrows_all * 2 * J);
        if (e == cudaSuccess) e = cudaMalloc(&l->bdst, sizeof(long long) * std::max<size_t>(ed.size(), 1));
        if (e == cudaSuccess) e = cudaMalloc(&l->bopp, sizeof(long long) * std::max<size_t>(eo.size(), 1));
        if (e == cudaSuccess && !ed.empty())
          e = cudaMemcpy(l->bdst, ed.data(), sizeof(long long) * ed.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !eo.empty())
          e = cudaMemcpy(l->bopp, eo.data(), sizeof(long long) * eo.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&l->bent, sizeof(long long) * std::max<size_t>(ek.size(), 1));
        if (e == cudaSuccess) e = cudaMalloc(&l->bmap, sizeof(int32_t) * std::max<size_t>(er.size(), 1));
        if (e == cudaSuccess && !ek.empty())
          e = cudaMemcpy(l->bent, ek.data(), sizeof(long long) * ek.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !er.empty())
          e = cudaMemcpy(l->bmap, er.data(), sizeof(int32_t) * er.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(cuda_fail(l, e, "dense boundary data"));
      }
    }
    e = cudaMalloc(&l->bsites, sizeof(int32_t) * sites.size());
    if (e != cudaSuccess) return bail(cuda_fail(l, e, "cudaMalloc(boundary nodes)"));
    e = cudaMemcpy(l->bsites, sites.data(), sizeof(int32_t) * sites.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(cuda_fail(l, e, "cudaMemcpy(boundary nodes)"));
    e = cudaMalloc(&l->bc_table, sizeof(double) * ((size_t)kMaxModes * kMaxQ * 3 + kMaxModes));
    if (e != cudaSuccess) return bail(cuda_fail(l, e, "cudaMalloc(boundary table)"));
    int64_t sum_n = 0;
    for (int i = 0; i < p->d; ++i) sum_n += p->n[i];
    e = cudaMalloc(&l->bc_axis, sizeof(double) * 2 * (size_t)kMaxModes * (size_t)sum_n);
    if (e != cudaSuccess) return bail(cuda_fail(l, e, "cudaMalloc(boundary phase table)"));
  }
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l->sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (p->d == 3 && p->bc == LHE_BC_PERIODIC && p->precision == LHE_FP32_DEV && !(p->flags & LHE_FLAG_NO_STAGING)) {
    const int sms = l->sms;
    if (sms > 0 && plan_dev3_tma(l->g, sms, l->tma)) {
      e = cudaHostAlloc((void **)&l->tma_err_host, sizeof(int32_t), cudaHostAllocMapped);
      if (e != cudaSuccess) return bail(cuda_fail(l, e, "cudaHostAlloc(pipeline flag)"));
      *l->tma_err_host = 0;
      e = cudaHostGetDevicePointer((void **)&l->tma.err, l->tma_err_host, 0);
      if (e != cudaSuccess) return bail(cuda_fail(l, e, "cudaHostGetDevicePointer(pipeline flag)"));
      e = prepare_dev3_tma(l->tma);
      if (e != cudaSuccess) return bail(cuda_fail(l, e, "shared-memory size of the staged step"));
      l->staged = true;
      l->tma_expire_armed = (p->flags & LHE_FLAG_TEST_EXPIRE_WAIT) != 0;
    }
  }
  *out = l;
  return LHE_OK;
}

lhe_status lhe_lbm_destroy(lhe_lbm *l) {
  if (!l) return LHE_OK;
  forget_steps_of(l);
  cudaStreamSynchronize(l->stream);
  for (int b = 0; b < 2; ++b) {
    cudaFree(l->pop[b]);
    cudaFree(l->phi[b]);
    cudaFree(l->adj[b]);
    cudaFree(l->adjW[b]);
  }
  cudaFree(l->gR);
  cudaFree(l->Rfield);
  cudaFree(l->Rnext);
  cudaFree(l->fdgrad);
  cudaFree(l->bsites);
  cudaFree(l->broff);
  cudaFree(l->brec);
  cudaFree(l->sp_R0);
  cudaFree(l->sp_rec0);
  cudaFree(l->xface);
  cudaFree(l->bdata);
  cudaFree(l->bent);
  cudaFree(l->bmap);
  cudaFree(l->bdst);
  cudaFree(l->bopp);
  cudaFree(l->fsep);
  cudaFree(l->bc_table);
  cudaFree(l->bc_axis);
  cudaFree(l->red_partials);
  if (l->tma_err_host) cudaFreeHost(l->tma_err_host);
  delete l;
  return LHE_OK;
}

const char *lhe_lbm_last_error(const lhe_lbm *l) { return l ? l->err.c_str() : g_last_error.c_str(); }

lhe_status lhe_lbm_info(const lhe_lbm *l, lhe_lbm_info_t *info) {
  if (!l || !info) return fail(nullptr, LHE_ERR_ARG, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->d = l->p.d;
  info->Q = l->Q;
  info->S = l->g.S;
  info->n_boundary = l->nb;
  info->step = l->step;
  info->dx = l->dx;
  info->dt = l->dt;
  info->s = l->s;
  std::memcpy(info->m4, l->m4, sizeof(l->m4));
  std::memcpy(info->omega, l->omega, sizeof(double) * l->Q);
  std::memcpy(info->e, l->e, sizeof(int32_t) * l->Q * l->p.d);
  info->state_bytes = pop_bytes(l) + (l->p.precision == LHE_FP32_DEV ? sizeof(float2) * (size_t)l->g.S : 0);
  return LHE_OK;
}

lhe_status lhe_lbm_set_source(lhe_lbm *l, const double *Rf) {
  if (lhe_status s = check_handle(l)) return s;
  l->sp_mode = false;  // a caller's source ends the manufactured solution's
  if (Rf) {
    if (!l->Rnext) LHE_CK(l, cudaMalloc(&l->Rnext, sizeof(double) * (size_t)l->g.S));
    LHE_CK(l, cudaMemcpyAsync(l->Rnext, Rf, sizeof(double) * (size_t)l->g.S, cudaMemcpyDefault, l->stream));
    l->Rnext_state = 1;
  } else {
    l->Rnext_state = 2;
  }
  return LHE_OK;
}

namespace {
// The source set by lhe_lbm_set_source becomes the step's source when the step starts (the stored
// post-collision state keeps needing the source of its own collision until then: macro).
void activate_source(lhe_lbm *l) {
  if (l->Rnext_state == 1) {
    std::swap(l->Rfield, l->Rnext);
  } else if (l->Rnext_state == 2 && l->Rfield) {
    std::swap(l->Rfield, l->Rnext);  // keep the buffer for a later field
    l->Rfield = nullptr;
  }
  l->Rnext_state = 0;
}

// The source the next step will use.
const double *next_source(const lhe_lbm *l) {
  return l->Rnext_state == 1 ? l->Rnext : (l->Rnext_state == 2 ? nullptr : l->Rfield);
}
}  // namespace

lhe_status lhe_lbm_set_stream(lhe_lbm *l, void *stream) {
  if (lhe_status s = check_handle(l)) return s;
  l->stream = static_cast<cudaStream_t>(stream);
  return LHE_OK;
}

lhe_status lhe_lbm_init(lhe_lbm *l, const double *phi0, const double *grad, const double *Rf) {
  if (lhe_status s = check_handle(l)) return s;
  if (!phi0) return fail(l, LHE_ERR_ARG, "phi0 is NULL");
  const int d = l->p.d;
  const size_t S = (size_t)l->g.S;
  if (!grad && l->p.init_order == 3 && l->p.bc != LHE_BC_PERIODIC)
    return fail(l, LHE_ERR_ARG, "Dirichlet boxes need an explicit grad phi0 for the third-order initialisation");
  if (lhe_status st = clear_pipeline(l)) return st;
  l->Rnext_state = 0;
  if (Rf) {
    if (!l->Rfield) LHE_CK(l, cudaMalloc(&l->Rfield, sizeof(double) * S));
    LHE_CK(l, cudaMemcpyAsync(l->Rfield, Rf, sizeof(double) * S, cudaMemcpyDefault, l->stream));
  } else if (l->Rfield) {
    LHE_CK(l, cudaFree(l->Rfield));
    l->Rfield = nullptr;
  }
  const double *gptr = grad;
  l->grad_was_fd = false;
  if (!grad && l->p.init_order == 3) {
    if (!l->fdgrad) LHE_CK(l, cudaMalloc(&l->fdgrad, sizeof(double) * S * d));
    LHE_CK(l, launch_fd_grad(d, l->g, l->dx, phi0, l->fdgrad, l->stream));
    gptr = l->fdgrad;
    l->grad_was_fd = true;
  }
  InitArgs a{};
  a.g = l->g;
  a.phi0 = phi0;
  a.grad = gptr;
  a.Rfield = l->Rfield;
  a.dst = l->pop[0];
  a.phi_dst = l->phi[0];
  for (int k = 0; k < l->Q; ++k) {
    a.omega[k] = l->omega[k];
    a.c1[k] = (1.0 - l->s) * 0.5 * l->dt * l->omega[k];
    a.c2[k] = l->p.c * a.c1[k];
  }
  a.s = l->s;
  a.oms = 1.0 - l->s;
  a.dt = l->dt;
  a.dtR = l->dt * l->R;
  a.c = l->p.c;
  for (int i = 0; i < d; ++i) a.u[i] = l->p.u[i];
  a.order = l->p.init_order;
  l->init_order_used = l->p.init_order;
  LHE_CK(l, launch_init(d, l->p.precision == LHE_FP32_DEV, a, l->stream));
  l->cur = 0;
  l->step = 0;
  l->initialised = true;
  l->scale_j[0] = 0;
  l->scale_acc[0] = 0.0;
  l->adj_ready = false;
  return LHE_OK;
}

static BoundaryArgs boundary_args(const lhe_lbm *l);
static lhe_status ensure_jet_buffers(lhe_lbm *l);

lhe_status lhe_lbm_set_boundary_wave(lhe_lbm *l, const lhe_wave *w) {
  if (lhe_status s = check_handle(l)) return s;
  if (!w) return fail(l, LHE_ERR_ARG, "wave is NULL");
  if (l->p.bc == LHE_BC_PERIODIC) return fail(l, LHE_ERR_STATE, "boundary data on a periodic box");
  if (w->nmodes < 0 || w->nmodes > kMaxModes || w->reserved0 != 0) return fail(l, LHE_ERR_ARG, "nmodes must be in 0..16");
  const int d = l->p.d, Q = l->Q, M = w->nmodes, P = l->p.bc_order;
  const double dt = l->dt, dx = l->dx, c = l->p.c, R = l->R;
  // Per (mode, k) coefficients and per-k constants of the boundary schemes (see lhe_boundary.cu):
  //   full-way: f_k = omega_k [h - C_k - sum_m T_mk cos xi_m]
  //   half-way: f_k = wp_k lin + K_k + sum_m (U_mk sin xi_m + V_mk cos xi_m) - f*_kbar
  std::vector<double> tab((size_t)2 * M * Q + 2 * (size_t)Q, 0.0);
  double gu = 0.0;
  for (int i = 0; i < d; ++i) gu += w->g[i] * l->p.u[i];
  for (int k = 0; k < Q; ++k) {
    int kb = -1;
    for (int j = 0; j < Q; ++j) {
      bool opp = true;
      for (int i = 0; i < d; ++i)
        if (l->e[j * d + i] != -l->e[k * d + i]) opp = false;
      if (opp) kb = j;
    }
    double ge = 0.0;  // g . e_k
    for (int i = 0; i < d; ++i) ge += w->g[i] * l->e[k * d + i];
    const double wp = l->omega[k] + l->omega[kb], wm = l->omega[k] - l->omega[kb];
    double *kc = &tab[2 * (size_t)M * Q + 2 * (size_t)k];
    if (l->p.bc == LHE_BC_FULLWAY) {
      kc[0] = P >= 3 ? 0.5 * dt * (c * ge - gu) : 0.0;  // C_k: -(dt/2)(g.c_k + R - g.u) + (dt/2) R, over omega_k
    } else {
      kc[0] = wp;
      kc[1] = -wp * 0.5 * dx * ge + (P >= 2 ? wp * 0.5 * dt * (2.0 * R - gu) : 0.0);
    }
    for (int m = 0; m < M; ++m) {
      double ke = 0.0, ku = 0.0;
      for (int i = 0; i < d; ++i) {
        ke += w->kappa[m * LHE_MAX_DIM + i] * l->e[k * d + i];
        ku += w->kappa[m * LHE_MAX_DIM + i] * l->p.u[i];
      }
      const double A = c * ke, B = -ku, am = w->a[m];
      double *cf = &tab[2 * ((size_t)m * Q + k)];
      if (l->p.bc == LHE_BC_FULLWAY) {
        const double ab = A + B;
        double T = 0.0;
        if (P >= 3) T += 0.5 * dt * am * ab;
        if (P >= 4) T += dt * dt * dt / 24.0 * am * ab * ab * ab;
        cf[0] = T;
      } else {
        double Ps = wp, Qc = 0.0;  // coefficients of sin and cos at the mid-link point x_b
        if (P >= 2) Qc += wp * 0.5 * dt * B;
        if (P >= 3) Ps += wp * dt * dt / 8.0 * A * A + wm * dt * dt / 4.0 * A * B;
        if (P >= 4) Qc += wp * dt * dt * dt / 16.0 * A * A * B + wp * dt * dt * dt / 24.0 * B * B * B +
                          wm * dt * dt * dt / 8.0 * A * B * B;
        Ps *= am;
        Qc *= am;
        const double alpha = 0.5 * dx * ke;  // xi(x_b) = xi(x) - alpha
        cf[0] = Ps * std::cos(alpha) + Qc * std::sin(alpha);
        cf[1] = -Ps * std::sin(alpha) + Qc * std::cos(alpha);
      }
    }
  }
  // cos/sin of kappa_mi X_i for every mode, axis and node index: the phase of a node is the product
  // of its axis factors and the time factor exp(i (theta_m - kappa_m . u t)) of the step.
  int64_t sum_n = 0;
  for (int i = 0; i < d; ++i) sum_n += l->p.n[i];
  std::vector<double> ax((size_t)2 * w->nmodes * sum_n);
  for (int m = 0; m < w->nmodes; ++m) {
    int64_t off = 0;
    for (int i = 0; i < d; ++i) {
      for (int64_t j = 0; j < l->p.n[i]; ++j) {
        const double arg = w->kappa[m * LHE_MAX_DIM + i] * (l->x0[i] + (double)j * l->dx);
        ax[2 * ((size_t)m * sum_n + off + j) + 0] = std::cos(arg);
        ax[2 * ((size_t)m * sum_n + off + j) + 1] = std::sin(arg);
      }
      off += l->p.n[i];
    }
  }
  LHE_CK(l, cudaStreamSynchronize(l->stream));
  if (!tab.empty()) LHE_CK(l, cudaMemcpy(l->bc_table, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
  if (!ax.empty()) LHE_CK(l, cudaMemcpy(l->bc_axis, ax.data(), sizeof(double) * ax.size(), cudaMemcpyHostToDevice));
  l->wave = *w;
  l->have_wave = true;
  l->jet_mode = false;
  l->sp_mode = false;
  l->jet_ready = false;
  if (l->bdata) {
    // the family's data separated in time, per entry of the dense array
    const size_t len = (size_t)std::max<int64_t>(l->nrec, 1) * (1 + 2 * (size_t)M);
    if (len > l->fsep_len) {
      LHE_CK(l, cudaFree(l->fsep));
      l->fsep = nullptr;
      l->fsep_len = 0;
      LHE_CK(l, cudaMalloc(&l->fsep, sizeof(double) * len));
      l->fsep_len = len;
    }
    BoundaryArgs b = boundary_args(l);
    LHE_CK(l, launch_family_sep(d, l->p.bc, b, l->bent, l->nrec, l->fsep, l->stream));
  }
  return LHE_OK;
}


static BoundaryArgs boundary_args(const lhe_lbm *l) {
  BoundaryArgs b{};
  b.g = l->g;
  b.sites = l->bsites;
  b.nsites = l->nb;
  b.Rfield = l->Rfield;
  b.table = l->bc_table;
  b.axis = l->bc_axis;
  int32_t off = 0;
  for (int i = 0; i < l->p.d; ++i) {
    b.axis_off[i] = off;
    off += (int32_t)l->p.n[i];
  }
  b.axis_len = off;
  for (int k = 0; k < l->Q; ++k) {
    b.omega[k] = l->omega[k];
    for (int j = 0; j < l->Q; ++j) {
      bool opp = true;
      for (int i = 0; i < l->p.d; ++i)
        if (l->e[j * l->p.d + i] != -l->e[k * l->p.d + i]) opp = false;
      if (opp) {
        b.wratio[k] = l->omega[k] / l->omega[j];
        b.kbar[k] = (int8_t)j;
      }
    }
  }
  b.nrow_ent = l->nrow_ent;
  b.s = l->s;
  b.oms = 1.0 - l->s;
  b.R = l->R;
  b.dt = l->dt;
  b.dx = l->dx;
  b.c = l->p.c;
  for (int i = 0; i < l->p.d; ++i) {
    b.x0[i] = l->x0[i];
    b.u[i] = l->p.u[i];
  }
  b.order = l->p.bc_order;
  b.nmodes = l->wave.nmodes;
  b.b = l->wave.b;
  for (int i = 0; i < kMaxD; ++i) b.gl[i] = l->wave.g[i];
  for (int m = 0; m < kMaxModes; ++m) {
    b.a[m] = l->wave.a[m];
    b.theta[m] = l->wave.theta[m];
    for (int i = 0; i < kMaxD; ++i) b.kappa[m * kMaxD + i] = l->wave.kappa[m * LHE_MAX_DIM + i];
  }
  return b;
}

lhe_status lhe_lbm_boundary_points(const lhe_lbm *l, double *xyz_host, int64_t *P, double *t_offset) {
  if (!l) return fail(nullptr, LHE_ERR_ARG, "handle is NULL");
  lhe_lbm *lm = const_cast<lhe_lbm *>(l);
  if (!P) return fail(lm, LHE_ERR_ARG, "P is NULL");
  if (l->p.bc == LHE_BC_PERIODIC) return fail(lm, LHE_ERR_STATE, "boundary points of a periodic box");
  const int d = l->p.d;
  const bool full = l->p.bc == LHE_BC_FULLWAY;
  *P = full ? l->nb : l->nrec;
  if (t_offset) *t_offset = full ? l->dt : 0.0;
  if (!xyz_host) return LHE_OK;
  int64_t q = 0;
  for (size_t j = 0; j < l->bsites_host.size(); ++j) {
    int64_t r = l->bsites_host[j];
    int64_t idx[kMaxD];
    double x[kMaxD];
    for (int i = 0; i < d; ++i) {
      idx[i] = r % l->p.n[i];
      r /= l->p.n[i];
      x[i] = l->x0[i] + (double)idx[i] * l->dx;
    }
    if (full) {
      for (int i = 0; i < d; ++i) xyz_host[q * d + i] = x[i];
      ++q;
      continue;
    }
    for (int k = 0; k < l->Q; ++k) {  // half-way: the mid-link point x - e_k dx/2 of every unknown link
      bool unknown = false;
      for (int i = 0; i < d; ++i) {
        const int64_t src = idx[i] - l->e[k * d + i];
        if (src < 0 || src >= l->p.n[i]) unknown = true;
      }
      if (!unknown) continue;
      for (int i = 0; i < d; ++i) xyz_host[q * d + i] = x[i] - 0.5 * l->dx * l->e[k * d + i];
      ++q;
    }
  }
  return LHE_OK;
}

}  // extern "C"

// Position of each derivative in a boundary jet: orders 0..3, index tuples v1 <= .. <= vq in
// lexicographic order (v = 0: t, v = i: x_i); entries [a*36 + b*6 + c] (order 3) and [216 + a*6 + b]
// (order 2) list every ordering of a tuple.
static std::vector<int16_t> jet_index_table(int d) {
  std::vector<int16_t> jidx(216 + 36, 0);
  int16_t pos = (int16_t)(1 + (d + 1));
  for (int a = 0; a <= d; ++a)
    for (int b = a; b <= d; ++b) {
      jidx[216 + a * 6 + b] = pos;
      jidx[216 + b * 6 + a] = pos;
      ++pos;
    }
  for (int a = 0; a <= d; ++a)
    for (int b = a; b <= d; ++b)
      for (int c = b; c <= d; ++c) {
        const int perm[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
        for (const auto &q : perm) jidx[q[0] * 36 + q[1] * 6 + q[2]] = pos;
        ++pos;
      }
  return jidx;
}

// The per-node offsets of the unknown populations (device) and the record buffer, on first use.
static lhe_status ensure_jet_buffers(lhe_lbm *l) {
  if (l->broff) return LHE_OK;
  LHE_CK(l, cudaMalloc((void **)&l->broff, sizeof(int32_t) * l->broff_host.size()));
  LHE_CK(l, cudaMemcpy(l->broff, l->broff_host.data(), sizeof(int32_t) * l->broff_host.size(), cudaMemcpyHostToDevice));
  LHE_CK(l, cudaMalloc((void **)&l->brec, sizeof(double) * (size_t)std::max<int64_t>(l->nrec, 1)));
  return LHE_OK;
}

extern "C" {

lhe_status lhe_lbm_set_boundary_jet(lhe_lbm *l, const double *jet_dev) {
  if (lhe_status s = check_handle(l)) return s;
  if (l->p.bc == LHE_BC_PERIODIC) return fail(l, LHE_ERR_STATE, "boundary data on a periodic box");
  if (!jet_dev) return fail(l, LHE_ERR_ARG, "jet is NULL");
  if (lhe_status st = check_pipeline(l)) return st;
  if (lhe_status st = ensure_jet_buffers(l)) return st;
  BoundaryArgs b = boundary_args(l);
  b.roff = l->broff;  // the kernel writes l->brec; b.rec stays null (the data are being formed)
  b.rmap = l->bmap;   // in the order of the dense entries when the handle has them
  // the schemes' R terms (a source varying in time): full-way at the new time t_{n+1} (the source of
  // this step's collision), half-way at t_n (the source of the collision of f*_kbar)
  b.Rfield = l->p.bc == LHE_BC_FULLWAY ? next_source(l) : l->Rfield;
  LHE_CK(l, launch_jet_records(l->p.d, l->p.bc, b, jet_dev, jet_index_table(l->p.d).data(), l->brec, l->stream));
  l->jet_mode = true;
  l->jet_ready = true;
  l->sp_mode = false;
  return LHE_OK;
}

lhe_status lhe_lbm_set_boundary_sine_product(lhe_lbm *l, const lhe_sine_product *sp) {
  if (lhe_status s = check_handle(l)) return s;
  if (l->p.bc == LHE_BC_PERIODIC) return fail(l, LHE_ERR_STATE, "boundary data on a periodic box");
  if (!sp) return fail(l, LHE_ERR_ARG, "sine product is NULL");
  const int d = l->p.d;
  bool finite = std::isfinite(sp->A) && std::isfinite(sp->lambda);
  for (int i = 0; i < d; ++i) finite = finite && std::isfinite(sp->kappa[i]) && std::isfinite(sp->theta[i]);
  if (!finite) return fail(l, LHE_ERR_ARG, "sine product parameters must be finite");
  if (lhe_status st = check_pipeline(l)) return st;
  if (lhe_status st = ensure_jet_buffers(l)) return st;
  int64_t P = 0;
  if (lhe_status st = lhe_lbm_boundary_points(l, nullptr, &P, nullptr)) return st;
  std::vector<double> pts((size_t)std::max<int64_t>(P, 1) * d);
  if (lhe_status st = lhe_lbm_boundary_points(l, pts.data(), &P, nullptr)) return st;
  // count of each variable (0: t, i: x_i) in every jet entry, in the jet order
  std::vector<int8_t> tup;
  for (int q = 0; q <= 3; ++q) {
    int v[3] = {0, 0, 0};
    for (;;) {
      int8_t cnt[6] = {0, 0, 0, 0, 0, 0};
      for (int j = 0; j < q; ++j) ++cnt[v[j]];
      tup.insert(tup.end(), cnt, cnt + 6);
      int j = q - 1;  // next non-decreasing tuple
      while (j >= 0 && v[j] == d) --j;
      if (j < 0) break;
      ++v[j];
      for (int m = j + 1; m < q; ++m) v[m] = v[j];
    }
  }
  const int64_t JL = LHE_JET_LEN(d);
  if ((int64_t)tup.size() != JL * 6) return fail(l, LHE_ERR_ARG, "jet table");
  SineProductArgs a{};
  a.A = sp->A;
  a.lambda = sp->lambda;
  for (int i = 0; i < d; ++i) {
    a.kappa[i] = sp->kappa[i];
    a.theta[i] = sp->theta[i];
    a.u[i] = l->p.u[i];
    a.x0[i] = l->x0[i];
  }
  a.dx = l->dx;
  const size_t S = (size_t)l->g.S;
  if (!l->sp_R0) LHE_CK(l, cudaMalloc(&l->sp_R0, sizeof(double) * S));
  if (!l->sp_rec0) LHE_CK(l, cudaMalloc(&l->sp_rec0, sizeof(double) * (size_t)std::max<int64_t>(l->nrec, 1)));
  if (!l->Rnext) LHE_CK(l, cudaMalloc(&l->Rnext, sizeof(double) * S));
  double *dpts = nullptr, *djet = nullptr;
  int8_t *dtup = nullptr;
  auto release = [&]() {
    cudaFree(dpts);
    cudaFree(djet);
    cudaFree(dtup);
  };
  cudaError_t e = cudaMalloc(&dpts, sizeof(double) * pts.size());
  if (e == cudaSuccess) e = cudaMalloc(&djet, sizeof(double) * (size_t)std::max<int64_t>(P, 1) * JL);
  if (e == cudaSuccess) e = cudaMalloc(&dtup, tup.size());
  if (e == cudaSuccess) e = cudaMemcpy(dpts, pts.data(), sizeof(double) * pts.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dtup, tup.data(), tup.size(), cudaMemcpyHostToDevice);
  // jets of the solution at unit time factor, its source field R0, and the records they give
  if (e == cudaSuccess) e = launch_sp_jets(d, a, dpts, P, dtup, djet, l->stream);
  if (e == cudaSuccess) e = launch_sp_source(a, l->g, l->sp_R0, l->stream);
  if (e == cudaSuccess) {
    BoundaryArgs b = boundary_args(l);
    b.roff = l->broff;
    b.rmap = l->bmap;
    b.Rfield = l->sp_R0;  // data and source share the time factor in both schemes
    e = launch_jet_records(d, l->p.bc, b, djet, jet_index_table(d).data(), l->sp_rec0, l->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(l->stream);
  release();
  if (e != cudaSuccess) return cuda_fail(l, e, "sine-product boundary data");
  l->sp_mode = true;
  l->sp_lambda = sp->lambda;
  l->jet_mode = true;
  l->jet_ready = false;
  l->Rnext_state = 0;
  return LHE_OK;
}

lhe_status lhe_lbm_adjoint_jet_grad(lhe_lbm *l, double *out) {
  if (lhe_status s = check_handle(l)) return s;
  if (l->p.bc == LHE_BC_PERIODIC) return fail(l, LHE_ERR_STATE, "boundary jets on a periodic box");
  if (!out) return fail(l, LHE_ERR_ARG, "dL/djet is NULL");
  if (!l->adj_ready) return fail(l, LHE_ERR_STATE, "lhe_lbm_adjoint_jet_grad before lhe_lbm_adjoint_seed");
  if (lhe_status st = check_pipeline(l)) return st;
  if (lhe_status st = ensure_jet_buffers(l)) return st;
  BoundaryArgs b = boundary_args(l);
  b.roff = l->broff;
  b.src = l->adj[l->acur];
  b.phi_src = l->adjW[l->acur];
  LHE_CK(l, launch_jet_grad(l->p.d, l->p.bc, l->p.precision == LHE_FP32_DEV, b, jet_index_table(l->p.d).data(), out,
                            l->stream));
  return LHE_OK;
}

lhe_status lhe_lbm_step(lhe_lbm *l, int64_t n) {
  if (lhe_status s = check_handle(l)) return s;
  if (n < 0) return fail(l, LHE_ERR_ARG, "n must be >= 0");
  if (!l->initialised) return fail(l, LHE_ERR_STATE, "lhe_lbm_step before lhe_lbm_init");
  if (lhe_status st = check_pipeline(l)) return st;
  const bool periodic = l->p.bc == LHE_BC_PERIODIC;
  if (!periodic && !l->have_wave && !l->jet_mode)
    return fail(l, LHE_ERR_STATE, "Dirichlet box without boundary data (lhe_lbm_set_boundary_wave or _jet)");
  if (!periodic && next_source(l) && !l->jet_mode && n > 0)
    return fail(l, LHE_ERR_STATE, "a per-site source on a Dirichlet box needs the boundary data as jets "
                                  "(the exact-solution family assumes a constant R)");
  if (!periodic && l->jet_mode && !l->sp_mode && n > 0) {
    if (n != 1) return fail(l, LHE_ERR_STATE, "boundary jets hold one step's data: step n = 1 at a time");
    if (!l->jet_ready) return fail(l, LHE_ERR_STATE, "set the boundary jets of this step first (lhe_lbm_set_boundary_jet)");
  }
  const int d = l->p.d;
  const bool dev = l->p.precision == LHE_FP32_DEV;
  if (n > 0) activate_source(l);
  StepArgs a = step_args(l);
  BoundaryArgs b{};
  if (!periodic) b = boundary_args(l);
  const bool scaled = scaled_eligible(l);
  const bool chained = n > 0 && pdl_ok(l) && continues_own_steps(l);
  if (n > 0) note_own_steps(l);
  for (int64_t it = 0; it < n; ++it) {
    if (scaled) plan_scaled_step(l, 0, a);
    a.src = l->pop[l->cur];
    a.dst = l->pop[1 - l->cur];
    a.phi_src = l->phi[l->cur];
    a.phi_dst = l->phi[1 - l->cur];
    a.nwork = periodic ? l->g.S : l->g.S_rows;
    a.pdl = (it > 0 || chained) && pdl_ok(l);
    if (!periodic) {
      b.src = a.src;
      b.dst = a.dst;
      b.phi_src = a.phi_src;
      b.phi_dst = a.phi_dst;
      b.t_eval = (double)(l->p.bc == LHE_BC_FULLWAY ? l->step + 1 : l->step) * l->dt;
      for (int m = 0; m < l->wave.nmodes; ++m) {
        double ph = l->wave.theta[m];
        for (int i = 0; i < d; ++i) ph -= l->wave.kappa[m * LHE_MAX_DIM + i] * l->p.u[i] * b.t_eval;
        b.ph_c[m] = std::cos(ph);
        b.ph_s[m] = std::sin(ph);
      }
    }
    double rec_scale = 1.0;
    if (l->sp_mode) {
      // the manufactured solution: its source at t_{n+1} (this step's collision) and its records at the
      // time of the step's data, both the unit-factor fields times exp(-lambda t)
      if (!l->Rnext) LHE_CK(l, cudaMalloc(&l->Rnext, sizeof(double) * (size_t)l->g.S));
      cudaError_t e0 = launch_scale_field(l->sp_R0, std::exp(-l->sp_lambda * (double)(l->step + 1) * l->dt), l->g.S, l->Rnext,
                              l->sms, l->stream);
      if (e0 != cudaSuccess) return cuda_fail(l, e0, "source kernel launch");
      std::swap(l->Rfield, l->Rnext);
      a.Rfield = l->Rfield;
      b.Rfield = l->Rfield;
      rec_scale = std::exp(-l->sp_lambda * (double)(l->p.bc == LHE_BC_FULLWAY ? l->step + 1 : l->step) * l->dt);
    }
    // boundary data of the step: the exact-solution family, or records (jets, the manufactured solution)
    BoundaryArgs rest = b;
    if (!periodic) {
      if (l->sp_mode) {
        rest.roff = l->broff;
        rest.rec = l->sp_rec0;
        rest.rec_scale = rec_scale;
      } else if (l->jet_mode) {
        rest.roff = l->broff;
        rest.rec = l->brec;
        l->jet_ready = false;
      }
    }
    // FP64 Dirichlet boxes: the whole box as rows with dense boundary data (default), or the interior
    // rows with their x_1-face nodes and then the other boundary nodes one by one (LHE_FLAG_NODE_BOUNDARY)
    const bool dense = !periodic && !dev && l->bdata;
    const bool fused = !periodic && !dev && l->xface && !dense;
    cudaError_t e = cudaSuccess;
    if (dense) {
      // this step's unknown populations into the dense array, then the whole box
      if (!rest.rec) {
        // the exact-solution family: this step's term linear in t_eval per link
        double gu = 0.0;
        for (int i = 0; i < d; ++i) gu += l->wave.g[i] * l->p.u[i];
        for (int k = 0; k < l->Q; ++k) {
          const double wk = l->p.bc == LHE_BC_FULLWAY ? l->omega[k] : l->omega[k] + l->omega[opposite_link(l, k)];
          rest.lt[k] = wk * (l->R - gu) * rest.t_eval;
        }
      }
      e = launch_bdata_step(l->p.bc, rest.rec != nullptr, rest, l->bent, l->bdst, l->bopp, l->nrec,
                            rest.rec ? rest.rec : l->fsep, l->bdata, l->stream);
      if (e != cudaSuccess) return cuda_fail(l, e, "boundary data kernel launch");
      e = launch_step_box_dense(d, a, l->bdata, l->stream);
      if (e != cudaSuccess) return cuda_fail(l, e, "step kernel launch");
    } else {
      e = l->staged ? launch_step_dev3_tma(false, a, staged_plan(l), l->stream)
          : fused   ? launch_step_box_fp64(d, l->p.bc, a, rest, l->xface, l->g.S_rows / l->g.n[0], l->stream)
          : dev     ? launch_step_dev(d, false, !periodic, a, l->stream)
                    : launch_step_fp64(d, false, !periodic, a, l->stream);
      if (e != cudaSuccess) return cuda_fail(l, e, "step kernel launch");
      if (!periodic) {
        if (fused) {  // the x_1-face-only nodes lead the list and are done
          rest.sites = b.sites + l->nb_xface;
          rest.nsites = b.nsites - l->nb_xface;
          if (rest.roff) rest.roff += l->nb_xface;
        }
        e = launch_boundary(d, l->p.bc, dev, rest, l->stream);
        if (e != cudaSuccess) return cuda_fail(l, e, "boundary kernel launch");
      }
    }
    l->cur ^= 1;
    l->step += 1;
  }
  return LHE_OK;
}

lhe_status lhe_lbm_macro(lhe_lbm *l, double *phi_out) {
  if (lhe_status s = check_handle(l)) return s;
  if (!phi_out) return fail(l, LHE_ERR_ARG, "phi_out is NULL");
  if (!l->initialised) return fail(l, LHE_ERR_STATE, "lhe_lbm_macro before lhe_lbm_init");
  if (lhe_status st = check_pipeline(l)) return st;
  if (l->p.precision == LHE_FP32_DEV) {
    LHE_CK(l, launch_df_to_double(l->phi[l->cur], phi_out, l->g.S, l->stream));
    return LHE_OK;
  }
  StepArgs a = step_args(l);
  a.src = l->pop[l->cur];
  if (l->scale_j[0] != 0) a.pscale = std::pow(1.0 - l->s, (double)l->scale_j[0]);
  LHE_CK(l, launch_macro_fp64(l->p.d, a, phi_out, l->stream));
  return LHE_OK;
}

lhe_status lhe_lbm_diagnostics(lhe_lbm *l, double *out_host) {
  if (lhe_status s = check_handle(l)) return s;
  if (!out_host) return fail(l, LHE_ERR_ARG, "out_host is NULL");
  if (!l->initialised) return fail(l, LHE_ERR_STATE, "lhe_lbm_diagnostics before lhe_lbm_init");
  if (lhe_status st = unscale(l, 0)) return st;
  ReduceArgs a{};
  a.g = l->g;
  a.pop = l->pop[l->cur];
  a.phi = l->phi[l->cur];
  a.Rfield = l->Rfield;
  for (int k = 0; k < l->Q; ++k) a.omega[k] = l->omega[k];
  a.s = l->s;
  a.dt = l->dt;
  a.dtR = l->dt * l->R;
  a.partials = l->red_partials;
  a.out = l->red_out;
  LHE_CK(l, launch_reduce(l->p.d, l->p.precision == LHE_FP32_DEV, a, l->red_blocks, l->stream));
  LHE_CK(l, cudaMemcpyAsync(out_host, l->red_out, sizeof(double) * 4, cudaMemcpyDeviceToHost, l->stream));
  LHE_CK(l, cudaStreamSynchronize(l->stream));
  if (lhe_status st = check_pipeline(l)) return st;  // the stream has drained: a failure is visible now
  if (out_host[3] > 0.0) return fail(l, LHE_ERR_NONFINITE, "non-finite values in the state");
  return LHE_OK;
}

lhe_status lhe_lbm_get_state(lhe_lbm *l, void *buf) {
  if (lhe_status s = check_handle(l)) return s;
  if (!buf) return fail(l, LHE_ERR_ARG, "buf is NULL");
  if (!l->initialised) return fail(l, LHE_ERR_STATE, "no state before lhe_lbm_init");
  if (lhe_status st = unscale(l, 0)) return st;
  const size_t pb = pop_bytes(l);
  LHE_CK(l, cudaMemcpyAsync(buf, l->pop[l->cur], pb, cudaMemcpyDefault, l->stream));
  if (l->p.precision == LHE_FP32_DEV)
    LHE_CK(l, cudaMemcpyAsync(static_cast<char *>(buf) + pb, l->phi[l->cur], sizeof(float2) * (size_t)l->g.S,
                              cudaMemcpyDefault, l->stream));
  return LHE_OK;
}

lhe_status lhe_lbm_set_state(lhe_lbm *l, const void *buf, int64_t step) {
  if (lhe_status s = check_handle(l)) return s;
  if (!buf) return fail(l, LHE_ERR_ARG, "buf is NULL");
  if (step < 0) return fail(l, LHE_ERR_ARG, "step must be >= 0");
  if (lhe_status st = clear_pipeline(l)) return st;
  const size_t pb = pop_bytes(l);
  LHE_CK(l, cudaMemcpyAsync(l->pop[l->cur], buf, pb, cudaMemcpyDefault, l->stream));
  if (l->p.precision == LHE_FP32_DEV)
    LHE_CK(l, cudaMemcpyAsync(l->phi[l->cur], static_cast<const char *>(buf) + pb, sizeof(float2) * (size_t)l->g.S,
                              cudaMemcpyDefault, l->stream));
  l->step = step;
  l->initialised = true;
  l->scale_j[0] = 0;
  l->scale_acc[0] = 0.0;
  if (l->sp_mode) {
    // the manufactured solution's source of the restored state's last collision, R(x, t_step)
    if (!l->Rfield) LHE_CK(l, cudaMalloc(&l->Rfield, sizeof(double) * (size_t)l->g.S));
    LHE_CK(l, launch_scale_field(l->sp_R0, std::exp(-l->sp_lambda * (double)step * l->dt), l->g.S, l->Rfield, l->sms,
                                 l->stream));
  }
  return LHE_OK;
}

lhe_status lhe_lbm_adjoint_seed(lhe_lbm *l, const double *seed) {
  if (lhe_status s = check_handle(l)) return s;
  if (!seed) return fail(l, LHE_ERR_ARG, "dL/dphi_T is NULL");
  if (!l->initialised) return fail(l, LHE_ERR_STATE, "lhe_lbm_adjoint_seed before lhe_lbm_init");
  const bool dev = l->p.precision == LHE_FP32_DEV;
  const size_t S = (size_t)l->g.S;
  if (!l->adj[0]) {
    for (int b = 0; b < 2; ++b) {
      LHE_CK(l, cudaMalloc(&l->adj[b], pop_bytes(l)));
      if (dev) LHE_CK(l, cudaMalloc(&l->adjW[b], sizeof(float2) * S));
    }
    LHE_CK(l, cudaMalloc(&l->gR, sizeof(double) * S));
  }
  LHE_CK(l, launch_adjoint_seed(l->p.d, dev, l->g, l->omega, seed, l->adj[0], l->adjW[0], l->gR, l->stream));
  l->acur = 0;
  l->adj_ready = true;
  l->scale_j[1] = 0;
  l->scale_acc[1] = 0.0;
  return LHE_OK;
}

lhe_status lhe_lbm_adjoint_step(lhe_lbm *l, int64_t n) {
  if (lhe_status s = check_handle(l)) return s;
  if (n < 0) return fail(l, LHE_ERR_ARG, "n must be >= 0");
  if (!l->adj_ready) return fail(l, LHE_ERR_STATE, "lhe_lbm_adjoint_step before lhe_lbm_adjoint_seed");
  if (lhe_status st = check_pipeline(l)) return st;
  const bool dev = l->p.precision == LHE_FP32_DEV;
  StepArgs a = step_args(l);
  const bool periodic = l->p.bc == LHE_BC_PERIODIC;
  a.Rfield = nullptr;
  a.gR = periodic ? l->gR : nullptr;  // Dirichlet boxes: constant R only, no dL/dR(x)
  a.nwork = periodic ? l->g.S : l->g.S_rows;
  BoundaryArgs b{};
  if (!periodic) b = boundary_args(l);
  const bool scaled = scaled_eligible(l);
  const bool chained = n > 0 && pdl_ok(l) && continues_own_steps(l);
  if (n > 0) note_own_steps(l);
  for (int64_t it = 0; it < n; ++it) {
    if (scaled) plan_scaled_step(l, 1, a);
    a.src = l->adj[l->acur];
    a.dst = l->adj[1 - l->acur];
    a.phi_src = l->adjW[l->acur];
    a.phi_dst = l->adjW[1 - l->acur];
    a.pdl = (it > 0 || chained) && pdl_ok(l);
    cudaError_t e = l->staged ? launch_step_dev3_tma(true, a, staged_plan(l), l->stream)
                    : dev         ? launch_step_dev(l->p.d, true, !periodic, a, l->stream)
                                  : launch_step_fp64(l->p.d, true, !periodic, a, l->stream);
    if (e != cudaSuccess) return cuda_fail(l, e, "adjoint step kernel launch");
    if (!periodic) {
      b.src = a.src;
      b.dst = a.dst;
      b.phi_src = a.phi_src;
      b.phi_dst = a.phi_dst;
      e = launch_adjoint_boundary(l->p.d, l->p.bc, dev, b, l->stream);
      if (e != cudaSuccess) return cuda_fail(l, e, "adjoint boundary kernel launch");
    }
    l->acur ^= 1;
  }
  return LHE_OK;
}

lhe_status lhe_lbm_stability_map(const lhe_lbm_params *p, const double *sigma, int64_t npoints, int32_t nxi,
                                 double *rho_max, double *omega_min) {
  if (!p || (npoints > 0 && (!sigma || !rho_max || !omega_min))) return fail(nullptr, LHE_ERR_ARG, "NULL argument");
  const int d = p->d;
  if (d < 1 || d > 4) return fail(nullptr, LHE_ERR_ARG, "stability maps take d = 1..4");
  if (npoints < 0) return fail(nullptr, LHE_ERR_ARG, "npoints must be >= 0");
  if (nxi < 1 || nxi > 4096) return fail(nullptr, LHE_ERR_ARG, "nxi must be in 1..4096");
  int64_t nper = 1;
  for (int i = 0; i < d; ++i) nper *= nxi;
  if (npoints > 0 && nper > ((int64_t)1 << 40) / npoints) return fail(nullptr, LHE_ERR_ARG, "npoints * nxi^d is too large");
  if (!(p->tau > 0.0) || !std::isfinite(p->tau)) return fail(nullptr, LHE_ERR_ARG, "tau must be positive");
  if (p->m4_mode != LHE_M4_RULE && p->m4_mode != LHE_M4_EXPLICIT) return fail(nullptr, LHE_ERR_ARG, "unknown m4_mode");
  if (p->m4_mode == LHE_M4_RULE && !(p->g >= 0.0 && p->g <= 1.0)) return fail(nullptr, LHE_ERR_ARG, "g must be in [0, 1]");
  if (npoints == 0) return LHE_OK;
  int32_t e[kMaxQ * kMaxD];
  const int Q = lattice_vectors(d, e);
  const int npairs = d * (d - 1) / 2;
  std::vector<double> om((size_t)npoints * Q);
  for (int64_t q = 0; q < npoints; ++q) {
    double sig[kMaxD], m4[10] = {};
    for (int i = 0; i < d; ++i) {
      sig[i] = sigma[q * d + i];
      if (!std::isfinite(sig[i])) return fail(nullptr, LHE_ERR_ARG, "sigma must be finite");
    }
    for (int k = 0; k < npairs; ++k) m4[k] = p->m4_mode == LHE_M4_RULE ? m4_rule(d, sig, p->g) : p->m4[k];
    weights(d, e, Q, sig, m4, &om[(size_t)q * Q]);
    double mn = om[(size_t)q * Q];
    for (int k = 1; k < Q; ++k) mn = std::fmin(mn, om[(size_t)q * Q + k]);
    omega_min[q] = mn;
  }
  cudaStream_t st = static_cast<cudaStream_t>(p->stream);
  double *dom = nullptr;
  unsigned long long *drho = nullptr;
  auto release = [&]() {
    cudaFree(dom);
    cudaFree(drho);
  };
  cudaError_t e1 = cudaMalloc(&dom, sizeof(double) * om.size());
  if (e1 == cudaSuccess) e1 = cudaMalloc(&drho, sizeof(unsigned long long) * (size_t)npoints);
  if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(dom, om.data(), sizeof(double) * om.size(), cudaMemcpyHostToDevice, st);
  if (e1 == cudaSuccess) e1 = cudaMemsetAsync(drho, 0, sizeof(unsigned long long) * (size_t)npoints, st);
  if (e1 == cudaSuccess) e1 = launch_stability(d, dom, npoints, nxi, 1.0 / p->tau, drho, st);
  std::vector<unsigned long long> bits((size_t)npoints);
  if (e1 == cudaSuccess)
    e1 = cudaMemcpyAsync(bits.data(), drho, sizeof(unsigned long long) * bits.size(), cudaMemcpyDeviceToHost, st);
  if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(st);
  release();
  if (e1 != cudaSuccess) return cuda_fail(nullptr, e1, "stability map");
  for (int64_t q = 0; q < npoints; ++q) std::memcpy(&rho_max[q], &bits[(size_t)q], sizeof(double));
  return LHE_OK;
}

lhe_status lhe_lbm_adjoint_grads(lhe_lbm *l, double *gphi0, double *ggrad, double *gR) {
  if (lhe_status s = check_handle(l)) return s;
  if (!l->adj_ready) return fail(l, LHE_ERR_STATE, "lhe_lbm_adjoint_grads before lhe_lbm_adjoint_seed");
  if (!gphi0) return fail(l, LHE_ERR_ARG, "dL/dphi0 is NULL");
  if (gR && l->p.bc != LHE_BC_PERIODIC)
    return fail(l, LHE_ERR_ARG, "dL/dR(x) is not available on Dirichlet boxes (their source is a constant R)");
  if (lhe_status st = unscale(l, 1)) return st;
  const bool dev = l->p.precision == LHE_FP32_DEV;
  const int d = l->p.d;
  AdjGradArgs a{};
  a.g = l->g;
  a.adj = l->adj[l->acur];
  a.adjW = l->adjW[l->acur];
  a.gphi0 = gphi0;
  a.order = l->init_order_used;
  double *G = nullptr;
  if (a.order == 3) {
    if (l->grad_was_fd) {
      if (!l->fdgrad) LHE_CK(l, cudaMalloc(&l->fdgrad, sizeof(double) * (size_t)l->g.S * d));
      G = l->fdgrad;
    } else {
      G = ggrad;
    }
  }
  a.G = G;
  for (int k = 0; k < l->Q; ++k) a.omega[k] = l->omega[k];
  a.dt = l->dt;
  a.c = l->p.c;
  for (int i = 0; i < d; ++i) a.u[i] = l->p.u[i];
  LHE_CK(l, launch_adjoint_grads(d, dev, a, l->stream));
  if (a.order == 3 && l->grad_was_fd) LHE_CK(l, launch_fd_grad_transpose_add(d, l->g, l->dx, G, gphi0, l->stream));
  if (gR) LHE_CK(l, cudaMemcpyAsync(gR, l->gR, sizeof(double) * (size_t)l->g.S, cudaMemcpyDefault, l->stream));
  return LHE_OK;
}

}  // extern "C"

/*
 * lhe_lbm.h -- C ABI of the GB300 (sm_103a) library for the unified fourth-order BGK lattice
 * Boltzmann model of the d-dimensional linear hyperbolic equation (L-HE)
 *
 *     d_t phi + u . grad phi = R,   phi(x, 0) = phi0(x),                       (Sec. 2.1, Eq. (HE))
 *
 * on the DdQ(2d^2+1) lattice with the fourth-order equilibrium moments of Chen, Chai & Shi,
 * arXiv:2410.13165. Citations below name the paper's sections and equations.
 *
 * Conventions shared by every entry point
 *   - All pointers named *_dev are CUDA device pointers; *_host are host pointers. The caller owns
 *     every pointer it passes; the library never frees or retains them beyond the call, except
 *     where stated. The library owns the population buffers it allocates in lhe_lbm_create().
 *   - Every call is asynchronous on the handle's CUDA stream (params.stream, 0 = legacy default
 *     stream) unless it says it synchronises. Device pointers must stay valid until the stream
 *     has executed the call.
 *   - Fields are laid out with x_1 fastest: site = i_1 + n_1*(i_2 + n_2*(...)), S = prod(n_i).
 *     Vector fields (gradients) are component-major: v[i*S + site].
 *   - Lattice: square, spacing dx; time step dt = dx / c (acoustic scaling, Sec. 2.2).
 *       periodic : node i at lo + i dx,        dx = (hi - lo)/n
 *       full-way : node i at lo + i dx,        dx = (hi - lo)/(n - 1)   (nodes on the faces)
 *       half-way : node i at lo + (i + 1/2)dx, dx = (hi - lo)/n         (walls at mid-link)
 *     (the lattice-point sets of Eq. (rmse)); dx must be equal in every dimension.
 *   - Errors: every call returns an lhe_status; it never throws, traps or aborts the device.
 *     A human-readable message is available from lhe_lbm_last_error(). Device-side errors that
 *     are only known after kernels ran (non-finite values) surface at the next synchronising call.
 *   - Thread safety: a handle must not be used from two host threads at once.
 */
#ifndef LHE_LBM_H
#define LHE_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LHE_API __attribute__((visibility("default")))
#else
#define LHE_API
#endif

#define LHE_ABI_VERSION 1
#define LHE_MAX_DIM 5   /* the entropy conditions need d < 6 (Proposition 1, Eq. (sigma=0)) */
#define LHE_MAX_Q 51    /* 2 d^2 + 1 for d = 5 */
#define LHE_MAX_MODES 16

typedef struct lhe_lbm lhe_lbm; /* opaque handle */

typedef enum {
  LHE_OK = 0,
  LHE_ERR_ARG = 1,       /* invalid argument (message says which) */
  LHE_ERR_UNSTABLE = 2,  /* some EDF weight omega_k <= 0: not entropy stable (Sec. 4.1, Eq. (skfk)) */
  LHE_ERR_CUDA = 3,      /* a CUDA runtime call or kernel launch failed */
  LHE_ERR_OOM = 4,       /* device allocation failed */
  LHE_ERR_NONFINITE = 5, /* a NaN or Inf was found in the state */
  LHE_ERR_STATE = 6      /* call out of order (e.g. step before init) or unsupported combination */
} lhe_status;

typedef enum { LHE_BC_PERIODIC = 0, LHE_BC_FULLWAY = 1, LHE_BC_HALFWAY = 2 } lhe_bc_kind;

/* LHE_FP64: populations stored and updated in FP64.
 * LHE_FP32_DEV: populations stored as FP32 deviations g_k = f_k - omega_k phi from the local
 * equilibrium, phi stored and accumulated in FP64 (the library's precision form; the paper is
 * precision-agnostic). */
typedef enum { LHE_FP64 = 0, LHE_FP32_DEV = 1 } lhe_precision;

/* Fourth-order EDF moments m4_ij = m^{eq|4}_{x_i^2 x_j^2} (free after Eq. (third-condition-2)):
 * LHE_M4_RULE     -- Eq. (meq-4rd) with parameter g (the paper's numerics use g = 1/2), equal for all pairs;
 * LHE_M4_EXPLICIT -- m4[p] for the pairs i<j in lexicographic order, in units of c^4. */
typedef enum { LHE_M4_RULE = 0, LHE_M4_EXPLICIT = 1 } lhe_m4_mode;

/* lhe_lbm_params.flags. LHE_FLAG_NO_STAGING: run the FP32-deviation step of periodic D3Q19 boxes
 * with the register-pull kernel instead of the one that stages the pulled rows in shared memory
 * by bulk asynchronous copies (both compute the same bits; the staged one is the default where
 * its layout conditions hold: n_1 a multiple of 4 and at most 512). */
#define LHE_FLAG_NO_STAGING 1
/* LHE_FLAG_NO_PDL: launch every step kernel with plain stream ordering. By default the second and
 * later step kernels of one lhe_lbm_step / lhe_lbm_adjoint_step call are launched with programmatic
 * stream serialization: such a kernel may be scheduled while the step before it finishes, and waits
 * for that step to complete before it touches global memory (same results, shorter gaps between
 * consecutive steps). So is the first step kernel of a call when the step kernels that the library
 * launched last, in this process, were this handle's and on the same stream (consecutive calls of one
 * handle); work that the caller queued in between keeps its ordering (such a kernel then starts only
 * once that work is complete). Otherwise the first kernel of a call is ordered plainly behind the
 * stream. */
#define LHE_FLAG_NO_PDL 2
/* LHE_FLAG_TEST_EXPIRE_WAIT: a test hook for the failure path of the staged FP32-deviation kernel. Its
 * waits for copies are bounded (1 s); on expiry the kernel stops, waits (bounded) for the copies it
 * has in flight, sets a host-visible flag and returns; once that kernel has finished, lhe_lbm_step,
 * lhe_lbm_adjoint_step, lhe_lbm_macro and lhe_lbm_diagnostics (which synchronises, so it always sees
 * it) report LHE_ERR_CUDA until lhe_lbm_init or lhe_lbm_set_state starts a new state. With this flag the handle's first staged launch gives its compute warps a zero
 * limit, so that the path runs without any fault: that step stops early and leaves an invalid
 * state. No effect on other handles or kernels. */
#define LHE_FLAG_TEST_EXPIRE_WAIT 4
/* LHE_FLAG_NODE_BOUNDARY: in the FP64 step of a Dirichlet box, treat the boundary nodes with the
 * boundary-node kernels (the x_1-face nodes in the lanes of their rows, the others one thread per node
 * with the boundary data evaluated per node) instead of stepping the whole box as rows that take the
 * unknown populations from a dense array of the step's boundary data (the default, which holds one
 * more array of Q*S doubles). Same results: bit for bit with records of jets or the manufactured
 * solution, to rounding with the exact-solution family (whose data the dense form evaluates from
 * coefficients separated in time). */
#define LHE_FLAG_NODE_BOUNDARY 8

typedef struct {
  int32_t d;              /* spatial dimension, 1..5 */
  int32_t bc;             /* lhe_bc_kind */
  int32_t precision;      /* lhe_precision */
  int32_t init_order;     /* 1: f = f^eq;  3: Eq. (ini-simp) (Sec. 3.2) */
  int32_t bc_order;       /* full-way: 1, 3 or 4 (Eq. (bun1)); half-way: 1..4 (Eq. (bun2)); unused if periodic */
  int32_t m4_mode;        /* lhe_m4_mode */
  int32_t allow_unstable; /* nonzero: accept weights with omega_k <= 0 (otherwise LHE_ERR_UNSTABLE) */
  int32_t flags;          /* 0, or LHE_FLAG_* bits (kernel choices with identical results; a test hook) */
  int64_t n[LHE_MAX_DIM]; /* nodes per dimension (first d used); full-way n >= 3, otherwise n >= 3 */
  double lo[LHE_MAX_DIM]; /* box [lo, hi] per dimension */
  double hi[LHE_MAX_DIM];
  double c;               /* lattice velocity c = dx/dt > 0 (the paper's numerics use c = 1) */
  double u[LHE_MAX_DIM];  /* transport velocity u of Eq. (HE) */
  double R;               /* constant source R of Eq. (HE); see lhe_lbm_init for a per-site field */
  double tau;             /* relaxation time, s = 1/tau (Eq. (BGK-LB-Evolution)); the paper's method: tau = 0.5 */
  double g;               /* parameter of Eq. (meq-4rd), 0 < g < 1 */
  double m4[10];          /* explicit m4_ij (LHE_M4_EXPLICIT) */
  void *stream;           /* cudaStream_t used by every call on this handle (0 = default stream) */
} lhe_lbm_params;

/* Read-only description of a created handle. */
typedef struct {
  int32_t d, Q;            /* Q = 2 d^2 + 1 */
  int64_t S;               /* number of lattice nodes */
  int64_t n_boundary;      /* number of boundary nodes (Dirichlet), 0 if periodic */
  int64_t step;            /* current time index: the state holds t_n = step * dt */
  double dx, dt, s;        /* lattice spacing, time step, relaxation parameter */
  double m4[10];           /* fourth moments used, pairs i<j (units of c^4) */
  double omega[LHE_MAX_Q]; /* EDF weights omega_k (Eq. (omega_k-2)), f^eq_k = omega_k phi */
  int32_t e[LHE_MAX_Q * LHE_MAX_DIM]; /* unit lattice vectors e[k*d + i] (c_k = c e_k), paper's order */
  uint64_t state_bytes;    /* bytes of one forward state (see lhe_lbm_get_state) */
} lhe_lbm_info_t;

/* Dirichlet data phi = h on the boundary, taken from the exact-solution family
 *   h(x, t) = b + R t + sum_i g_i (x_i - u_i t) + sum_m a_m sin(kappa_m . (x - u t) + theta_m),
 * which solves Eq. (HE) for constant R. The boundary kernels evaluate it and the space-time
 * derivatives the boundary schemes need on the device, at every step's time. */
typedef struct {
  int32_t nmodes;                            /* 0..LHE_MAX_MODES */
  int32_t reserved0;                         /* must be 0 */
  double b;
  double g[LHE_MAX_DIM];
  double a[LHE_MAX_MODES];
  double kappa[LHE_MAX_MODES * LHE_MAX_DIM]; /* kappa[m*LHE_MAX_DIM + i] */
  double theta[LHE_MAX_MODES];
} lhe_wave;

/* Library version of this header (LHE_ABI_VERSION) and sizeof(lhe_lbm_params), for bindings
 * to check their struct layout. */
LHE_API int32_t lhe_lbm_abi_version(void);
LHE_API uint64_t lhe_lbm_params_size(void);

/* Fill *p with defaults: d = 3, periodic, FP64, init_order 3, bc_order 4, m4 rule with g = 1/2,
 * c = 1, tau = 0.5, R = 0, u = 0, n = 16, box [0,1]^d, default stream. */
LHE_API lhe_status lhe_lbm_default_params(lhe_lbm_params *p);

/* Compute the model without allocating device memory: m4 (Eq. (meq-4rd) or explicit), the EDF
 * weights omega (Eq. (omega_k-2)) and the lattice vectors. omega_host (Q doubles), m4_host
 * (d(d-1)/2 doubles) and e_host (Q*d int32) may each be NULL. Returns LHE_ERR_UNSTABLE when some
 * omega_k <= 0 (the arrays are still filled). */
LHE_API lhe_status lhe_lbm_model(const lhe_lbm_params *p, double *omega_host, double *m4_host, int32_t *e_host,
                         int32_t *Q_out);

/* Validate params, compute the model (as lhe_lbm_model), allocate two population buffers on the
 * current CUDA device (plus the boundary-node list for Dirichlet boxes) and return a handle.
 * Errors: LHE_ERR_ARG, LHE_ERR_UNSTABLE (unless allow_unstable), LHE_ERR_OOM, LHE_ERR_CUDA.
 * On error *out is NULL and lhe_lbm_last_error(NULL) holds the message. */
LHE_API lhe_status lhe_lbm_create(const lhe_lbm_params *p, lhe_lbm **out);

/* Synchronise the handle's stream and free everything the handle owns. NULL is accepted. */
LHE_API lhe_status lhe_lbm_destroy(lhe_lbm *lbm);

/* Message of the last failed call on this handle; with NULL, of the last failed create/model
 * call on this thread. The string lives until the next failing call. */
LHE_API const char *lhe_lbm_last_error(const lhe_lbm *lbm);

/* Fill *info (host). */
LHE_API lhe_status lhe_lbm_info(const lhe_lbm *lbm, lhe_lbm_info_t *info);

/* Source of the following steps: R_dev (device or host, S doubles, copied) is the per-site source
 * R(x) used from the next lhe_lbm_step on; NULL returns to the constant params.R. It lets a caller
 * drive a source that varies in time: before the step t_n -> t_{n+1} pass R(x, t_{n+1}). A step
 * streams, then collides at the new time (R_k = omega_k R(x), Eq. (BGK-LB-Evolution)); the R term of
 * the full-way scheme is taken at t_{n+1} (this source), those of the half-way scheme at t_n (the
 * source of the last collision); lhe_lbm_init's field is R(x, 0). Until the next step, macro and
 * diagnostics keep using the source of the last collision. On a Dirichlet box with jets, call it
 * before lhe_lbm_set_boundary_jet. The paper's fourth-order analysis assumes a constant R; with a
 * source that varies the scheme converges at about first order (measured). */
LHE_API lhe_status lhe_lbm_set_source(lhe_lbm *lbm, const double *R_dev);

/* Replace the CUDA stream used by subsequent calls. */
LHE_API lhe_status lhe_lbm_set_stream(lhe_lbm *lbm, void *stream);

/* Initialise the state at t = 0 (step index 0) from phi0_dev (S doubles):
 *   init_order 3: f_k(x,0) = omega_k [phi0 + (dt/2)(u - c_k) . grad phi0]    Eq. (ini-simp)
 *   init_order 1: f_k(x,0) = omega_k phi0                                     (f = f^eq)
 * grad_dev: d*S doubles (component-major), or NULL, in which case the gradient is the periodic
 * fourth-order central difference of phi0 (periodic boxes only; LHE_ERR_ARG otherwise).
 * R_dev: per-site source R(x) (S doubles; the discrete source is R_k = omega_k R(x)), or NULL for
 * the constant params.R. The field is copied. On Dirichlet boxes a field needs the boundary data as
 * jets (lhe_lbm_set_boundary_jet), whose R terms then take R at the boundary node.
 * The library stores post-collision populations internally, so init also applies one collision. */
LHE_API lhe_status lhe_lbm_init(lhe_lbm *lbm, const double *phi0_dev, const double *grad_dev, const double *R_dev);

/* Set the Dirichlet data (copied). Required before lhe_lbm_step on a full-way or half-way box. */
LHE_API lhe_status lhe_lbm_set_boundary_wave(lhe_lbm *lbm, const lhe_wave *w_host);

/* Number of values in a boundary jet: every derivative of phi of order 0..3 in the d + 1 variables
 * (t, x_1, ..., x_d), C(d + 4, 3) = 10, 20, 35, 56, 84 for d = 1..5. */
#define LHE_JET_LEN(d) (((d) + 4) * ((d) + 3) * ((d) + 2) / 6)

/* Points at which lhe_lbm_set_boundary_jet needs the Dirichlet data of the next step (Sec. 3.2):
 *   full-way (Eq. (bun1)): the boundary nodes, data at the new time t_{n+1};
 *   half-way (Eq. (bun2)): for every boundary node x_f and unknown population k (source x_f - e_k
 *     outside the box), the mid-link point x_f - c_k dt/2, data at the current time t_n.
 * Nodes come in the library's boundary-node order; half-way, a node's unknown links in the order of
 * k. *P_host receives the number of points; xyz_host (host, P*d doubles, point-major) receives the
 * coordinates, or is NULL to query P only; *t_offset_host (or NULL) receives the time of the data
 * minus t_n (dt full-way, 0 half-way), with t_n = info.step * dt. Errors: LHE_ERR_STATE on a
 * periodic box, LHE_ERR_ARG when P_host is NULL. */
LHE_API lhe_status lhe_lbm_boundary_points(const lhe_lbm *lbm, double *xyz_host, int64_t *P_host, double *t_offset_host);

/* Dirichlet data of the next step as jets of phi at the points of lhe_lbm_boundary_points, for
 * data that the exact-solution family of lhe_lbm_set_boundary_wave does not cover. jet_dev (device,
 * P * LHE_JET_LEN(d) doubles, point-major) holds at each point every derivative d^q phi / (dv_1 ..
 * dv_q), q = 0..3, over the non-decreasing tuples v_1 <= .. <= v_q of the variables (v = 0: t, v = i:
 * x_i), tuples of one length in lexicographic order: phi, phi_t, phi_x1, .., phi_tt, phi_tx1, ...
 * The library forms the unknown populations of Eq. (bun1) (orders 1, 3, 4) or the B_k of Eq. (bun2)
 * (orders 1..4) from them, asynchronously on the handle's stream (jet_dev must stay valid until the
 * stream has passed this call). The data serve exactly one step: the next lhe_lbm_step must have
 * n = 1 and needs new jets after it (LHE_ERR_STATE otherwise). lhe_lbm_set_boundary_wave switches
 * back to the exact-solution family. The constant R of the box enters as in the family's case.
 * Errors: LHE_ERR_STATE on a periodic box, LHE_ERR_ARG for NULL, LHE_ERR_CUDA. */
LHE_API lhe_status lhe_lbm_set_boundary_jet(lhe_lbm *lbm, const double *jet_dev);

/* Advance n >= 0 time steps of Eq. (BGK-LB-Evolution) (collide with s = 1/tau, stream), with
 * the full-way (Eq. (bun1)) or half-way (Eq. (bun2)) scheme for the unknown populations of the
 * boundary nodes of a Dirichlet box. Errors: LHE_ERR_STATE before init / without boundary data, and
 * with boundary jets when n > 1 or no jets were set since the last step. */
LHE_API lhe_status lhe_lbm_step(lhe_lbm *lbm, int64_t n);

/* Macroscopic variable phi(x, t_step) = sum_k f_k (Eq. (0-1-meq)) into phi_dev (S doubles). */
LHE_API lhe_status lhe_lbm_macro(lhe_lbm *lbm, double *phi_dev);

/* Synchronising diagnostics of the current state, into out_host[4]:
 *   [0] sum_x phi (mass), [1] sum_x sum_k f_k^2 / (2 omega_k) (total kinetic entropy, Eq. (skfk)),
 *   [2] max_x |phi|, [3] number of non-finite populations.
 * Returns LHE_ERR_NONFINITE when [3] > 0. */
LHE_API lhe_status lhe_lbm_diagnostics(lhe_lbm *lbm, double *out_host);

/* Diagnostics of a caller-owned FP64 state without allocating device memory (the paper has no
 * counterpart; this is a library service). For callers that cannot allocate at this point: code
 * whose device memory comes from a framework's allocator or a fixed budget, or that runs where the
 * CUDA runtime refuses cudaMalloc. It creates no handle and calls no allocating routine; its only
 * scratch memory is a 128 KiB array compiled into the library (one per device, alive until exit),
 * which holds the partial sums of at most 4096 reduction blocks.
 *   p       : the lattice (d, n, lo, hi, bc, c, u, tau, R, m4 settings, allow_unstable, stream);
 *             precision must be LHE_FP64. At most 268435456 nodes, the stated maximum of this entry
 *             point: larger lattices are rejected with LHE_ERR_ARG before anything is launched. As
 *             lhe_lbm_create, it returns LHE_ERR_UNSTABLE when some omega_k <= 0 unless
 *             allow_unstable is set (the entropy then has terms of either sign).
 *   pop_dev : Q*S post-collision FP64 populations, k-major (what lhe_lbm_get_state writes for an
 *             LHE_FP64 handle); R_dev: per-site source (S doubles) or NULL for the constant p->R.
 *   out_dev : 4 doubles of device memory receiving the values of lhe_lbm_diagnostics, in order.
 * Asynchronous on p->stream. The scratch array's device address is looked up (cudaGetSymbolAddress)
 * by the first call on a device, and again by the first call after the device's context was
 * created anew (cudaDeviceReset); make those calls before any stream capture. Every call overwrites
 * the same scratch array, so calls whose kernels overlap on the GPU (other streams or threads) race;
 * order them on one stream. */
LHE_API lhe_status lhe_lbm_diagnostics_noalloc(const lhe_lbm_params *p, const double *pop_dev, const double *R_dev,
                                               double *out_dev);

/* Copy the forward state (post-collision populations, and phi for LHE_FP32_DEV) to/from a
 * caller buffer of info.state_bytes bytes (device or host memory; cudaMemcpyKind default), for
 * checkpoint/restart. set_state also sets the step index. */
LHE_API lhe_status lhe_lbm_get_state(lhe_lbm *lbm, void *buf);
LHE_API lhe_status lhe_lbm_set_state(lhe_lbm *lbm, const void *buf, int64_t step);

/* ---------------- discrete adjoint ----------------
 * The scheme is affine in the populations, so its adjoint needs no forward state: given the
 * cotangent dL/dphi(t_T) of any loss L of the final field, lhe_lbm_adjoint_seed() sets the
 * adjoint state, each lhe_lbm_adjoint_step() applies the transpose of one step (reverse stream,
 * transposed collision) and accumulates dL/dR(x), and lhe_lbm_adjoint_grads() applies the
 * transpose of the initialisation. The adjoint uses the handle's precision and allocates its own
 * buffers on first use. Dirichlet boxes (both precisions): the transpose of
 * the boundary schemes drops the populations that leave the box (full-way, Eq. (bun1)) or returns
 * them, negated, to the opposite link of the same node (half-way, Eq. (bun2)); the boundary data
 * enter additively: lhe_lbm_adjoint_jet_grad gives their cotangent per step as jets. dL/dR(x) is not
 * available on Dirichlet boxes (constant R). */
LHE_API lhe_status lhe_lbm_adjoint_seed(lhe_lbm *lbm, const double *dL_dphiT_dev);
LHE_API lhe_status lhe_lbm_adjoint_step(lhe_lbm *lbm, int64_t n);
/* dL/dphi0 (S doubles), dL/d(grad phi0) (d*S doubles, only meaningful when lhe_lbm_init got an
 * explicit gradient; NULL to skip), dL/dR(x) (S doubles, NULL to skip; must be NULL on Dirichlet
 * boxes, else LHE_ERR_ARG). When init used the finite-difference gradient, its transpose is folded
 * into dL/dphi0. */
LHE_API lhe_status lhe_lbm_adjoint_grads(lhe_lbm *lbm, double *dL_dphi0_dev, double *dL_dgrad_dev, double *dL_dR_dev);

/* The manufactured solution phi*(x, t) = A exp(-lambda t) prod_i sin(kappa_i x_i + theta_i) of
 * phi_t + u . grad phi = R with its own source R(x, t) = -lambda phi* + sum_i u_i d_i phi*, which
 * varies in x and t (kappa and theta: the first d entries are used). */
typedef struct {
  double A, lambda;
  double kappa[LHE_MAX_DIM];
  double theta[LHE_MAX_DIM];
} lhe_sine_product;

/* Dirichlet data and source from the manufactured solution *sp_host (copied), formed on the device.
 * Every following lhe_lbm_step (any n) takes, for its step t_n -> t_{n+1}, the source R(x, t_{n+1}) of
 * its collision and the boundary data of Eq. (bun1) (at t_{n+1}) or Eq. (bun2) (at t_n) exactly as
 * lhe_lbm_set_boundary_jet would form them from the solution's jets at lhe_lbm_boundary_points, with
 * the R terms at the boundary node (lhe_lbm_set_source). The solution separates, phi* = exp(-lambda t)
 * P(x): this call forms the jets of P, the field R(x, t) exp(lambda t) and their records once
 * (synchronising the stream; P * LHE_JET_LEN(d) doubles of scratch); each step scales them by
 * exp(-lambda t). Initialise with lhe_lbm_init's R_dev = R(x, 0) so that the stored state carries the
 * solution's source; lhe_lbm_set_state re-forms R(x, t_step) of the restored state. lhe_lbm_set_boundary_wave, lhe_lbm_set_boundary_jet and lhe_lbm_set_source end
 * it. Errors: LHE_ERR_STATE on a periodic box, LHE_ERR_ARG for NULL or non-finite parameters,
 * LHE_ERR_OOM / LHE_ERR_CUDA. */
LHE_API lhe_status lhe_lbm_set_boundary_sine_product(lhe_lbm *lbm, const lhe_sine_product *sp_host);

/* Cotangent of the Dirichlet data of one step, as jets (Sec. 3.2; the transpose of the map from jets
 * to unknown populations of lhe_lbm_set_boundary_jet, Eq. (bun1) / Eq. (bun2)). When the adjoint
 * state is dL/df(t_m) (after lhe_lbm_adjoint_seed at t_T and T - m adjoint steps), dL_djet_dev
 * (device, P * LHE_JET_LEN(d) doubles, point-major, the points and derivative order of
 * lhe_lbm_boundary_points and lhe_lbm_set_boundary_jet) receives dL/d(jet) of the data of the step
 * t_{m-1} -> t_m: full-way the jets at the boundary nodes and t_m, half-way those at the mid-link
 * points and t_{m-1}. Call it before each lhe_lbm_adjoint_step(lbm, 1) to collect every step's. It
 * does not depend on whether the forward step took jets or lhe_lbm_set_boundary_wave's family: the
 * scheme is the same linear map of its data. Asynchronous on the handle's stream; the adjoint state is
 * unchanged. Errors: LHE_ERR_STATE on a periodic box or before lhe_lbm_adjoint_seed, LHE_ERR_ARG for
 * NULL, LHE_ERR_CUDA. */
LHE_API lhe_status lhe_lbm_adjoint_jet_grad(lhe_lbm *lbm, double *dL_djet_dev);

/* ---------------- stability maps (Sec. 4) ----------------
 * For npoints velocities sigma = u/c (sigma_host: npoints*d doubles, point-major, host memory):
 *   omega_min_host[p] = min_k omega_k(sigma_p), the EDF weights of Eq. (omega_k-2) with the handle-
 *                       less model given by params (d, tau, m4_mode/g/m4); Prop. 1's microscopic
 *                       entropy conditions are omega_min > 0;
 *   rho_max_host[p]   = max over xi in the grid xi_i = -pi + 2 pi j/nxi (j = 0..nxi-1, i = 1..d) of the
 *                       spectral radius of the amplification matrix G(xi) of Eq. (G) (one step on a
 *                       Fourier mode; von Neumann L2 stability: rho <= 1). +inf where the eigenvalue
 *                       iteration did not converge.
 * Only params->d (1..4), tau, m4_mode, g, m4 and stream are read. Synchronous; allocates and frees
 * its device scratch. Errors: LHE_ERR_ARG (NULL outputs, d outside 1..4, nxi outside 1..4096,
 * npoints * nxi^d above 2^40, non-finite sigma), LHE_ERR_CUDA. */
LHE_API lhe_status lhe_lbm_stability_map(const lhe_lbm_params *p, const double *sigma_host, int64_t npoints,
                                         int32_t nxi, double *rho_max_host, double *omega_min_host);

#ifdef __cplusplus
}
#endif
#endif /* LHE_LBM_H */

/*
 * pd.h - C ABI of the GB300 patch-dynamics library (libpd.so).
 *
 * Patch dynamics for unsteady, linear, heterogeneous 2D convection-diffusion-
 * reaction problems in orthogonal curvilinear coordinates (arXiv 2405.08764,
 * Sections 2-3).  One macro step (Section 3.3, steps (i)-(vi)) is
 *   edge data (eq. edge) -> lift (eqs. Lifting, C_0) -> micro burst of K
 *   forward-Euler steps of eq. (Computational_Problem) inside every patch ->
 *   restriction (eq. Restriction, trapezoid rule) -> time-derivative estimate
 *   and projective forward Euler (eqs. Time_Derivative, Extrapolation).
 *
 * General conventions
 *   - Every function returns a pd_status; nothing aborts or throws across the
 *     ABI.  On failure pd_last_error(g) returns a message for that grid.
 *   - Pointers named *_dev are device pointers owned by the caller (for example
 *     torch tensor data_ptr()); pointers without the suffix are host pointers.
 *     The library never frees caller memory.  It owns its coefficient, table and
 *     scratch buffers and frees them in pd_destroy_grid.
 *   - All device work is enqueued asynchronously on the grid's CUDA stream
 *     (given at creation, changeable with pd_set_stream).  Errors raised on the
 *     device (non-finite restriction values) are recorded in a device flag and
 *     reported by pd_sync or by the next call that reads it.
 *   - A grid object is not thread-safe; use one grid per host thread.
 *
 * Indexing (identical to the CPU oracle, written separately)
 *   macro node (i, j):  U[j * nxp + i], nxp = n_xi + 1, or n_xi if periodic_xi;
 *                       j = 0..n_eta; instance k starts at U_dev + info.u_offset.
 *   patch of node (i,j): p = (j - 1) * ncols + (i - i0), i0 = 1 (Dirichlet in xi)
 *                       or 0 (periodic), ncols = n_xi - 1 or n_xi, j = 1..n_eta-1.
 *   micro point (a, b): a along xi (0..m_xi-1), b along eta (0..m_eta-1),
 *                       array offset p * m_xi * m_eta + b * m_xi + a,
 *                       coordinate xi_a = xi_i - h_xi / 2 + a * dxi, dxi = h_xi / (m_xi - 1).
 */
#ifndef PD_H
#define PD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PD_ABI_VERSION 2

typedef enum {
    PD_OK = 0,
    PD_EINVAL = 1,     /* invalid argument or descriptor */
    PD_ENOMEM = 2,     /* device allocation failed */
    PD_ECUDA = 3,      /* CUDA runtime error (message in pd_last_error) */
    PD_ESTATE = 4,     /* call out of order (e.g. coefficients not set) */
    PD_EUNSTABLE = 5,  /* time step above the explicit stability bound */
    PD_ETIMEOUT = 6,   /* a bounded device wait gave up */
    PD_ENUMERIC = 7    /* non-finite values produced on the device */
} pd_status;

typedef enum { PD_MAP_IDENTITY = 0, PD_MAP_SINE = 1, PD_MAP_TANH = 2, PD_MAP_POLAR = 3 } pd_map;
typedef enum { PD_FP64 = 0, PD_FP32 = 1 } pd_precision;
typedef enum { PD_CONV_UPWIND = 0, PD_CONV_CENTRAL = 1 } pd_conv;
typedef enum { PD_RESTRICT_LIFTED = 0, PD_RESTRICT_MACRO = 1 } pd_restrict_mode;
/* Micro time stepper inside the patches: forward Euler (Section 4.2), or the
 * alternating direction implicit scheme of Section 4.1, read as the
 * Peaceman-Rachford splitting: with h = dt/2, Lx the xi part (alpha u_xixi -
 * nu u_xi + phi u/2), Ly the eta part and Lc = beta u_xieta (explicit),
 *   (I - h Lx) u* = u + h (Ly u + Lc u + g(t + h)),
 *   (I - h Ly) u' = u* + h (Lx u* + Lc u* + g(t + h)),
 * each line system tridiagonal with the ghost-point Neumann data.  Second
 * order in dt when beta = 0, first order otherwise. */
typedef enum { PD_MICRO_FE = 0, PD_MICRO_ADI = 1 } pd_micro_solver;
typedef enum { PD_SRC_NONE = 0, PD_SRC_MMS_SINPROD = 1, PD_SRC_EXP_LINEAR = 2,
               PD_SRC_GAUSS_PATCH = 3 } pd_source;
typedef enum { PD_TIME_CONST = 0, PD_TIME_EXP = 1, PD_TIME_SIN = 2 } pd_time_kind;
typedef enum { PD_SOL_NONE = 0, PD_SOL_EXP_XYT = 1, PD_SOL_SINPROD_DECAY = 2 } pd_solution;
typedef enum { PD_INIT_ZERO = 0, PD_INIT_EXACT = 1, PD_INIT_BESSEL = 2, PD_INIT_BUMP = 3,
               PD_INIT_ANNULUS_POLY = 4 } pd_init_kind;

/* One problem instance: macro mesh, mapping and micro discretisation.
 * Section 3: equidistant macro mesh on the computational box, patches of width
 * h = h_ratio * Delta centred on every interior node (h / Delta < 1), n = m - 1
 * nano steps per side, K micro steps per burst. */
typedef struct {
    int n_xi, n_eta;              /* macro intervals (>= 2; >= 3 if periodic) */
    int periodic_xi;              /* 1: xi is periodic (annulus, eq. Ann_C_IC_BCs) */
    double xi0, xi1, eta0, eta1;  /* computational box */
    int map;                      /* pd_map */
    double map_p[4];              /* SINE: lambda (eq. Stretching_Transformation);
                                     TANH: s_xi, s_eta (x = x0 + L tanh(s z)/tanh(s), z in [0,1]);
                                     POLAR: r_in, r_out, s_r (x = r(eta) cos xi, y = r(eta) sin xi,
                                     r = r_in + (r_out - r_in) rho(z), rho = z if s_r = 0, else
                                     (1 + tanh(s_r (2z - 1)) / tanh(s_r)) / 2) */
    int m_xi, m_eta;              /* micro points per side, 3..32 */
    double h_ratio_xi, h_ratio_eta; /* h / Delta in (0, 1) */
    int k_micro;                  /* micro steps per burst, 1..4096 */
    double cfl_micro;             /* micro dt = cfl * explicit limit (0 < cfl <= 1) */
    int prec;                     /* pd_precision of the micro burst */
    int conv_scheme;              /* pd_conv for the first derivatives */
    int restrict_mode;            /* pd_restrict_mode (reference value U^0 of eq. Time_Derivative) */
    int micro_solver;             /* pd_micro_solver; ADI needs one instance with per-point
                                     coefficients and m_xi == m_eta in {3,5,7,9,11} and runs
                                     in pd_step (fused path, any outer integrator) */
    double dt_micro;              /* > 0: fixed micro step (Section 4.1: tau / n_t), replacing
                                     cfl_micro; forward Euler still needs dt within its
                                     explicit bound (else PD_EUNSTABLE at pd_set_coeffs) */
} pd_grid_desc;

/* Coefficients of eq. (1), u_t = div(K grad u - v u) + f u + g, with
 *   K = d(x,y) [[M11, M12], [M12, M22]],
 *   d = d0 + dx x + dy y + ds sin(2 pi dk x) sin(2 pi dk y)
 *       + sum_{k=1..n_four} four_c[k-1] cos(k theta + four_phi[k-1]) cos(k pi rho),
 *       rho = (r - four_ra) / (four_rb - four_ra), (r, theta) polar angle of (x, y);
 *   v = (va0 + va1 x + va2 y, vb0 + vb1 x + vb2 y), f = f0;
 *   g = s(t) G(x, y): G by `src`, s by `tkind` (CONST 1, EXP exp(tc t), SIN sin(tc t));
 *     MMS_SINPROD: source of u = exp(-t) sin(pi x) sin(pi y) (constant K, affine v);
 *     EXP_LINEAR:  (src_p0 + src_p1 x + src_p2 y) exp(x + y)      (eq. P1_P family);
 *     GAUSS_PATCH: src_amp[p] exp(-(x^2 + y^2)), one amplitude per patch.
 * `sol` selects the Dirichlet data on the boundary nodes (NONE = 0). */
typedef struct {
    double M11, M12, M22;
    double d0, dx, dy, ds, dk;
    int n_four; double four_c[3], four_phi[3], four_ra, four_rb;
    double va[3], vb[3];
    double f0;
    int src; double src_p[3];
    const double* src_amp;        /* host pointer, n_patch values (GAUSS_PATCH only); copied */
    int tkind; double tc;
    int sol;
} pd_coeff_desc;

typedef struct pd_grid pd_grid;

/* Sizes and layout of one instance (pd_query). Byte offsets are into the
 * micro-state buffer of pd_lift / pd_micro_burst / pd_restrict. */
typedef struct {
    int n_patch, n_macro;         /* patches, macro nodes */
    int nxp, nyp;                 /* macro nodes along xi, eta */
    int m_xi, m_eta, k_micro, prec;
    long long u_offset;           /* offset (in doubles) of this instance in U_dev */
    long long patch_offset;       /* offset (in patches) of this instance in dU_dev and the bias section */
    long long point_offset;       /* offset (in micro points) of this instance in the u0, r, w sections */
    long long edge_offset;        /* offset (in entries) of this instance in the edge section */
    double dt_micro;              /* micro step (cfl rule G8, or the descriptor's fixed step) */
    double tau;                   /* burst length K * dt_micro */
    double dt_macro_suggested;    /* half the macro explicit bound (reading G9) */
    size_t state_bytes;           /* whole micro-state buffer (all instances) */
    size_t off_u0, off_r, off_w, off_edge, off_bias; /* section offsets, 256-byte aligned */
    int edge_stride;              /* max(m_xi, m_eta) + 2 of this instance */
    int exec_path;                /* pd_step path: 0 separate passes, 1 one fused kernel per
                                     macro step, 2 persistent dataflow kernel, 3 batched
                                     work-queue kernel (several instances or table storage) */
    int chunk_steps;              /* macro steps per persistent launch (path 2) */
    int has_cross;                /* 1 when beta (the mixed-derivative coefficient) is not
                                     identically zero on this instance */
    int has_tsrc;                 /* 1 when the source has a time factor */
} pd_info;

/* Create a grid of n_inst instances, descs[0..n_inst-1] (host array, copied);
 * instances may differ in every field except the precision.
 * `cuda_stream` is a cudaStream_t (NULL = default stream).  Allocates the
 * per-instance coefficient and scratch buffers on the current device, which
 * becomes the grid's device: later calls on the grid make it current for
 * their own work and restore the caller's current device before returning.
 * Errors: PD_EINVAL (bad descriptor), PD_ENOMEM, PD_ECUDA. */
pd_status pd_create_grid(const pd_grid_desc* descs, int n_inst, void* cuda_stream, pd_grid** out);
pd_status pd_destroy_grid(pd_grid* g);
pd_status pd_set_stream(pd_grid* g, void* cuda_stream);

/* Eq. (Computational_Problem): evaluate the transformed coefficients alpha,
 * beta, gamma, nu, omega, phi and the source factor G of instance `inst` at
 * every micro point on the device in FP64 (metric and Jacobian precompute),
 * then fix the micro step dt = cfl * min over points of the explicit bound
 * and the suggested macro step.  Synchronises the stream (setup only).
 * Errors: PD_EINVAL (bad kind, missing src_amp, J == 0 or non-finite
 * coefficients somewhere), PD_ECUDA. */
pd_status pd_set_coeffs(pd_grid* g, int inst, const pd_coeff_desc* c);

pd_status pd_query(const pd_grid* g, int inst, pd_info* out);
/* total doubles of U_dev / patches of dU_dev over all instances */
pd_status pd_sizes(const pd_grid* g, long long* n_macro_total, long long* n_patch_total,
                   size_t* state_bytes);

/* Copy the coefficients of instance `inst` to coef_dev (FP64) as
 * [n_patch][m_eta][m_xi][8] = alpha, beta, gamma, nu, omega, phi, G (times the
 * patch amplitude), 0: the values as stored (rounded to FP32 on PD_FP32 grids).
 * PD_ESTATE before pd_set_coeffs. */
pd_status pd_get_coeffs(pd_grid* g, int inst, double* coef_dev);

/* Fill the macro field of instance `inst` at time t (Section 4 initial data):
 * ZERO; EXACT (the `sol` of pd_set_coeffs); BESSEL: params = {n_modes (<= 8),
 * r_in, r_out, a_1..a_n}, sum_k a_k Z_k(mu_k r) cos(k theta) exp(-d0 mu_k^2 t)
 * with Z_k the Bessel cross product of eq. (Annulus_AS); BUMP: sin(pi z_eta) times
 * sin(pi z_xi) (or 1 + cos(xi)/2 if periodic); ANNULUS_POLY: params = {r_in, r_out},
 * (r - r_in)(r_out - r) sin(theta).  `params` is a host array. */
pd_status pd_init_field(pd_grid* g, int inst, int kind, const double* params, int n_params,
                        double t, double* U_dev);

/* Section 3.3 (i)-(ii), eqs. (edge), (Lifting), (C_0): for every patch of every
 * instance read the 3x3 macro stencil of U_dev at time t and write into the
 * micro-state buffer state_dev (pd_info.state_bytes, caller-owned, 256-byte
 * aligned): the lifted field u0 (FP64), the four edge-derivative vectors
 * (FP64, [p][4][edge_stride]: g_L(eta_b), g_R(eta_b) for b = -1..m_eta,
 * g_B(xi_a), g_T(xi_a) for a = -1..m_xi), the burst forcing
 * r = L_h(u0) + g(t) (grid precision), the departure w = 0 (grid precision)
 * and the restriction bias (FP64).  The burst evolves u = u0 + w. */
pd_status pd_lift(pd_grid* g, const double* U_dev, double t, void* state_dev);

/* Section 3.3 (iii): k_steps forward-Euler micro steps of the departure w in
 * every patch, starting at time t (t = lift time + steps already taken * dt),
 * Neumann edge data held fixed (Q = 1), ghost points as in reading G5. */
pd_status pd_micro_burst(pd_grid* g, void* state_dev, double t, int k_steps);

/* Section 3.3 (iv)-(v), eqs. (Restriction), (Time_Derivative): trapezoid
 * average of the burst, written as the restricted change over the burst
 * dU_dev[p] = U^{1,n} - U^{0,n} (FP64, one per patch over all instances),
 * formed without subtracting two nearly equal averages. */
pd_status pd_restrict(pd_grid* g, const void* state_dev, double* dU_dev);

/* Eq. (Extrapolation): U += dt_macro * dU / tau on the interior nodes of every
 * instance, then the Dirichlet data at t + dt_macro on the boundary nodes. */
pd_status pd_project(pd_grid* g, double* U_dev, const double* dU_dev, double t, double dt_macro);

/* n_macro whole macro steps (Section 3.3 (i)-(vi) repeated) from time t0 with
 * step dt_macro (<= 0: each instance's suggested step), fused into one kernel
 * per macro step; U_dev holds the result at t0 + n_macro * dt_macro.  When the
 * grid's graph mode is on (default), the launch sequence for a given
 * (U_dev, n_macro) is captured once into a CUDA graph and replayed.
 * Errors: PD_EINVAL, PD_ESTATE (coefficients missing), PD_ECUDA. */
pd_status pd_step(pd_grid* g, double* U_dev, double t0, double dt_macro, int n_macro);
pd_status pd_set_graph_mode(pd_grid* g, int enabled);

/* Outer (projective) integrator of pd_step.  PD_INT_EULER is the paper's
 * forward Euler, eq. (Extrapolation).  The paper names second-order
 * Runge-Kutta and Adams-Bashforth outer integrators as the higher-order
 * alternatives (Section 1); with F(U, T) = (U^1 - U^0)/tau from eq.
 * (Time_Derivative):
 *   PD_INT_HEUN: U* = U_n + dt F(U_n, T_n) (boundary data at T_{n+1}),
 *                U_{n+1} = U_n + dt/2 (F(U_n, T_n) + F(U*, T_{n+1}));
 *   PD_INT_AB2:  U_{n+1} = U_n + dt (3/2 F(U_n, T_n) - 1/2 F(U_{n-1}, T_{n-1})),
 *                each pd_step call starting with one Heun step.
 * The second-order integrators run one-instance grids with per-point records
 * and m_xi == m_eta in {3,5,7,9,11} (PD_EINVAL otherwise), without graph
 * capture or the persistent path: two fused kernels and one combination per
 * Heun step, one restricted-change kernel and one update per AB2 step. */
typedef enum { PD_INT_EULER = 0, PD_INT_HEUN = 1, PD_INT_AB2 = 2 } pd_integrator;
pd_status pd_set_integrator(pd_grid* g, int kind);

/* Edge-data refresh during the burst (Section 3: the Neumann data of eq. (edge)
 * are held fixed over the burst, the Q = 1 case; refreshing them is named as
 * the more accurate alternative).  With q > 1 every burst of pd_step is cut
 * into q sub-bursts of K/q forward-Euler steps, and before sub-burst s >= 1 the
 * edge data of every patch are rebuilt from the interpolant of the macro
 * estimate U + (restricted change of the departure so far) on interior nodes
 * and the Dirichlet data at the sub-burst start time on boundary nodes; the
 * micro field is not lifted again.  pd_step then runs the separate passes
 * (lift, q bursts, q restrictions, q - 1 refreshes, projection) for any m <= 32,
 * without graph capture.  q = 1 restores fixed edge data.
 * Errors: PD_EINVAL for q < 1, a K not divisible by q on some instance, or the
 * ADI micro solver; pd_step returns PD_EINVAL when q > 1 meets a second-order
 * outer integrator or 1-D coefficient tables. */
pd_status pd_set_edge_refresh(pd_grid* g, int q);

/* The same macro steps as pd_step with one fused kernel per step, for callers
 * that may not allocate device memory during a step.  The paper has no
 * counterpart; it is a deployment variant.  Such callers are, e.g., a
 * solver loop embedded in a host application whose memory pool already
 * reserves nearly all of HBM (a cudaMalloc there can fail mid-run), or a
 * latency-bound loop that cannot afford cudaMalloc's implicit device
 * synchronisation.  pd_step allocates its second macro field and its time
 * tables on first use; this call instead carves both out of one fixed
 * 4 MiB device array per device (524288 doubles) that lives in the library.
 * Limits: a grid of one instance, per-point coefficient records (the default
 * for one instance), m_xi == m_eta in {3,5,7,9,11}, the forward-Euler outer
 * step and fixed edge data (a grid set to Heun or AB2 by pd_set_integrator,
 * or to q > 1 by pd_set_edge_refresh, is refused with PD_EINVAL rather than
 * stepped differently from pd_step); forward-Euler and ADI bursts both run.
 * The need is
 * roundup32(nxp*nyp) + n_macro*(k_micro + 3) doubles, and a larger request
 * is rejected with PD_EINVAL (take fewer macro steps per call).  Nothing in
 * the array has to start at zero: every step writes the whole next field and
 * the time table is written before it is read.  All calls on a device share
 * the array: two calls whose work overlaps in time (different streams,
 * grids or host threads without ordering between them) race and corrupt
 * each other's results; order them on one stream.  Every call looks up the
 * array's address in the current context of the grid's device (so a context
 * created again after cudaDeviceReset is served correctly); the first lookup
 * in a context loads the library's device code (set-up work in the CUDA
 * runtime), so the first call on a device should precede any stream capture.
 * The caller's current device is unchanged on return.  Results equal
 * pd_step's per-step kernel path.  Errors: PD_EINVAL, PD_ESTATE, PD_ECUDA. */
pd_status pd_step_noalloc(pd_grid* g, double* U_dev, double t0, double dt_macro, int n_macro);

/* Coefficient storage (call before pd_set_coeffs): 0 auto (default: 1-D metric
 * tables for constant-coefficient, source-free instances when the grid holds
 * several instances, else per-point records), 1 records, 2 tables where
 * possible.  Table storage needs O(N m) memory per instance instead of O(N^2 m^2). */
pd_status pd_set_coeff_storage(pd_grid* g, int mode);

/* Batched execution (grids with several instances, or table storage): one
 * kernel per macro step over all instances, warps pulling patch groups from a
 * device work queue (costliest micro size first).  The autotuner times
 * n_trial_steps macro steps of each candidate (64/128 threads per block x
 * full/half patches per warp) on scratch fields and keeps the fastest; it runs
 * on the first batched pd_step unless disabled with pd_set_autotune(g, 0, ...),
 * which fixes the configuration instead. */
pd_status pd_autotune(pd_grid* g, int n_trial_steps, int* block, int* half_patches);
pd_status pd_set_autotune(pd_grid* g, int enabled, int block, int half_patches);

/* Persistent dataflow execution of pd_step (default on).  When all patch warps
 * of an instance fit on the device at once, a chunk of macro steps runs in one
 * cooperative launch: each warp keeps its micro-stencil weights in registers and
 * waits only for the neighbouring warps that produce its 3x3 macro stencil
 * (per-warp step counters, release/acquire).  Every wait gives up after
 * `wait_ns` nanoseconds (default 250 ms, pd_set_wait_limit); the kernel then sets a
 * device flag and returns, and pd_sync reports PD_ETIMEOUT.  Otherwise pd_step
 * launches one fused kernel per macro step. */
pd_status pd_set_persistent(pd_grid* g, int enabled);
pd_status pd_set_wait_limit(pd_grid* g, long long wait_ns);
/* Test hook for the failure path: item warp `warp` of the persistent kernel
 * never publishes its step counter, so its neighbours' bounded waits expire
 * (-1 restores normal operation). */
pd_status pd_test_silence_warp(pd_grid* g, int warp);

/* Wait for the stream and report device-side errors (PD_ENUMERIC). */
pd_status pd_sync(pd_grid* g);

/* Checkpoint (host file): U of every instance, time and step counter, plus a
 * hash of the grid descriptors; pd_load_checkpoint refuses a mismatched hash. */
pd_status pd_save_checkpoint(pd_grid* g, const double* U_dev, double t, long long step,
                             const char* path);
pd_status pd_load_checkpoint(pd_grid* g, double* U_dev, double* t, long long* step,
                             const char* path);

/* Number of kernels this grid has launched (graph replays count their nodes). */
long long pd_launch_count(const pd_grid* g);

/* Kernel timing for roofline figures: when enabled, every pd_step records two
 * CUDA events on the grid's stream around its macro-step kernels (after the
 * time-table kernel).  pd_get_timing waits for the last event and returns the
 * summed event time in milliseconds and the number of macro steps it covers;
 * pd_set_timing(g, 1) also resets the sums. */
pd_status pd_set_timing(pd_grid* g, int enabled);
pd_status pd_get_timing(pd_grid* g, double* ms, long long* n_macro_steps);

const char* pd_status_str(pd_status s);
const char* pd_last_error(const pd_grid* g);
int pd_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif

/*
 * Plain FP64 CPU oracle for curvilinear patch dynamics (arXiv 2405.08764).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code with the CUDA
 * path: everything here is written from the paper (Sections 2-3) and from the
 * readings listed in the design notes, evaluated loop by loop in double
 * precision with no blocking or fusion.
 *
 * Conventions (identical indexing to the CUDA path, written separately):
 *   macro node (i, j):    U[j * nxp + i], nxp = n_xi + 1 (or n_xi if periodic in xi)
 *   patch (i, j):         p = (j - 1) * ncols + (i - i0); i0 = 1 (Dirichlet) or 0 (periodic),
 *                         ncols = n_xi - 1 (Dirichlet) or n_xi (periodic)
 *   micro point (a, b):   p * m_xi * m_eta + b * m_xi + a, a along xi, b along eta
 *   micro coordinate:     xi_a = xi_i - h_xi / 2 + a * dxi, dxi = h_xi / (m_xi - 1)
 */
#ifndef PD_ORACLE_H
#define PD_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_MAP_IDENTITY = 0, ORC_MAP_SINE = 1, ORC_MAP_TANH = 2, ORC_MAP_POLAR = 3 };
enum { ORC_CONV_UPWIND = 0, ORC_CONV_CENTRAL = 1 };
enum { ORC_RESTRICT_LIFTED = 0, ORC_RESTRICT_MACRO = 1 };
enum { ORC_SRC_NONE = 0, ORC_SRC_MMS_SINPROD = 1, ORC_SRC_EXP_LINEAR = 2, ORC_SRC_GAUSS_PATCH = 3 };
enum { ORC_TIME_CONST = 0, ORC_TIME_EXP = 1, ORC_TIME_SIN = 2 };
enum { ORC_SOL_NONE = 0, ORC_SOL_EXP_XYT = 1, ORC_SOL_SINPROD_DECAY = 2 };
enum { ORC_INIT_ZERO = 0, ORC_INIT_EXACT = 1, ORC_INIT_BESSEL = 2, ORC_INIT_BUMP = 3, ORC_INIT_ANNULUS_POLY = 4 };
enum { ORC_FORM_SPLIT = 0, ORC_FORM_LITERAL = 1 };
enum { ORC_MICRO_FE = 0, ORC_MICRO_ADI = 1 };

/* One problem instance: geometry, micro discretisation and CDR coefficients. */
typedef struct {
    int n_xi, n_eta;             /* macro intervals */
    int periodic_xi;             /* 1: xi periodic (annulus) */
    double xi0, xi1, eta0, eta1; /* computational box */
    int map;                     /* ORC_MAP_* */
    double map_p[4];             /* sine: lambda | tanh: s_x, s_y | polar: r_in, r_out, s_r */
    int m_xi, m_eta;             /* micro points per patch side */
    double h_ratio_xi, h_ratio_eta; /* h / Delta */
    int k_micro;                 /* micro steps per burst */
    double cfl_micro;            /* fraction of the explicit micro limit */
    int conv;                    /* ORC_CONV_* */
    int restrict_mode;           /* ORC_RESTRICT_* */
    /* diffusion tensor K(x,y) = d(x,y) * [[M11, M12], [M12, M22]], with
       d = d0 + dx x + dy y + ds sin(2 pi k x) sin(2 pi k y)
           + sum_k c_k cos(k theta + phi_k) cos(k pi rho(r)),  rho = (r - ra)/(rb - ra) */
    double M11, M12, M22;
    double d0, dx, dy;
    double ds, dk;
    int n_four; double four_c[3], four_phi[3]; double four_ra, four_rb;
    /* velocity v = (a0 + a1 x + a2 y, b0 + b1 x + b2 y), reaction f = f0 */
    double va[3], vb[3];
    double f0;
    /* source g = s(t) G(x,y) [* amp[p] for ORC_SRC_GAUSS_PATCH] */
    int src; double src_p[3]; const double* src_amp;
    int tkind; double tc;
    /* exact solution used for Dirichlet data and errors */
    int sol;
    /* micro time stepper: forward Euler (Section 4.2) or the ADI scheme of
       Section 4.1; a positive dt_micro_fixed replaces the cfl rule (G8) */
    int micro;
    double dt_micro_fixed;
    /* Q: edge data refreshed Q times per burst (Q = 1 or 0: fixed over the
       burst, Section 3); Q > 1 needs k_micro divisible by Q and forward Euler */
    int q_refresh;
} orc_problem;

/* sizes */
int orc_n_patch(const orc_problem* P);
int orc_n_macro(const orc_problem* P);
int orc_validate(const orc_problem* P); /* 0 = ok */

/* map value and derivatives: out[12] = x, y, x_xi, x_eta, y_xi, y_eta,
   x_xixi, x_xieta, x_etaeta, y_xixi, y_xieta, y_etaeta */
void orc_map(const orc_problem* P, double xi, double eta, double* out);
/* transformed coefficients at a computational point: out[7] = alpha, beta,
   gamma, nu, omega, phi, G (spatial source factor without patch amplitude) */
void orc_coeffs(const orc_problem* P, double xi, double eta, double* out);
/* physical-space quantities for independent pins: out[13] = K11, K12, K22,
   dK11/dx, dK12/dx, dK22/dx, dK11/dy, dK12/dy, dK22/dy, v1, v2, div v, f */
void orc_physical(const orc_problem* P, double x, double y, double* out);
double orc_time_factor(const orc_problem* P, double t);
double orc_exact(const orc_problem* P, double x, double y, double t);

/* step sizes (readings G8, G9) */
double orc_dt_micro(const orc_problem* P);
double orc_dt_macro(const orc_problem* P);

/* initial / exact fields at macro nodes */
void orc_init_field(const orc_problem* P, int kind, const double* params, double t, double* U);
/* micro-point coordinates of every patch: xi[n_patch*m*m], eta[...] */
void orc_micro_coords(const orc_problem* P, double* xi, double* eta);

/* S1 + S2: edge data and lifted field of every patch at macro state U.
   u0: [n_patch][m_eta][m_xi]; edge: [n_patch][4][m+2] with g_L(eta_b), g_R(eta_b) for
   b = -1..m_eta, g_B(xi_a), g_T(xi_a) for a = -1..m_xi (end entries are extrapolated). */
void orc_lift(const orc_problem* P, const double* U, double* u0, double* edge);
/* S2 forcing used by the split burst: r0 = L_h(u0 with ghosts) + g(t) */
void orc_forcing(const orc_problem* P, const double* U, double t, double* r0);
/* S3: burst of k steps of forward Euler from the lifted state at time t.
   form SPLIT:   out = departure w = u(t + k dt) - u0
   form LITERAL: out = u(t + k dt) */
void orc_burst(const orc_problem* P, const double* U, double t, int k, double dt,
               int form, double* out);
/* S4: restricted change dU = U^{1} - U^{0} per patch from a burst result */
void orc_restrict(const orc_problem* P, const double* U, const double* burst_out,
                  int form, double* dU);
/* S5: projective forward Euler + boundary data at t + dt_macro */
void orc_project(const orc_problem* P, double* U, const double* dU, double t,
                 double dt_macro, double tau);
void orc_apply_bc(const orc_problem* P, double* U, double t);
/* whole macro steps (S1..S5), n_steps of size dt_macro from t0 */
void orc_step(const orc_problem* P, double* U, double t0, double dt_macro, int n_steps,
              double dt_micro, int form);

/* full-domain solve of the transformed PDE on the uniform computational grid with
   spacing (Delta_xi / refine, Delta_eta / refine), forward Euler with step dt, over
   n_steps; u: full fine grid [(n_eta*refine+1)][nxf], nxf = n_xi*refine(+1 if not periodic) */
int orc_full_domain_size(const orc_problem* P, int refine, int* nxf, int* nyf);
void orc_full_domain(const orc_problem* P, int refine, double* u, double t0, double dt,
                     int n_steps);

/* The micro solver of patch p alone in the split form: from the departure
   w0 [m_eta][m_xi] (mirror ghosts, zero edge data) with the forcing r
   [m_eta][m_xi] (NULL = 0) plus the source change (s(t) - s(T)) G, K steps of
   dt from time T by P->micro (forward Euler or ADI); out = departure after K. */
void orc_micro_patch(const orc_problem* P, int p, const double* w0, const double* r, double T,
                     int K, double dt, double* out);

/* dU for a selection of patches only (sampled checks at full size) */
void orc_patch_dU(const orc_problem* P, const double* U, double t, double dt, int form,
                  int n_sel, const int* sel, double* dU);

/* annulus eigenfunctions Z_k(mu r) = J_k(mu ra) Y_k(mu r) - Y_k(mu ra) J_k(mu r) */
double orc_bessel_root(int k, double ra, double rb, int which);
double orc_bessel_Z(int k, double mu, double ra, double r);
/* int_ra^rb r Z_1(mu r)^2 dr (composite Simpson) */
double orc_bessel_norm(double mu, double ra, double rb, int n_int);
/* eq. (Annulus_AS): diffusion (D = 1) of (r - ra)(rb - r) sin(theta) in the annulus,
   truncated at n_roots terms */
double orc_annulus_series(double ra, double rb, double r, double theta, double t, int n_roots);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif

/*
 * Plain FP64 CPU oracle for curvilinear patch dynamics (arXiv 2405.08764).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.  It shares no
 * code with the CUDA library.  Each function names the passage of the paper it
 * follows; where the paper is silent the reading used is stated in the comment
 * (the same readings are listed in the design notes).
 *
 * Parity status: every stage is pinned by tests against closed forms, special
 * cases or brute force (see tests/test_oracle_*.py); none is "parity unpinned".
 */
#include "pd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* threads the parallel loops over patches use (1 without OpenMP) */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_MAXM 64

/* ------------------------------------------------------------------------- */
/* sizes and indexing (Section 3: macro mesh, patches centred on interior nodes) */

static int n_xpts(const orc_problem* P) { return P->periodic_xi ? P->n_xi : P->n_xi + 1; }
static int n_cols(const orc_problem* P) { return P->periodic_xi ? P->n_xi : P->n_xi - 1; }
static int i_first(const orc_problem* P) { return P->periodic_xi ? 0 : 1; }
static int n_rows(const orc_problem* P) { return P->n_eta - 1; }
static double d_xi(const orc_problem* P) { return (P->xi1 - P->xi0) / P->n_xi; }
static double d_eta(const orc_problem* P) { return (P->eta1 - P->eta0) / P->n_eta; }

int orc_n_patch(const orc_problem* P) { return n_cols(P) * n_rows(P); }
int orc_n_macro(const orc_problem* P) { return n_xpts(P) * (P->n_eta + 1); }

int orc_validate(const orc_problem* P)
{
    if (P->n_xi < 2 || P->n_eta < 2) return 1;
    if (P->periodic_xi && P->n_xi < 3) return 1;
    if (P->m_xi < 3 || P->m_eta < 3 || P->m_xi > ORC_MAXM || P->m_eta > ORC_MAXM) return 2;
    /* h / Delta < 1 keeps patches apart (Section 3) */
    if (!(P->h_ratio_xi > 0.0 && P->h_ratio_xi < 1.0)) return 3;
    if (!(P->h_ratio_eta > 0.0 && P->h_ratio_eta < 1.0)) return 3;
    if (P->k_micro < 1) return 4;
    if (!(P->xi1 > P->xi0) || !(P->eta1 > P->eta0)) return 5;
    if (P->micro != ORC_MICRO_FE && P->micro != ORC_MICRO_ADI) return 6;
    if (!(P->dt_micro_fixed >= 0.0) || !isfinite(P->dt_micro_fixed)) return 6;
    if (P->q_refresh < 0 || (P->q_refresh > 1 && (P->k_micro % P->q_refresh != 0 || P->micro != ORC_MICRO_FE)))
        return 7;
    return 0;
}

static int wrap_i(const orc_problem* P, int i)
{
    if (!P->periodic_xi) return i;
    int n = P->n_xi;
    return ((i % n) + n) % n;
}

static double macro_U(const orc_problem* P, const double* U, int i, int j)
{
    return U[j * n_xpts(P) + wrap_i(P, i)];
}

/* ------------------------------------------------------------------------- */
/* Mappings: the sine stretching of Section 4.1 (x = xi + lambda/pi sin(pi xi)),
   the polar map of Section 4.2 (x = eta cos xi, y = eta sin xi) generalised to
   a radial profile r(eta), and the tanh stretching used by the heterogeneous
   workloads (reading: x = x0 + L tanh(s zeta) / tanh(s), zeta in [0,1]). */

static void stretch_tanh(double s, double q0, double q1, double q, double* X, double* X1, double* X2)
{
    double L = q1 - q0;
    double z = (q - q0) / L;
    if (s == 0.0) { *X = q; *X1 = 1.0; *X2 = 0.0; return; }
    double T = tanh(s);
    double th = tanh(s * z);
    double sech2 = 1.0 - th * th;
    *X = q0 + L * th / T;
    *X1 = s * sech2 / T;
    *X2 = -2.0 * s * s * sech2 * th / (T * L);
}

static void radial_profile(const orc_problem* P, double eta, double* R, double* R1, double* R2)
{
    double ra = P->map_p[0], rb = P->map_p[1], sr = P->map_p[2];
    double L = P->eta1 - P->eta0;
    double z = (eta - P->eta0) / L;
    double rho, rho1, rho2;
    if (sr == 0.0) { rho = z; rho1 = 1.0; rho2 = 0.0; }
    else {
        double T = tanh(sr);
        double q = sr * (2.0 * z - 1.0);
        double th = tanh(q);
        double sech2 = 1.0 - th * th;
        rho = 0.5 * (1.0 + th / T);
        rho1 = sr * sech2 / T;
        rho2 = -4.0 * sr * sr * sech2 * th / T;
    }
    *R = ra + (rb - ra) * rho;
    *R1 = (rb - ra) * rho1 / L;
    *R2 = (rb - ra) * rho2 / (L * L);
}

void orc_map(const orc_problem* P, double xi, double eta, double* o)
{
    memset(o, 0, 12 * sizeof(double));
    switch (P->map) {
    case ORC_MAP_IDENTITY:
        o[0] = xi; o[1] = eta; o[2] = 1.0; o[5] = 1.0;
        break;
    case ORC_MAP_SINE: {
        double lam = P->map_p[0];
        o[0] = xi + lam / M_PI * sin(M_PI * xi);
        o[1] = eta + lam / M_PI * sin(M_PI * eta);
        o[2] = 1.0 + lam * cos(M_PI * xi);
        o[5] = 1.0 + lam * cos(M_PI * eta);
        o[6] = -lam * M_PI * sin(M_PI * xi);
        o[11] = -lam * M_PI * sin(M_PI * eta);
        break;
    }
    case ORC_MAP_TANH: {
        double X, X1, X2, Y, Y1, Y2;
        stretch_tanh(P->map_p[0], P->xi0, P->xi1, xi, &X, &X1, &X2);
        stretch_tanh(P->map_p[1], P->eta0, P->eta1, eta, &Y, &Y1, &Y2);
        o[0] = X; o[1] = Y; o[2] = X1; o[5] = Y1; o[6] = X2; o[11] = Y2;
        break;
    }
    case ORC_MAP_POLAR: {
        double R, R1, R2;
        radial_profile(P, eta, &R, &R1, &R2);
        double c = cos(xi), s = sin(xi);
        o[0] = R * c;       o[1] = R * s;
        o[2] = -R * s;      o[3] = R1 * c;      /* x_xi, x_eta */
        o[4] = R * c;       o[5] = R1 * s;      /* y_xi, y_eta */
        o[6] = -R * c;      o[7] = -R1 * s;     o[8] = R2 * c;   /* x_xixi, x_xieta, x_etaeta */
        o[9] = -R * s;      o[10] = R1 * c;     o[11] = R2 * s;  /* y_xixi, y_xieta, y_etaeta */
        break;
    }
    default: break;
    }
}

/* ------------------------------------------------------------------------- */
/* Physical problem, eq. (1): u_t = div(K grad u - v u) + f u + g.  The paper
   takes K = D(x,y) I; the tensor K = d(x,y) M is the heterogeneous extension
   the workloads ask for. */

static void scalar_d(const orc_problem* P, double x, double y, double* d, double* dxo, double* dyo)
{
    double v = P->d0 + P->dx * x + P->dy * y;
    double gx = P->dx, gy = P->dy;
    if (P->ds != 0.0) {
        double k2 = 2.0 * M_PI * P->dk;
        double sx = sin(k2 * x), sy = sin(k2 * y);
        v += P->ds * sx * sy;
        gx += P->ds * k2 * cos(k2 * x) * sy;
        gy += P->ds * k2 * sx * cos(k2 * y);
    }
    for (int k = 1; k <= P->n_four; ++k) {
        double r = sqrt(x * x + y * y);
        double th = atan2(y, x);
        double ra = P->four_ra, rb = P->four_rb;
        double rho = (r - ra) / (rb - ra);
        double ck = P->four_c[k - 1], ph = P->four_phi[k - 1];
        double A = cos(k * th + ph), dA = -k * sin(k * th + ph);
        double B = cos(k * M_PI * rho), dB = -k * M_PI * sin(k * M_PI * rho) / (rb - ra);
        /* d/dx = cos(th) d/dr - sin(th)/r d/dth ; d/dy = sin(th) d/dr + cos(th)/r d/dth */
        double ct = x / r, st = y / r;
        v += ck * A * B;
        gx += ck * (ct * A * dB - st / r * dA * B);
        gy += ck * (st * A * dB + ct / r * dA * B);
    }
    *d = v; *dxo = gx; *dyo = gy;
}

void orc_physical(const orc_problem* P, double x, double y, double* o)
{
    double d, gx, gy;
    scalar_d(P, x, y, &d, &gx, &gy);
    o[0] = d * P->M11; o[1] = d * P->M12; o[2] = d * P->M22;
    o[3] = gx * P->M11; o[4] = gx * P->M12; o[5] = gx * P->M22;
    o[6] = gy * P->M11; o[7] = gy * P->M12; o[8] = gy * P->M22;
    o[9] = P->va[0] + P->va[1] * x + P->va[2] * y;
    o[10] = P->vb[0] + P->vb[1] * x + P->vb[2] * y;
    o[11] = P->va[1] + P->vb[2];
    o[12] = P->f0;
}

/* spatial source factor G(x,y); the full source is s(t) G (times a per-patch
   amplitude for ORC_SRC_GAUSS_PATCH) */
static double source_G(const orc_problem* P, double x, double y)
{
    switch (P->src) {
    case ORC_SRC_MMS_SINPROD: {
        /* g for u = exp(-t) sin(pi x) sin(pi y) with constant K and affine v:
           g = u_t - div(K grad u) + v.grad u + (div v - f) u */
        double ph[13];
        orc_physical(P, x, y, ph);
        double sx = sin(M_PI * x), sy = sin(M_PI * y), cx = cos(M_PI * x), cy = cos(M_PI * y);
        double S = sx * sy;
        double lapK = -M_PI * M_PI * (ph[0] + ph[2]) * S + 2.0 * M_PI * M_PI * ph[1] * cx * cy;
        double vgrad = M_PI * (ph[9] * cx * sy + ph[10] * sx * cy);
        return -S - lapK + vgrad + (ph[11] - ph[12]) * S;
    }
    case ORC_SRC_EXP_LINEAR:
        /* eq. (P1_P) family: g = (p0 + p1 x + p2 y) exp(x + y) exp(t) */
        return (P->src_p[0] + P->src_p[1] * x + P->src_p[2] * y) * exp(x + y);
    case ORC_SRC_GAUSS_PATCH:
        return exp(-(x * x + y * y));
    default:
        return 0.0;
    }
}

double orc_time_factor(const orc_problem* P, double t)
{
    switch (P->tkind) {
    case ORC_TIME_EXP: return exp(P->tc * t);
    case ORC_TIME_SIN: return sin(P->tc * t);
    default: return 1.0;
    }
}

double orc_exact(const orc_problem* P, double x, double y, double t)
{
    switch (P->sol) {
    case ORC_SOL_EXP_XYT: return exp(x + y + t);              /* eq. (CDR_Phy_Exact) */
    case ORC_SOL_SINPROD_DECAY: return exp(-t) * sin(M_PI * x) * sin(M_PI * y);
    default: return 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* Eq. (Computational_Problem): coefficients of the transformed operator.
   Derived operator (reading R2; it reproduces the worked examples of
   eqs. (P1_C), (P1_C_Vari_Diff), (Ann_Diff_Computational)):
     J = x_xi y_eta - x_eta y_xi (signed), a = (y_eta, -x_eta), b = (-y_xi, x_xi),
     grad xi = a / J, grad eta = b / J, K^{ab} = grad a . K grad b,
     alpha = K^{xixi}, beta = 2 K^{xieta}, gamma = K^{etaeta},
     c_xi  = (1/J) [d_xi (a.Ka / J) + d_eta (a.Kb / J)],
     c_eta = (1/J) [d_xi (a.Kb / J) + d_eta (b.Kb / J)],
     nu = a.v / J - c_xi, omega = b.v / J - c_eta, phi = f - div v. */

static double qf(const double K[3], const double p[2], const double q[2])
{
    return p[0] * (K[0] * q[0] + K[1] * q[1]) + p[1] * (K[1] * q[0] + K[2] * q[1]);
}

void orc_coeffs(const orc_problem* P, double xi, double eta, double* out)
{
    double m[12];
    orc_map(P, xi, eta, m);
    double x = m[0], y = m[1];
    double xa = m[2], xb = m[3], ya = m[4], yb = m[5];          /* a = xi, b = eta */
    double xaa = m[6], xab = m[7], xbb = m[8], yaa = m[9], yab = m[10], ybb = m[11];
    double ph[13];
    orc_physical(P, x, y, ph);
    double K[3] = { ph[0], ph[1], ph[2] };
    double Kx[3] = { ph[3], ph[4], ph[5] };
    double Ky[3] = { ph[6], ph[7], ph[8] };
    double Kxi[3], Keta[3];
    for (int c = 0; c < 3; ++c) {
        Kxi[c] = Kx[c] * xa + Ky[c] * ya;
        Keta[c] = Kx[c] * xb + Ky[c] * yb;
    }
    double J = xa * yb - xb * ya;
    double Jxi = xaa * yb + xa * yab - xab * ya - xb * yaa;
    double Jeta = xab * yb + xa * ybb - xbb * ya - xb * yab;
    double a[2] = { yb, -xb }, b[2] = { -ya, xa };
    double a_xi[2] = { yab, -xab }, a_eta[2] = { ybb, -xbb };
    double b_xi[2] = { -yaa, xaa }, b_eta[2] = { -yab, xab };

    double Kaa = qf(K, a, a), Kab = qf(K, a, b), Kbb = qf(K, b, b);
    /* d_xi (a.Ka / J) */
    double t1 = (2.0 * qf(K, a_xi, a) + qf(Kxi, a, a)) / J - Kaa * Jxi / (J * J);
    /* d_eta (a.Kb / J) */
    double t2 = (qf(K, a_eta, b) + qf(K, a, b_eta) + qf(Keta, a, b)) / J - Kab * Jeta / (J * J);
    /* d_xi (a.Kb / J) */
    double t3 = (qf(K, a_xi, b) + qf(K, a, b_xi) + qf(Kxi, a, b)) / J - Kab * Jxi / (J * J);
    /* d_eta (b.Kb / J) */
    double t4 = (2.0 * qf(K, b_eta, b) + qf(Keta, b, b)) / J - Kbb * Jeta / (J * J);
    double c_xi = (t1 + t2) / J;
    double c_eta = (t3 + t4) / J;
    double v[2] = { ph[9], ph[10] };
    double Vxi = (a[0] * v[0] + a[1] * v[1]) / J;
    double Veta = (b[0] * v[0] + b[1] * v[1]) / J;

    out[0] = Kaa / (J * J);
    out[1] = 2.0 * Kab / (J * J);
    out[2] = Kbb / (J * J);
    out[3] = Vxi - c_xi;
    out[4] = Veta - c_eta;
    out[5] = ph[12] - ph[11];
    out[6] = source_G(P, x, y);
}

/* ------------------------------------------------------------------------- */
/* micro geometry of patch (i,j): Section 3, patch [xi_i - h/2, xi_i + h/2] with
   n = m - 1 equal nano steps */

typedef struct {
    int i, j;
    double xc, yc;    /* centre (xi_i, eta_j) */
    double hx, hy;    /* patch widths */
    double dx, dy;    /* nano steps */
    double Dx, Dy;    /* macro steps */
    int mx, my;
} patch_geo;

static patch_geo patch_of(const orc_problem* P, int p)
{
    patch_geo g;
    int nc = n_cols(P);
    g.i = i_first(P) + p % nc;
    g.j = 1 + p / nc;
    g.Dx = d_xi(P); g.Dy = d_eta(P);
    g.xc = P->xi0 + g.i * g.Dx;
    g.yc = P->eta0 + g.j * g.Dy;
    g.hx = P->h_ratio_xi * g.Dx;
    g.hy = P->h_ratio_eta * g.Dy;
    g.mx = P->m_xi; g.my = P->m_eta;
    g.dx = g.hx / (g.mx - 1);
    g.dy = g.hy / (g.my - 1);
    return g;
}

void orc_micro_coords(const orc_problem* P, double* xi, double* eta)
{
    int np = orc_n_patch(P);
    for (int p = 0; p < np; ++p) {
        patch_geo g = patch_of(P, p);
        for (int b = 0; b < g.my; ++b)
            for (int a = 0; a < g.mx; ++a) {
                size_t o = (size_t)p * g.mx * g.my + (size_t)b * g.mx + a;
                xi[o] = g.xc - 0.5 * g.hx + a * g.dx;
                eta[o] = g.yc - 0.5 * g.hy + b * g.dy;
            }
    }
}

/* coefficients of every micro point of one patch: c[(b*mx+a)*7 + k] */
static void patch_coeffs(const orc_problem* P, const patch_geo* g, double* c)
{
    for (int b = 0; b < g->my; ++b)
        for (int a = 0; a < g->mx; ++a) {
            double xa = g->xc - 0.5 * g->hx + a * g->dx;
            double yb = g->yc - 0.5 * g->hy + b * g->dy;
            orc_coeffs(P, xa, yb, c + 7 * (b * g->mx + a));
        }
}

/* ------------------------------------------------------------------------- */
/* Step sizes.  Reading G8: one micro step per instance, cfl times the smallest
   explicit forward-Euler bound over all patch micro points.  Reading G9: macro
   step = half the explicit bound of the same operator on the macro spacing,
   evaluated at the patch centres. */

static double rate_bound(const orc_problem* P, const double* c, double hx, double hy)
{
    double r = 2.0 * fabs(c[0]) / (hx * hx) + 2.0 * fabs(c[2]) / (hy * hy)
             + fabs(c[1]) / (hx * hy) + fabs(c[5]);
    if (P->conv == ORC_CONV_UPWIND) r += fabs(c[3]) / hx + fabs(c[4]) / hy;
    return r;
}

double orc_dt_micro(const orc_problem* P)
{
    if (P->dt_micro_fixed > 0.0) return P->dt_micro_fixed;
    int np = orc_n_patch(P);
    double rmax = 0.0;
    double* c = (double*)malloc(sizeof(double) * 7 * P->m_xi * P->m_eta);
    for (int p = 0; p < np; ++p) {
        patch_geo g = patch_of(P, p);
        patch_coeffs(P, &g, c);
        for (int q = 0; q < g.mx * g.my; ++q) {
            double r = rate_bound(P, c + 7 * q, g.dx, g.dy);
            if (r > rmax) rmax = r;
        }
    }
    free(c);
    return P->cfl_micro / rmax;
}

double orc_dt_macro(const orc_problem* P)
{
    int np = orc_n_patch(P);
    double rmax = 0.0, c[7];
    for (int p = 0; p < np; ++p) {
        patch_geo g = patch_of(P, p);
        orc_coeffs(P, g.xc, g.yc, c);
        double r = 2.0 * fabs(c[0]) / (g.Dx * g.Dx) + 2.0 * fabs(c[2]) / (g.Dy * g.Dy)
                 + fabs(c[1]) / (g.Dx * g.Dy) + fabs(c[3]) / g.Dx + fabs(c[4]) / g.Dy
                 + fabs(c[5]);
        if (r > rmax) rmax = r;
    }
    return 0.5 / rmax;
}

/* ------------------------------------------------------------------------- */
/* Bessel cross products for the annulus (eq. (Annulus_AS)): Z_k(mu r) =
   J_k(mu ra) Y_k(mu r) - Y_k(mu ra) J_k(mu r); mu are the positive roots of
   Z_k(mu rb) = 0.  Roots by sign scan + bisection on libm's jn / yn. */

double orc_bessel_Z(int k, double mu, double ra, double r)
{
    return jn(k, mu * ra) * yn(k, mu * r) - yn(k, mu * ra) * jn(k, mu * r);
}

double orc_bessel_root(int k, double ra, double rb, int which)
{
    double step = 0.01 * M_PI / (rb - ra);
    double lo = step, flo = orc_bessel_Z(k, lo, ra, rb);
    int found = 0;
    for (int it = 0; it < 1000000; ++it) {
        double hi = lo + step, fhi = orc_bessel_Z(k, hi, ra, rb);
        if ((flo < 0.0) != (fhi < 0.0)) {
            if (++found == which) {
                double a = lo, b = hi, fa = flo;
                for (int bi = 0; bi < 200; ++bi) {
                    double mid = 0.5 * (a + b);
                    double fm = orc_bessel_Z(k, mid, ra, rb);
                    if ((fm < 0.0) == (fa < 0.0)) { a = mid; fa = fm; } else b = mid;
                    if (b - a <= 1e-15 * b) break;
                }
                return 0.5 * (a + b);
            }
        }
        lo = hi; flo = fhi;
    }
    return NAN;
}

/* ------------------------------------------------------------------------- */
/* initial and exact fields at the macro nodes */

void orc_init_field(const orc_problem* P, int kind, const double* prm, double t, double* U)
{
    int nx = n_xpts(P), ny = P->n_eta + 1;
    double Dx = d_xi(P), Dy = d_eta(P);
    double mu[8] = { 0 };
    if (kind == ORC_INIT_BESSEL) {
        int nm = (int)prm[0];
        for (int k = 1; k <= nm && k <= 8; ++k) mu[k - 1] = orc_bessel_root(k, prm[1], prm[2], 1);
    }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double xi = P->xi0 + i * Dx, eta = P->eta0 + j * Dy;
            double m[12];
            orc_map(P, xi, eta, m);
            double val = 0.0;
            switch (kind) {
            case ORC_INIT_EXACT: val = orc_exact(P, m[0], m[1], t); break;
            case ORC_INIT_BESSEL: {
                /* sum_k a_k Z_k(mu_k r) cos(k theta) exp(-d0 mu_k^2 t);
                   prm = {n_modes, ra, rb, a_1, ..., a_n} */
                int nm = (int)prm[0];
                double r = sqrt(m[0] * m[0] + m[1] * m[1]);
                double th = atan2(m[1], m[0]);
                for (int k = 1; k <= nm && k <= 8; ++k)
                    val += prm[2 + k] * orc_bessel_Z(k, mu[k - 1], prm[1], r) * cos(k * th)
                         * exp(-P->d0 * mu[k - 1] * mu[k - 1] * t);
                break;
            }
            case ORC_INIT_ANNULUS_POLY: {
                /* initial condition of Section 4.2: (r - ra)(rb - r) sin(theta);
                   prm = {ra, rb} */
                double r = sqrt(m[0] * m[0] + m[1] * m[1]);
                double th = atan2(m[1], m[0]);
                val = (r - prm[0]) * (prm[1] - r) * sin(th);
                break;
            }
            case ORC_INIT_BUMP: {
                double zx = (xi - P->xi0) / (P->xi1 - P->xi0);
                double zy = (eta - P->eta0) / (P->eta1 - P->eta0);
                double fx = P->periodic_xi ? (1.0 + 0.5 * cos(xi)) : sin(M_PI * zx);
                val = fx * sin(M_PI * zy);
                break;
            }
            default: val = 0.0;
            }
            U[j * nx + i] = val;
        }
}

/* ------------------------------------------------------------------------- */
/* Section 3.1: Lagrange fundamental polynomial of degree 2 over the nodes
   {-D, 0, +D} (offsets from the patch centre), index q in {0,1,2} <-> {-1,0,+1}. */
static double lagrange(int q, double s, double D)
{
    double nodes[3] = { -D, 0.0, D };
    double v = 1.0;
    for (int r = 0; r < 3; ++r)
        if (r != q) v *= (s - nodes[r]) / (nodes[q] - nodes[r]);
    return v;
}

/* extended (ghosted) micro grid of one patch: a in [-1, mx], b in [-1, my] */
#define EXT(u, a, b, mx) (u)[((b) + 1) * ((mx) + 2) + ((a) + 1)]

typedef struct {
    double st[3][3];                 /* st[p+1][q+1] = U_{i+p, j+q} */
    double gL[ORC_MAXM + 2], gR[ORC_MAXM + 2]; /* index b+1, b = -1..my */
    double gB[ORC_MAXM + 2], gT[ORC_MAXM + 2]; /* index a+1, a = -1..mx */
} patch_edge;

/* Eq. (edge): Neumann data on the four patch edges from the interpolant (9 macro
   values), held fixed over the burst (Q = 1). */
static void edge_data(const orc_problem* P, const double* U, const patch_geo* g, patch_edge* e)
{
    for (int p = -1; p <= 1; ++p)
        for (int q = -1; q <= 1; ++q) e->st[p + 1][q + 1] = macro_U(P, U, g->i + p, g->j + q);
    double rx = g->hx / (2.0 * g->Dx), ry = g->hy / (2.0 * g->Dy);
    for (int b = -1; b <= g->my; ++b) {
        double t = -0.5 * g->hy + b * g->dy;
        double A[3];
        for (int p = 0; p < 3; ++p) {
            A[p] = 0.0;
            for (int q = 0; q < 3; ++q) A[p] += lagrange(q, t, g->Dy) * e->st[p][q];
        }
        /* at xi_i - h/2 (lower signs) and xi_i + h/2 (upper signs) */
        e->gL[b + 1] = ((-0.5 - rx) * A[0] + 2.0 * rx * A[1] + (0.5 - rx) * A[2]) / g->Dx;
        e->gR[b + 1] = ((-0.5 + rx) * A[0] - 2.0 * rx * A[1] + (0.5 + rx) * A[2]) / g->Dx;
    }
    for (int a = -1; a <= g->mx; ++a) {
        double s = -0.5 * g->hx + a * g->dx;
        double B[3];
        for (int q = 0; q < 3; ++q) {
            B[q] = 0.0;
            for (int p = 0; p < 3; ++p) B[q] += lagrange(p, s, g->Dx) * e->st[p][q];
        }
        e->gB[a + 1] = ((-0.5 - ry) * B[0] + 2.0 * ry * B[1] + (0.5 - ry) * B[2]) / g->Dy;
        e->gT[a + 1] = ((-0.5 + ry) * B[0] - 2.0 * ry * B[1] + (0.5 + ry) * B[2]) / g->Dy;
    }
}

/* Eqs. (Lifting), (C_0) with central macro differences (reading G3). */
static void lift_patch(const patch_geo* g, const patch_edge* e, double* u0ext)
{
    double (*S)[3] = (double (*)[3])e->st;
    double U0 = S[1][1];
    double Ux = (S[2][1] - S[0][1]) / (2.0 * g->Dx);
    double Uy = (S[1][2] - S[1][0]) / (2.0 * g->Dy);
    double Uxx = (S[2][1] - 2.0 * S[1][1] + S[0][1]) / (g->Dx * g->Dx);
    double Uyy = (S[1][2] - 2.0 * S[1][1] + S[1][0]) / (g->Dy * g->Dy);
    double Uxy = (S[2][2] - S[2][0] - S[0][2] + S[0][0]) / (4.0 * g->Dx * g->Dy);
    double C0 = U0 - g->hx * g->hx * Uxx / 24.0 - g->hy * g->hy * Uyy / 24.0;
    for (int b = 0; b < g->my; ++b)
        for (int a = 0; a < g->mx; ++a) {
            double s = -0.5 * g->hx + a * g->dx;
            double t = -0.5 * g->hy + b * g->dy;
            EXT(u0ext, a, b, g->mx) = C0 + (s * Ux + t * Uy)
                                    + 0.5 * (s * s * Uxx + 2.0 * s * t * Uxy + t * t * Uyy);
        }
}

/* Reading G5: second-order ghost points for the Neumann data, eta ghost rows
   first (a = 0..n), then xi ghost columns over b = -1..n+1.  zero_data = 1
   gives the homogeneous mirror used for the split departure. */
static void fill_ghosts(const patch_geo* g, const patch_edge* e, double* u, int zero_data)
{
    int nx = g->mx - 1, ny = g->my - 1;
    for (int a = 0; a <= nx; ++a) {
        double gb = zero_data ? 0.0 : e->gB[a + 1];
        double gt = zero_data ? 0.0 : e->gT[a + 1];
        EXT(u, a, -1, g->mx) = EXT(u, a, 1, g->mx) - 2.0 * g->dy * gb;
        EXT(u, a, ny + 1, g->mx) = EXT(u, a, ny - 1, g->mx) + 2.0 * g->dy * gt;
    }
    for (int b = -1; b <= ny + 1; ++b) {
        double gl = zero_data ? 0.0 : e->gL[b + 1];
        double gr = zero_data ? 0.0 : e->gR[b + 1];
        EXT(u, -1, b, g->mx) = EXT(u, 1, b, g->mx) - 2.0 * g->dx * gl;
        EXT(u, nx + 1, b, g->mx) = EXT(u, nx - 1, b, g->mx) + 2.0 * g->dx * gr;
    }
}

/* Micro finite differences (Section 4.1 text): 3-point central for the second
   derivatives, the 4-point cross difference for u_xieta, and for the first
   derivatives the 2-point upwind difference taken against the sign of the
   coefficient (backward for positive nu), or 3-point central. */
static double op_at(const orc_problem* P, const patch_geo* g, const double* c,
                    const double* u, int a, int b)
{
    int mx = g->mx;
    double uc = EXT(u, a, b, mx);
    double uE = EXT(u, a + 1, b, mx), uW = EXT(u, a - 1, b, mx);
    double uN = EXT(u, a, b + 1, mx), uS = EXT(u, a, b - 1, mx);
    double uxx = (uE - 2.0 * uc + uW) / (g->dx * g->dx);
    double uyy = (uN - 2.0 * uc + uS) / (g->dy * g->dy);
    double uxy = (EXT(u, a + 1, b + 1, mx) - EXT(u, a + 1, b - 1, mx)
                - EXT(u, a - 1, b + 1, mx) + EXT(u, a - 1, b - 1, mx)) / (4.0 * g->dx * g->dy);
    double nu = c[3], om = c[4];
    double ux, uy;
    if (P->conv == ORC_CONV_CENTRAL) {
        ux = (uE - uW) / (2.0 * g->dx);
        uy = (uN - uS) / (2.0 * g->dy);
    } else {
        ux = nu > 0.0 ? (uc - uW) / g->dx : (uE - uc) / g->dx;
        uy = om > 0.0 ? (uc - uS) / g->dy : (uN - uc) / g->dy;
    }
    return c[0] * uxx + c[1] * uxy + c[2] * uyy - nu * ux - om * uy + c[5] * uc;
}

/* Trapezoid average of the lifted field minus U_ij (reading G4, MACRO
   reference): by eqs. (Lifting), (C_0) and the trapezoid rule on the nano grid
   it equals (dxi^2 U_xixi + deta^2 U_etaeta) / 12 exactly (the lift's
   continuous average is U_ij; the trapezoid rule adds d^2/12 times the second
   derivative).  The split form uses this closed form, so that no difference of
   two nearly equal averages is formed for small patches. */
static double lift_trapezoid_bias(const patch_geo* g, const patch_edge* e)
{
    const double (*S)[3] = (const double (*)[3])e->st;
    double Uxx = (S[2][1] - 2.0 * S[1][1] + S[0][1]) / (g->Dx * g->Dx);
    double Uyy = (S[1][2] - 2.0 * S[1][1] + S[1][0]) / (g->Dy * g->Dy);
    return (g->dx * g->dx * Uxx + g->dy * g->dy * Uyy) / 12.0;
}

/* composite trapezoid average over the patch (eq. (Restriction), Section 4.1) */
static double trapezoid(const patch_geo* g, const double* u)
{
    int nx = g->mx - 1, ny = g->my - 1;
    double s = 0.0;
    for (int b = 0; b <= ny; ++b)
        for (int a = 0; a <= nx; ++a) {
            double wa = (a == 0 || a == nx) ? 0.5 : 1.0;
            double wb = (b == 0 || b == ny) ? 0.5 : 1.0;
            s += wa * wb * EXT(u, a, b, g->mx);
        }
    return s / ((double)nx * ny);
}

/* ------------------------------------------------------------------------- */
/* ADI micro solver.  Section 4.1 runs the micro simulations with an alternating
   direction implicit scheme and two nano steps per burst but does not print
   the scheme.  Reading: Peaceman-Rachford splitting of the micro operator of
   op_at into line parts
     Lx u = alpha u_xixi - nu u_xi + phi u / 2   (along xi),
     Ly u = gamma u_etaeta - omega u_eta + phi u / 2   (along eta),
     Lc u = beta u_xieta   (mixed part, always explicit),
   with the same differences and ghost points as the explicit scheme, and the
   source g taken at the middle of the step:
     (I - dt/2 Lx) u*      = u^k + dt/2 (Ly u^k + Lc u^k + g(t_k + dt/2)),
     (I - dt/2 Ly) u^{k+1} = u*  + dt/2 (Lx u* + Lc u* + g(t_k + dt/2)).
   Each line operator is affine (the ghost points carry the edge data); it is
   assembled column by column from its values on unit vectors, and each line
   system is solved by Gaussian elimination with partial pivoting. */

/* part dir of the micro operator at (a, b): 0 = Lx, 1 = Ly, 2 = Lc */
static double op_part(const orc_problem* P, const patch_geo* g, const double* c,
                      const double* u, int a, int b, int dir)
{
    int mx = g->mx;
    double uc = EXT(u, a, b, mx);
    if (dir == 0) {
        double uE = EXT(u, a + 1, b, mx), uW = EXT(u, a - 1, b, mx);
        double uxx = (uE - 2.0 * uc + uW) / (g->dx * g->dx);
        double ux;
        if (P->conv == ORC_CONV_CENTRAL) ux = (uE - uW) / (2.0 * g->dx);
        else ux = c[3] > 0.0 ? (uc - uW) / g->dx : (uE - uc) / g->dx;
        return c[0] * uxx - c[3] * ux + 0.5 * c[5] * uc;
    }
    if (dir == 1) {
        double uN = EXT(u, a, b + 1, mx), uS = EXT(u, a, b - 1, mx);
        double uyy = (uN - 2.0 * uc + uS) / (g->dy * g->dy);
        double uy;
        if (P->conv == ORC_CONV_CENTRAL) uy = (uN - uS) / (2.0 * g->dy);
        else uy = c[4] > 0.0 ? (uc - uS) / g->dy : (uN - uc) / g->dy;
        return c[2] * uyy - c[4] * uy + 0.5 * c[5] * uc;
    }
    double uxy = (EXT(u, a + 1, b + 1, mx) - EXT(u, a + 1, b - 1, mx)
                - EXT(u, a - 1, b + 1, mx) + EXT(u, a - 1, b - 1, mx)) / (4.0 * g->dx * g->dy);
    return c[1] * uxy;
}

/* ghost points of one line only (row b for dir 0, column a for dir 1), as in
   fill_ghosts */
static void line_ghosts(const patch_geo* g, const patch_edge* e, double* u, int dir, int line, int zero_data)
{
    int nx = g->mx - 1, ny = g->my - 1;
    if (dir == 0) {
        double gl = zero_data ? 0.0 : e->gL[line + 1];
        double gr = zero_data ? 0.0 : e->gR[line + 1];
        EXT(u, -1, line, g->mx) = EXT(u, 1, line, g->mx) - 2.0 * g->dx * gl;
        EXT(u, nx + 1, line, g->mx) = EXT(u, nx - 1, line, g->mx) + 2.0 * g->dx * gr;
    } else {
        double gb = zero_data ? 0.0 : e->gB[line + 1];
        double gt = zero_data ? 0.0 : e->gT[line + 1];
        EXT(u, line, -1, g->mx) = EXT(u, line, 1, g->mx) - 2.0 * g->dy * gb;
        EXT(u, line, ny + 1, g->mx) = EXT(u, line, ny - 1, g->mx) + 2.0 * g->dy * gt;
    }
}

/* dense Gaussian elimination with partial pivoting: A (n x n, row-major) is
   overwritten, x holds the right-hand side on entry and the solution on exit */
static void solve_dense(int n, double* A, double* x)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[r * n + k]) > fabs(A[piv * n + k])) piv = r;
        if (piv != k) {
            for (int c = 0; c < n; ++c) {
                double t = A[k * n + c]; A[k * n + c] = A[piv * n + c]; A[piv * n + c] = t;
            }
            double t = x[k]; x[k] = x[piv]; x[piv] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double f = A[r * n + k] / A[k * n + k];
            for (int c = k; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
            x[r] -= f * x[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = x[k];
        for (int c = k + 1; c < n; ++c) s -= A[k * n + c] * x[c];
        x[k] = s / A[k * n + k];
    }
}

/* (I - h L_dir) x = rhs + h L_dir(0) on one line; rhs and the result are the
   line's values of the [my][mx] array rhs and of the ghosted array out */
static void line_solve(const orc_problem* P, const patch_geo* g, const patch_edge* e, const double* coef,
                       int zero_data, int dir, int line, double h, const double* rhs, double* out,
                       double* t)
{
    int mx = g->mx, n = dir == 0 ? g->mx : g->my;
    double A[ORC_MAXM * ORC_MAXM], x[ORC_MAXM];
    /* the constant part: the operator on the zero line with the edge data */
    for (int q = 0; q < n; ++q) {
        if (dir == 0) EXT(t, q, line, mx) = 0.0; else EXT(t, line, q, mx) = 0.0;
    }
    line_ghosts(g, e, t, dir, line, zero_data);
    for (int q = 0; q < n; ++q) {
        int a = dir == 0 ? q : line, b = dir == 0 ? line : q;
        x[q] = rhs[b * mx + a] + h * op_part(P, g, coef + 7 * (b * mx + a), t, a, b, dir);
    }
    /* the linear part, column k from the unit vector e_k with zero edge data */
    for (int k = 0; k < n; ++k) {
        for (int q = 0; q < n; ++q) {
            double v = q == k ? 1.0 : 0.0;
            if (dir == 0) EXT(t, q, line, mx) = v; else EXT(t, line, q, mx) = v;
        }
        line_ghosts(g, e, t, dir, line, 1);
        for (int q = 0; q < n; ++q) {
            int a = dir == 0 ? q : line, b = dir == 0 ? line : q;
            A[q * n + k] = (q == k ? 1.0 : 0.0) - h * op_part(P, g, coef + 7 * (b * mx + a), t, a, b, dir);
        }
    }
    solve_dense(n, A, x);
    for (int q = 0; q < n; ++q) {
        if (dir == 0) EXT(out, q, line, mx) = x[q]; else EXT(out, line, q, mx) = x[q];
    }
}

/* One ADI step from t_k of size dt on the ghosted array u (in/out).  Split
   form (r0 != NULL): departure with zero edge data and forcing
   r0 + (s(t) - s(T)) G; literal form: full field with the edge data and
   forcing s(t) G.  us, rhs and t are scratch arrays. */
static void adi_step(const orc_problem* P, const patch_geo* g, const patch_edge* e, const double* coef,
                     double amp, const double* r0, double sT, double tk, double dt,
                     double* u, double* us, double* rhs, double* t)
{
    int mx = g->mx, my = g->my;
    int zero_data = r0 != NULL;
    double h = 0.5 * dt;
    double sm = orc_time_factor(P, tk + h);
    /* first half step: explicit in eta and the mixed part, implicit along xi */
    fill_ghosts(g, e, u, zero_data);
    for (int b = 0; b < my; ++b)
        for (int a = 0; a < mx; ++a) {
            const double* c = coef + 7 * (b * mx + a);
            double f = r0 ? r0[b * mx + a] + (sm - sT) * amp * c[6] : sm * amp * c[6];
            rhs[b * mx + a] = EXT(u, a, b, mx)
                + h * (op_part(P, g, c, u, a, b, 1) + op_part(P, g, c, u, a, b, 2) + f);
        }
    for (int b = 0; b < my; ++b) line_solve(P, g, e, coef, zero_data, 0, b, h, rhs, us, t);
    /* second half step: explicit in xi and the mixed part, implicit along eta */
    fill_ghosts(g, e, us, zero_data);
    for (int b = 0; b < my; ++b)
        for (int a = 0; a < mx; ++a) {
            const double* c = coef + 7 * (b * mx + a);
            double f = r0 ? r0[b * mx + a] + (sm - sT) * amp * c[6] : sm * amp * c[6];
            rhs[b * mx + a] = EXT(us, a, b, mx)
                + h * (op_part(P, g, c, us, a, b, 0) + op_part(P, g, c, us, a, b, 2) + f);
        }
    for (int a = 0; a < mx; ++a) line_solve(P, g, e, coef, zero_data, 1, a, h, rhs, u, t);
}

/* The split-form micro solve (departure w = u - u0 in the ghosted array u,
   mirror ghosts, forcing r0 = L_h(u0) + s(T) G): K steps of forward Euler or
   of the ADI scheme.  un is scratch of the same size. */
static void micro_split(const orc_problem* P, const patch_geo* g, const patch_edge* e, const double* coef,
                        double amp, const double* r0, double T, int K, double dt, double* u, double* un)
{
    int mx = g->mx, my = g->my, nx = mx - 1, ny = my - 1;
    double sT = orc_time_factor(P, T);
    if (P->micro == ORC_MICRO_ADI) {
        int ne = (mx + 2) * (my + 2);
        double* rhs = (double*)calloc((size_t)mx * my, sizeof(double));
        double* t = (double*)calloc((size_t)ne, sizeof(double));
        for (int k = 0; k < K; ++k) adi_step(P, g, e, coef, amp, r0, sT, T + k * dt, dt, u, un, rhs, t);
        free(rhs); free(t);
        return;
    }
    for (int k = 0; k < K; ++k) {
        double tk = T + k * dt;
        double dsk = orc_time_factor(P, tk) - sT;
        fill_ghosts(g, e, u, 1);
        for (int b = 0; b <= ny; ++b)
            for (int a = 0; a <= nx; ++a) {
                const double* c = coef + 7 * (b * mx + a);
                EXT(un, a, b, mx) = EXT(u, a, b, mx)
                    + dt * (op_at(P, g, c, u, a, b) + r0[b * mx + a] + dsk * amp * c[6]);
            }
        for (int b = 0; b <= ny; ++b)
            for (int a = 0; a <= nx; ++a) EXT(u, a, b, mx) = EXT(un, a, b, mx);
    }
}

/* One patch through S1-S4 (gap-tooth steps (i)-(iv)).  Returns dU = U^1 - U^0;
   optionally writes the burst result (w or u) and the lift / forcing. */
typedef struct {
    double* u0;     /* [my][mx] or NULL */
    double* edge;   /* [4][m+2] or NULL */
    double* r0;     /* [my][mx] or NULL */
    double* out;    /* [my][mx] or NULL */
} patch_out;

static double run_patch(const orc_problem* P, const double* U, int p, const double* coef,
                        double T, int K, double dt, int form, patch_out* po)
{
    patch_geo g = patch_of(P, p);
    int mx = g.mx, my = g.my, nx = mx - 1, ny = my - 1;
    int ne = (mx + 2) * (my + 2);
    double* u0 = (double*)calloc((size_t)ne, sizeof(double));
    double* u = (double*)calloc((size_t)ne, sizeof(double));
    double* un = (double*)calloc((size_t)ne, sizeof(double));
    double* r0 = (double*)calloc((size_t)mx * my, sizeof(double));
    patch_edge e;
    edge_data(P, U, &g, &e);
    lift_patch(&g, &e, u0);
    fill_ghosts(&g, &e, u0, 0);
    double amp = (P->src == ORC_SRC_GAUSS_PATCH && P->src_amp) ? P->src_amp[p] : 1.0;
    double sT = orc_time_factor(P, T);

    if (form == ORC_FORM_LITERAL && P->micro == ORC_MICRO_ADI) {
        memcpy(u, u0, sizeof(double) * ne);
        double* rhs = (double*)calloc((size_t)mx * my, sizeof(double));
        double* t = (double*)calloc((size_t)ne, sizeof(double));
        for (int k = 0; k < K; ++k) adi_step(P, &g, &e, coef, amp, NULL, sT, T + k * dt, dt, u, un, rhs, t);
        free(rhs); free(t);
    } else if (form == ORC_FORM_LITERAL) {
        memcpy(u, u0, sizeof(double) * ne);
        for (int k = 0; k < K; ++k) {
            double tk = T + k * dt;
            double sk = orc_time_factor(P, tk);
            fill_ghosts(&g, &e, u, 0);
            for (int b = 0; b <= ny; ++b)
                for (int a = 0; a <= nx; ++a) {
                    const double* c = coef + 7 * (b * mx + a);
                    EXT(un, a, b, mx) = EXT(u, a, b, mx)
                        + dt * (op_at(P, &g, c, u, a, b) + sk * amp * c[6]);
                }
            for (int b = 0; b <= ny; ++b)
                for (int a = 0; a <= nx; ++a) EXT(u, a, b, mx) = EXT(un, a, b, mx);
        }
    } else {
        /* split form: u = u0 + w, w^0 = 0, homogeneous mirror ghosts for w,
           r0 = L_h(u0) + g(T); exact rewriting of the forward-Euler recursion
           because the edge data and u0 are fixed over the burst */
        for (int b = 0; b <= ny; ++b)
            for (int a = 0; a <= nx; ++a) {
                const double* c = coef + 7 * (b * mx + a);
                r0[b * mx + a] = op_at(P, &g, c, u0, a, b) + sT * amp * c[6];
            }
        micro_split(P, &g, &e, coef, amp, r0, T, K, dt, u, un);
    }

    /* Restriction (step (iv)) and the reference value U^0 (reading G4):
       LIFTED: U^0 = trapezoid average of the lifted field; MACRO: U^0 = U_ij. */
    double dU;
    double Uij = e.st[1][1];
    if (form == ORC_FORM_LITERAL) {
        double U1 = trapezoid(&g, u);
        dU = U1 - (P->restrict_mode == ORC_RESTRICT_MACRO ? Uij : trapezoid(&g, u0));
    } else {
        dU = trapezoid(&g, u);
        if (P->restrict_mode == ORC_RESTRICT_MACRO) dU += lift_trapezoid_bias(&g, &e);
    }

    if (po) {
        for (int b = 0; b < my; ++b)
            for (int a = 0; a < mx; ++a) {
                if (po->u0) po->u0[b * mx + a] = EXT(u0, a, b, mx);
                if (po->r0) po->r0[b * mx + a] = r0[b * mx + a];
                if (po->out) po->out[b * mx + a] = EXT(u, a, b, mx);
            }
        if (po->edge) {
            int me = (mx > my ? mx : my) + 2;
            for (int q = 0; q < my + 2; ++q) { po->edge[0 * me + q] = e.gL[q]; po->edge[1 * me + q] = e.gR[q]; }
            for (int q = 0; q < mx + 2; ++q) { po->edge[2 * me + q] = e.gB[q]; po->edge[3 * me + q] = e.gT[q]; }
        }
    }
    free(u0); free(u); free(un); free(r0);
    return dU;
}

static double* all_coeffs(const orc_problem* P)
{
    int np = orc_n_patch(P), mm = P->m_xi * P->m_eta;
    double* c = (double*)malloc(sizeof(double) * 7 * (size_t)mm * np);
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < np; ++p) {
        patch_geo g = patch_of(P, p);
        patch_coeffs(P, &g, c + (size_t)7 * mm * p);
    }
    return c;
}

void orc_lift(const orc_problem* P, const double* U, double* u0, double* edge)
{
    int np = orc_n_patch(P), mm = P->m_xi * P->m_eta;
    int me = (P->m_xi > P->m_eta ? P->m_xi : P->m_eta) + 2;
    double* coef = all_coeffs(P);
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < np; ++p) {
        patch_out po = { u0 ? u0 + (size_t)mm * p : NULL, edge ? edge + (size_t)4 * me * p : NULL, NULL, NULL };
        run_patch(P, U, p, coef + (size_t)7 * mm * p, 0.0, 0, 1.0, ORC_FORM_SPLIT, &po);
    }
    free(coef);
}

void orc_forcing(const orc_problem* P, const double* U, double t, double* r0)
{
    int np = orc_n_patch(P), mm = P->m_xi * P->m_eta;
    double* coef = all_coeffs(P);
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < np; ++p) {
        patch_out po = { NULL, NULL, r0 + (size_t)mm * p, NULL };
        run_patch(P, U, p, coef + (size_t)7 * mm * p, t, 0, 1.0, ORC_FORM_SPLIT, &po);
    }
    free(coef);
}

void orc_burst(const orc_problem* P, const double* U, double t, int k, double dt, int form, double* out)
{
    int np = orc_n_patch(P), mm = P->m_xi * P->m_eta;
    double* coef = all_coeffs(P);
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < np; ++p) {
        patch_out po = { NULL, NULL, NULL, out + (size_t)mm * p };
        run_patch(P, U, p, coef + (size_t)7 * mm * p, t, k, dt, form, &po);
    }
    free(coef);
}

void orc_restrict(const orc_problem* P, const double* U, const double* bo, int form, double* dU)
{
    int np = orc_n_patch(P), mm = P->m_xi * P->m_eta;
    double* coef = all_coeffs(P);
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < np; ++p) {
        patch_geo g = patch_of(P, p);
        int mx = g.mx, my = g.my;
        int ne = (mx + 2) * (my + 2);
        double* u = (double*)calloc((size_t)ne, sizeof(double));
        double* u0 = (double*)calloc((size_t)ne, sizeof(double));
        patch_edge e;
        edge_data(P, U, &g, &e);
        lift_patch(&g, &e, u0);
        for (int b = 0; b < my; ++b)
            for (int a = 0; a < mx; ++a) EXT(u, a, b, mx) = bo[(size_t)mm * p + b * mx + a];
        double Uij = e.st[1][1];
        double d;
        if (form == ORC_FORM_LITERAL)
            d = trapezoid(&g, u) - (P->restrict_mode == ORC_RESTRICT_MACRO ? Uij : trapezoid(&g, u0));
        else {
            d = trapezoid(&g, u);
            if (P->restrict_mode == ORC_RESTRICT_MACRO) d += lift_trapezoid_bias(&g, &e);
        }
        dU[p] = d;
        free(u); free(u0);
    }
    free(coef);
}

/* Dirichlet data on the non-periodic boundary nodes at time t */
void orc_apply_bc(const orc_problem* P, double* U, double t)
{
    int nx = n_xpts(P), ny = P->n_eta + 1;
    double Dx = d_xi(P), Dy = d_eta(P);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int bnd = (j == 0 || j == ny - 1) || (!P->periodic_xi && (i == 0 || i == nx - 1));
            if (!bnd) continue;
            double m[12];
            orc_map(P, P->xi0 + i * Dx, P->eta0 + j * Dy, m);
            U[j * nx + i] = orc_exact(P, m[0], m[1], t);
        }
}

/* Eqs. (Time_Derivative), (Extrapolation): F = dU / tau, U += Delta t F on the
   interior nodes; then the boundary values at the new time. */
void orc_project(const orc_problem* P, double* U, const double* dU, double t, double dtm, double tau)
{
    int np = orc_n_patch(P), nx = n_xpts(P);
    for (int p = 0; p < np; ++p) {
        patch_geo g = patch_of(P, p);
        double F = dU[p] / tau;
        U[g.j * nx + g.i] = U[g.j * nx + g.i] + dtm * F;
    }
    orc_apply_bc(P, U, t + dtm);
}

/* Q > 1: the burst is cut into Q sub-bursts of K/Q forward-Euler steps.
   Section 3 keeps the edge data fixed over the whole burst (the Q = 1 case of
   the patch schemes it cites) and names refreshing them as the more accurate
   alternative.  Reading: before sub-burst q >= 1 the edge data of every patch
   are rebuilt by eq. (edge) from the macro estimate V_q, which is U plus each
   patch's restricted change of the departure so far on the interior nodes and
   the Dirichlet data at the sub-burst's start time T + q (K/Q) dt on the
   boundary nodes; the micro field goes on from its current state (no new
   lift).  In the split form the departure's ghost points carry the difference
   between the new and the lifted edge data.  The restricted change that
   enters the projection is that of the whole burst (plus the MACRO bias). */
static void step_refresh(const orc_problem* P, double* U, double t0, double dtm, int n_steps, double dt, int form)
{
    int np = orc_n_patch(P), mx = P->m_xi, my = P->m_eta, mm = mx * my, nx = mx - 1, ny = my - 1;
    int ne = (mx + 2) * (my + 2), Q = P->q_refresh, Ks = P->k_micro / Q;
    int nmac = orc_n_macro(P), nxp = n_xpts(P);
    double tau = P->k_micro * dt;
    double* coef = all_coeffs(P);
    double* u = (double*)calloc((size_t)np * ne, sizeof(double));
    double* u0 = (double*)calloc((size_t)np * ne, sizeof(double));
    double* r0 = (double*)calloc((size_t)np * mm, sizeof(double));
    patch_edge* e0 = (patch_edge*)calloc((size_t)np, sizeof(patch_edge));
    double* dR = (double*)calloc((size_t)np, sizeof(double));
    double* V = (double*)malloc(sizeof(double) * nmac);
    for (int s = 0; s < n_steps; ++s) {
        double T = t0 + s * dtm;
        double sT = orc_time_factor(P, T);
        #pragma omp parallel for schedule(static)
        for (int p = 0; p < np; ++p) {
            patch_geo g = patch_of(P, p);
            double* up = u + (size_t)p * ne;
            double* u0p = u0 + (size_t)p * ne;
            const double* c = coef + (size_t)7 * mm * p;
            double amp = (P->src == ORC_SRC_GAUSS_PATCH && P->src_amp) ? P->src_amp[p] : 1.0;
            memset(up, 0, sizeof(double) * ne);
            memset(u0p, 0, sizeof(double) * ne);
            edge_data(P, U, &g, &e0[p]);
            lift_patch(&g, &e0[p], u0p);
            fill_ghosts(&g, &e0[p], u0p, 0);
            for (int b = 0; b < my; ++b)
                for (int a = 0; a < mx; ++a) {
                    r0[(size_t)p * mm + b * mx + a] = op_at(P, &g, c + 7 * (b * mx + a), u0p, a, b) + sT * amp * c[7 * (b * mx + a) + 6];
                    if (form == ORC_FORM_LITERAL) EXT(up, a, b, mx) = EXT(u0p, a, b, mx);
                }
            dR[p] = 0.0;
        }
        for (int q = 0; q < Q; ++q) {
            double Tq = T + q * Ks * dt;
            /* the macro estimate at the start of sub-burst q */
            memcpy(V, U, sizeof(double) * nmac);
            if (q > 0) {
                for (int p = 0; p < np; ++p) {
                    patch_geo g = patch_of(P, p);
                    V[g.j * nxp + g.i] = U[g.j * nxp + g.i] + dR[p];
                }
                orc_apply_bc(P, V, Tq);
            }
            #pragma omp parallel for schedule(static)
            for (int p = 0; p < np; ++p) {
                patch_geo g = patch_of(P, p);
                double* up = u + (size_t)p * ne;
                double* un = (double*)calloc((size_t)ne, sizeof(double));
                const double* c = coef + (size_t)7 * mm * p;
                double amp = (P->src == ORC_SRC_GAUSS_PATCH && P->src_amp) ? P->src_amp[p] : 1.0;
                patch_edge eq;
                edge_data(P, V, &g, &eq);
                if (form == ORC_FORM_SPLIT) {
                    /* ghost data of the departure: new minus lifted edge data */
                    for (int k = 0; k < ORC_MAXM + 2; ++k) {
                        eq.gL[k] -= e0[p].gL[k]; eq.gR[k] -= e0[p].gR[k];
                        eq.gB[k] -= e0[p].gB[k]; eq.gT[k] -= e0[p].gT[k];
                    }
                }
                for (int k = 0; k < Ks; ++k) {
                    double tk = Tq + k * dt;
                    fill_ghosts(&g, &eq, up, 0);
                    for (int b = 0; b <= ny; ++b)
                        for (int a = 0; a <= nx; ++a) {
                            const double* cc = c + 7 * (b * mx + a);
                            double f = form == ORC_FORM_SPLIT
                                ? r0[(size_t)p * mm + b * mx + a] + (orc_time_factor(P, tk) - sT) * amp * cc[6]
                                : orc_time_factor(P, tk) * amp * cc[6];
                            EXT(un, a, b, mx) = EXT(up, a, b, mx) + dt * (op_at(P, &g, cc, up, a, b) + f);
                        }
                    for (int b = 0; b <= ny; ++b)
                        for (int a = 0; a <= nx; ++a) EXT(up, a, b, mx) = EXT(un, a, b, mx);
                }
                free(un);
                /* restricted change of the departure so far */
                dR[p] = form == ORC_FORM_SPLIT ? trapezoid(&g, up) : trapezoid(&g, up) - trapezoid(&g, u0 + (size_t)p * ne);
            }
        }
        for (int p = 0; p < np; ++p) {
            patch_geo g = patch_of(P, p);
            double d = dR[p];
            if (P->restrict_mode == ORC_RESTRICT_MACRO) d += lift_trapezoid_bias(&g, &e0[p]);
            U[g.j * nxp + g.i] = U[g.j * nxp + g.i] + dtm * (d / tau);
        }
        orc_apply_bc(P, U, t0 + (s + 1) * dtm);
    }
    free(coef); free(u); free(u0); free(r0); free(e0); free(dR); free(V);
}

void orc_step(const orc_problem* P, double* U, double t0, double dtm, int n_steps, double dt, int form)
{
    if (P->q_refresh > 1) {
        step_refresh(P, U, t0, dtm, n_steps, dt, form);
        return;
    }
    int np = orc_n_patch(P), mm = P->m_xi * P->m_eta;
    double* coef = all_coeffs(P);
    double* dU = (double*)malloc(sizeof(double) * np);
    double tau = P->k_micro * dt;
    for (int s = 0; s < n_steps; ++s) {
        double T = t0 + s * dtm;
        #pragma omp parallel for schedule(static)
        for (int p = 0; p < np; ++p)
            dU[p] = run_patch(P, U, p, coef + (size_t)7 * mm * p, T, P->k_micro, dt, form, NULL);
        int nx = n_xpts(P);
        for (int p = 0; p < np; ++p) {
            patch_geo g = patch_of(P, p);
            U[g.j * nx + g.i] = U[g.j * nx + g.i] + dtm * (dU[p] / tau);
        }
        orc_apply_bc(P, U, t0 + (s + 1) * dtm);
    }
    free(dU);
    free(coef);
}

/* ------------------------------------------------------------------------- */
/* Full-domain simulation (the comparison of Section 4.1.2): the transformed
   PDE on the uniform computational grid with the same micro differences,
   forward Euler in time (in place of the paper's variable-order stiff solver),
   Dirichlet data on the boundary, periodic wrap in xi where set. */

int orc_full_domain_size(const orc_problem* P, int refine, int* nxf, int* nyf)
{
    *nxf = P->n_xi * refine + (P->periodic_xi ? 0 : 1);
    *nyf = P->n_eta * refine + 1;
    return (*nxf) * (*nyf);
}

void orc_full_domain(const orc_problem* P, int refine, double* u, double t0, double dt, int n_steps)
{
    int nxf, nyf;
    orc_full_domain_size(P, refine, &nxf, &nyf);
    double hx = d_xi(P) / refine, hy = d_eta(P) / refine;
    size_t n = (size_t)nxf * nyf;
    double* c = (double*)malloc(sizeof(double) * 7 * n);
    double* un = (double*)malloc(sizeof(double) * n);
    for (int j = 0; j < nyf; ++j)
        for (int i = 0; i < nxf; ++i) orc_coeffs(P, P->xi0 + i * hx, P->eta0 + j * hy, c + 7 * ((size_t)j * nxf + i));
    for (int s = 0; s < n_steps; ++s) {
        double t = t0 + s * dt;
        double st = orc_time_factor(P, t);
        #pragma omp parallel for schedule(static)
        for (int j = 0; j < nyf; ++j)
            for (int i = 0; i < nxf; ++i) {
                size_t o = (size_t)j * nxf + i;
                int bnd = (j == 0 || j == nyf - 1) || (!P->periodic_xi && (i == 0 || i == nxf - 1));
                if (bnd) { un[o] = u[o]; continue; }
                int ie = P->periodic_xi ? (i + 1) % nxf : i + 1;
                int iw = P->periodic_xi ? (i - 1 + nxf) % nxf : i - 1;
                const double* cc = c + 7 * o;
                double uc = u[o];
                double uE = u[(size_t)j * nxf + ie], uW = u[(size_t)j * nxf + iw];
                double uN = u[(size_t)(j + 1) * nxf + i], uS = u[(size_t)(j - 1) * nxf + i];
                double uNE = u[(size_t)(j + 1) * nxf + ie], uNW = u[(size_t)(j + 1) * nxf + iw];
                double uSE = u[(size_t)(j - 1) * nxf + ie], uSW = u[(size_t)(j - 1) * nxf + iw];
                double uxx = (uE - 2.0 * uc + uW) / (hx * hx);
                double uyy = (uN - 2.0 * uc + uS) / (hy * hy);
                double uxy = (uNE - uSE - uNW + uSW) / (4.0 * hx * hy);
                double ux, uy;
                if (P->conv == ORC_CONV_CENTRAL) { ux = (uE - uW) / (2.0 * hx); uy = (uN - uS) / (2.0 * hy); }
                else {
                    ux = cc[3] > 0.0 ? (uc - uW) / hx : (uE - uc) / hx;
                    uy = cc[4] > 0.0 ? (uc - uS) / hy : (uN - uc) / hy;
                }
                double L = cc[0] * uxx + cc[1] * uxy + cc[2] * uyy - cc[3] * ux - cc[4] * uy + cc[5] * uc;
                un[o] = uc + dt * (L + st * cc[6]);
            }
        double tn = t0 + (s + 1) * dt;
        for (int j = 0; j < nyf; ++j)
            for (int i = 0; i < nxf; ++i) {
                size_t o = (size_t)j * nxf + i;
                int bnd = (j == 0 || j == nyf - 1) || (!P->periodic_xi && (i == 0 || i == nxf - 1));
                if (bnd) {
                    double m[12];
                    orc_map(P, P->xi0 + i * hx, P->eta0 + j * hy, m);
                    un[o] = orc_exact(P, m[0], m[1], tn);
                }
            }
        memcpy(u, un, sizeof(double) * n);
    }
    free(c); free(un);
}

void orc_micro_patch(const orc_problem* P, int p, const double* w0, const double* r, double T,
                     int K, double dt, double* out)
{
    patch_geo g = patch_of(P, p);
    int mx = g.mx, my = g.my, ne = (mx + 2) * (my + 2);
    double* c = (double*)malloc(sizeof(double) * 7 * mx * my);
    double* u = (double*)calloc((size_t)ne, sizeof(double));
    double* un = (double*)calloc((size_t)ne, sizeof(double));
    double* r0 = (double*)calloc((size_t)mx * my, sizeof(double));
    patch_edge e;
    memset(&e, 0, sizeof(e));
    patch_coeffs(P, &g, c);
    for (int b = 0; b < my; ++b)
        for (int a = 0; a < mx; ++a) {
            EXT(u, a, b, mx) = w0[b * mx + a];
            if (r) r0[b * mx + a] = r[b * mx + a];
        }
    double amp = (P->src == ORC_SRC_GAUSS_PATCH && P->src_amp) ? P->src_amp[p] : 1.0;
    micro_split(P, &g, &e, c, amp, r0, T, K, dt, u, un);
    for (int b = 0; b < my; ++b)
        for (int a = 0; a < mx; ++a) out[b * mx + a] = EXT(u, a, b, mx);
    free(c); free(u); free(un); free(r0);
}

/* dU for a selection of patches only (sampled checks at full size) */
void orc_patch_dU(const orc_problem* P, const double* U, double t, double dt, int form,
                  int n_sel, const int* sel, double* dU)
{
    int mm = P->m_xi * P->m_eta;
    #pragma omp parallel for schedule(static)
    for (int s = 0; s < n_sel; ++s) {
        patch_geo g = patch_of(P, sel[s]);
        double* c = (double*)malloc(sizeof(double) * 7 * mm);
        patch_coeffs(P, &g, c);
        dU[s] = run_patch(P, U, sel[s], c, t, P->k_micro, dt, form, NULL);
        free(c);
    }
}

/* ------------------------------------------------------------------------- */
/* Eq. (Annulus_AS) written as an eigenfunction expansion: coefficient of mode m
   = int r u0(r) Z_1(mu_m r) dr / int r Z_1(mu_m r)^2 dr, decay exp(-mu_m^2 t). */

double orc_bessel_norm(double mu, double ra, double rb, int n_int)
{
    if (n_int % 2) n_int++;
    double h = (rb - ra) / n_int, s = 0.0;
    for (int q = 0; q <= n_int; ++q) {
        double r = ra + q * h;
        double z = orc_bessel_Z(1, mu, ra, r);
        double w = (q == 0 || q == n_int) ? 1.0 : (q % 2 ? 4.0 : 2.0);
        s += w * r * z * z;
    }
    return s * h / 3.0;
}

double orc_annulus_series(double ra, double rb, double r, double theta, double t, int n_roots)
{
    const int n_int = 4000;
    double sum = 0.0;
    for (int m = 1; m <= n_roots; ++m) {
        double mu = orc_bessel_root(1, ra, rb, m);
        double h = (rb - ra) / n_int, num = 0.0;
        for (int q = 0; q <= n_int; ++q) {
            double x = ra + q * h;
            double w = (q == 0 || q == n_int) ? 1.0 : (q % 2 ? 4.0 : 2.0);
            num += w * x * (x - ra) * (rb - x) * orc_bessel_Z(1, mu, ra, x);
        }
        num *= h / 3.0;
        sum += num / orc_bessel_norm(mu, ra, rb, n_int) * orc_bessel_Z(1, mu, ra, r) * exp(-mu * mu * t);
    }
    return sum * sin(theta);
}

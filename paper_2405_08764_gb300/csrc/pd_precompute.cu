// S0: transformed-coefficient precompute (Section 2, eq. Computational_Problem),
// step bounds, initial fields and per-step time tables.  All arithmetic here is
// FP64: it runs once per problem (or once per pd_step call for the time table).
#include "pd_internal.h"

#include <math.h>

namespace pd {

namespace {

struct CoefDev {
    double M11, M12, M22, d0, dx, dy, ds, dk;
    int n_four; double four_c[3], four_phi[3], four_ra, four_rb;
    double va[3], vb[3], f0;
    int src; double src_p[3];
    int sol;
};

CoefDev to_dev(const pd_coeff_desc& c)
{
    CoefDev d;
    d.M11 = c.M11; d.M12 = c.M12; d.M22 = c.M22;
    d.d0 = c.d0; d.dx = c.dx; d.dy = c.dy; d.ds = c.ds; d.dk = c.dk;
    d.n_four = c.n_four;
    for (int k = 0; k < 3; ++k) {
        d.four_c[k] = c.four_c[k]; d.four_phi[k] = c.four_phi[k];
        d.va[k] = c.va[k]; d.vb[k] = c.vb[k]; d.src_p[k] = c.src_p[k];
    }
    d.four_ra = c.four_ra; d.four_rb = c.four_rb;
    d.f0 = c.f0; d.src = c.src; d.sol = c.sol;
    return d;
}

// x(xi, eta), y(xi, eta) with first and second derivatives.
struct Jet {
    double x, y;
    double x_a, x_b, y_a, y_b;            // a = xi, b = eta
    double x_aa, x_ab, x_bb, y_aa, y_ab, y_bb;
};

// one-dimensional stretchings: value, first and second derivative
__device__ void tanh_stretch(double s, double q0, double q1, double q, double& X, double& X1, double& X2)
{
    double L = q1 - q0;
    if (s == 0.0) { X = q; X1 = 1.0; X2 = 0.0; return; }
    double z = (q - q0) / L;
    double T = tanh(s);
    double th = tanh(s * z);
    double sech2 = 1.0 - th * th;
    X = q0 + L * th / T;
    X1 = s * sech2 / T;
    X2 = -2.0 * s * s * sech2 * th / (T * L);
}

__device__ Jet eval_map(const InstDev& I, double xi, double eta)
{
    Jet m = {};
    switch (I.map) {
    case PD_MAP_SINE: {
        // eq. (Stretching_Transformation)
        double lam = I.map_p[0];
        double sx, cx, sy, cy;
        sincospi(xi, &sx, &cx);
        sincospi(eta, &sy, &cy);
        m.x = xi + lam / M_PI * sx;      m.y = eta + lam / M_PI * sy;
        m.x_a = 1.0 + lam * cx;          m.y_b = 1.0 + lam * cy;
        m.x_aa = -lam * M_PI * sx;       m.y_bb = -lam * M_PI * sy;
        break;
    }
    case PD_MAP_TANH:
        tanh_stretch(I.map_p[0], I.xi0, I.xi1, xi, m.x, m.x_a, m.x_aa);
        tanh_stretch(I.map_p[1], I.eta0, I.eta1, eta, m.y, m.y_b, m.y_bb);
        break;
    case PD_MAP_POLAR: {
        // eq. (Transformation_Annulus) with a radial profile r(eta)
        double ra = I.map_p[0], rb = I.map_p[1], sr = I.map_p[2];
        double L = I.eta1 - I.eta0;
        double z = (eta - I.eta0) / L;
        double rho = z, rho1 = 1.0, rho2 = 0.0;
        if (sr != 0.0) {
            double T = tanh(sr), th = tanh(sr * (2.0 * z - 1.0)), sech2 = 1.0 - th * th;
            rho = 0.5 * (1.0 + th / T);
            rho1 = sr * sech2 / T;
            rho2 = -4.0 * sr * sr * sech2 * th / T;
        }
        double R = ra + (rb - ra) * rho, R1 = (rb - ra) * rho1 / L, R2 = (rb - ra) * rho2 / (L * L);
        double sn, cs;
        sincos(xi, &sn, &cs);
        m.x = R * cs;          m.y = R * sn;
        m.x_a = -R * sn;       m.x_b = R1 * cs;
        m.y_a = R * cs;        m.y_b = R1 * sn;
        m.x_aa = -R * cs;      m.x_ab = -R1 * sn;     m.x_bb = R2 * cs;
        m.y_aa = -R * sn;      m.y_ab = R1 * cs;      m.y_bb = R2 * sn;
        break;
    }
    default:
        m.x = xi; m.y = eta; m.x_a = 1.0; m.y_b = 1.0;
    }
    return m;
}

// symmetric 2x2 as (s11, s12, s22)
struct Sym { double a, b, c; };

struct PhysPoint {
    Sym K, Kx, Ky;
    double v1, v2, divv, f;
};

__device__ PhysPoint eval_phys(const CoefDev& C, double x, double y)
{
    double d = C.d0 + C.dx * x + C.dy * y, gx = C.dx, gy = C.dy;
    if (C.ds != 0.0) {
        double w = 2.0 * C.dk;
        double sx, cx, sy, cy;
        sincospi(w * x, &sx, &cx);
        sincospi(w * y, &sy, &cy);
        d += C.ds * sx * sy;
        gx += C.ds * w * M_PI * cx * sy;
        gy += C.ds * w * M_PI * sx * cy;
    }
    if (C.n_four > 0) {
        double r = hypot(x, y), th = atan2(y, x);
        double ir = 1.0 / r, ct = x * ir, st = y * ir;
        double span = C.four_rb - C.four_ra;
        double rho = (r - C.four_ra) / span;
        for (int k = 1; k <= C.n_four; ++k) {
            double ang = k * th + C.four_phi[k - 1];
            double sa, ca, sb, cb;
            sincos(ang, &sa, &ca);
            sincospi(k * rho, &sb, &cb);
            double ck = C.four_c[k - 1];
            double dr = -ck * ca * k * M_PI * sb / span;   // d/dr
            double dth = -ck * k * sa * cb;                // d/dtheta
            d += ck * ca * cb;
            gx += ct * dr - st * ir * dth;
            gy += st * dr + ct * ir * dth;
        }
    }
    PhysPoint P;
    P.K = { d * C.M11, d * C.M12, d * C.M22 };
    P.Kx = { gx * C.M11, gx * C.M12, gx * C.M22 };
    P.Ky = { gy * C.M11, gy * C.M12, gy * C.M22 };
    P.v1 = C.va[0] + C.va[1] * x + C.va[2] * y;
    P.v2 = C.vb[0] + C.vb[1] * x + C.vb[2] * y;
    P.divv = C.va[1] + C.vb[2];
    P.f = C.f0;
    return P;
}

__device__ double source_factor(const CoefDev& C, const PhysPoint& P, double x, double y)
{
    switch (C.src) {
    case PD_SRC_MMS_SINPROD: {
        // u = e^{-t} S, S = sin(pi x) sin(pi y):  g = u_t - div(K grad u) + v.grad u + (div v - f) u
        double sx, cx, sy, cy;
        sincospi(x, &sx, &cx);
        sincospi(y, &sy, &cy);
        double S = sx * sy;
        double divKgrad = -M_PI * M_PI * (P.K.a + P.K.c) * S + 2.0 * M_PI * M_PI * P.K.b * cx * cy;
        double adv = M_PI * (P.v1 * cx * sy + P.v2 * sx * cy);
        return (P.divv - P.f - 1.0) * S - divKgrad + adv;
    }
    case PD_SRC_EXP_LINEAR:
        return (C.src_p[0] + C.src_p[1] * x + C.src_p[2] * y) * exp(x + y);
    case PD_SRC_GAUSS_PATCH:
        return exp(-(x * x + y * y));
    default:
        return 0.0;
    }
}

__device__ __forceinline__ double quad(const Sym& K, double p0, double p1, double q0, double q1)
{
    return p0 * (K.a * q0 + K.b * q1) + p1 * (K.b * q0 + K.c * q1);
}

// Coefficients of eq. (Computational_Problem) for a tensor K on a general map.
// With the contravariant basis grad xi = a / J, grad eta = b / J,
// a = (y_eta, -x_eta), b = (-y_xi, x_xi), write S^{ab} = J K^{ab} = p.K q / J.
// The conservative form div(K grad u) = (1/J)[d_xi(S^{xx} u_xi + S^{xe} u_eta)
// + d_eta(S^{xe} u_xi + S^{ee} u_eta)] gives alpha = K^{xx}, beta = 2K^{xe},
// gamma = K^{ee} and first-derivative coefficients (1/J)(d_xi S^{xx} + d_eta S^{xe}),
// (1/J)(d_xi S^{xe} + d_eta S^{ee}); convection adds grad xi . v, grad eta . v.
__device__ void transformed(const Jet& m, const PhysPoint& P, double out[6])
{
    double J = m.x_a * m.y_b - m.x_b * m.y_a;
    double iJ = 1.0 / J;
    double J_a = m.x_aa * m.y_b + m.x_a * m.y_ab - m.x_ab * m.y_a - m.x_b * m.y_aa;
    double J_b = m.x_ab * m.y_b + m.x_a * m.y_bb - m.x_bb * m.y_a - m.x_b * m.y_ab;
    // covariant pieces and their derivatives
    double a0 = m.y_b, a1 = -m.x_b, b0 = -m.y_a, b1 = m.x_a;
    double a0_a = m.y_ab, a1_a = -m.x_ab, a0_b = m.y_bb, a1_b = -m.x_bb;
    double b0_a = -m.y_aa, b1_a = m.x_aa, b0_b = -m.y_ab, b1_b = m.x_ab;
    // K along the coordinate lines
    Sym K_a = { P.Kx.a * m.x_a + P.Ky.a * m.y_a, P.Kx.b * m.x_a + P.Ky.b * m.y_a, P.Kx.c * m.x_a + P.Ky.c * m.y_a };
    Sym K_b = { P.Kx.a * m.x_b + P.Ky.a * m.y_b, P.Kx.b * m.x_b + P.Ky.b * m.y_b, P.Kx.c * m.x_b + P.Ky.c * m.y_b };
    double Qaa = quad(P.K, a0, a1, a0, a1), Qab = quad(P.K, a0, a1, b0, b1), Qbb = quad(P.K, b0, b1, b0, b1);
    // derivatives of the quadratic forms (product rule)
    double Qaa_a = 2.0 * quad(P.K, a0_a, a1_a, a0, a1) + quad(K_a, a0, a1, a0, a1);
    double Qab_b = quad(P.K, a0_b, a1_b, b0, b1) + quad(P.K, a0, a1, b0_b, b1_b) + quad(K_b, a0, a1, b0, b1);
    double Qab_a = quad(P.K, a0_a, a1_a, b0, b1) + quad(P.K, a0, a1, b0_a, b1_a) + quad(K_a, a0, a1, b0, b1);
    double Qbb_b = 2.0 * quad(P.K, b0_b, b1_b, b0, b1) + quad(K_b, b0, b1, b0, b1);
    // d(Q / J) = dQ / J - Q dJ / J^2
    double Sxx_a = (Qaa_a - Qaa * J_a * iJ) * iJ;
    double Sxe_b = (Qab_b - Qab * J_b * iJ) * iJ;
    double Sxe_a = (Qab_a - Qab * J_a * iJ) * iJ;
    double See_b = (Qbb_b - Qbb * J_b * iJ) * iJ;
    double iJ2 = iJ * iJ;
    out[0] = Qaa * iJ2;
    out[1] = 2.0 * Qab * iJ2;
    out[2] = Qbb * iJ2;
    double Vx = (a0 * P.v1 + a1 * P.v2) * iJ, Ve = (b0 * P.v1 + b1 * P.v2) * iJ;
    out[3] = Vx - (Sxx_a + Sxe_b) * iJ;
    out[4] = Ve - (Sxe_a + See_b) * iJ;
    out[5] = P.f - P.divv;
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* p, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename real>
__global__ void precompute_kernel(const InstDev I, const CoefDev C, const double* __restrict__ amp,
                                  real* __restrict__ rec, unsigned long long* rate_max)
{
    long long n = (long long)I.n_patch * I.mx * I.my;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double rate = 0.0;
    if (idx < n) {
        // strip-image order: a fastest, then patch column, then micro row, then patch row
        int a = (int)(idx % I.mx);
        long long r1 = idx / I.mx;
        int ic = (int)(r1 % I.ncols);
        long long r2 = r1 / I.ncols;
        int b = (int)(r2 % I.my);
        int jr = (int)(r2 / I.my);
        int i = I.i0 + ic, j = 1 + jr;
        double xi = (I.xi0 + i * I.Dx) - 0.5 * I.hx + a * I.dx;
        double eta = (I.eta0 + j * I.Dy) - 0.5 * I.hy + b * I.dy;
        Jet m = eval_map(I, xi, eta);
        PhysPoint P = eval_phys(C, m.x, m.y);
        double c[6];
        transformed(m, P, c);
        double G = source_factor(C, P, m.x, m.y);
        if (C.src == PD_SRC_GAUSS_PATCH) G *= amp[jr * I.ncols + ic];
        double J = m.x_a * m.y_b - m.x_b * m.y_a;
        bool bad = !(J != 0.0);
        for (int k = 0; k < 6; ++k) bad |= !isfinite(c[k]);
        bad |= !isfinite(G);
        if (bad) atomicOr(I.err, ERR_JACOBIAN);
        if (rec) {
            real* o = rec + idx * 8;
            for (int k = 0; k < 6; ++k) o[k] = (real)c[k];
            o[6] = (real)G;
            o[7] = (real)0;
        }
        rate = 2.0 * fabs(c[0]) / (I.dx * I.dx) + 2.0 * fabs(c[2]) / (I.dy * I.dy)
             + fabs(c[1]) / (I.dx * I.dy) + fabs(c[5]);
        if (I.conv == PD_CONV_UPWIND) rate += fabs(c[3]) / I.dx + fabs(c[4]) / I.dy;
        if (!isfinite(rate)) rate = 0.0;
    }
    rate = warp_max(rate);
    if ((threadIdx.x & 31) == 0) atomic_max_pos(rate_max, rate);
}

// macro step bound at the patch centres (reading G9)
__global__ void macro_rate_kernel(const InstDev I, const CoefDev C, unsigned long long* rate_max)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    double rate = 0.0;
    if (p < I.n_patch) {
        int i = I.i0 + p % I.ncols, j = 1 + p / I.ncols;
        Jet m = eval_map(I, I.xi0 + i * I.Dx, I.eta0 + j * I.Dy);
        PhysPoint P = eval_phys(C, m.x, m.y);
        double c[6];
        transformed(m, P, c);
        rate = 2.0 * fabs(c[0]) / (I.Dx * I.Dx) + 2.0 * fabs(c[2]) / (I.Dy * I.Dy)
             + fabs(c[1]) / (I.Dx * I.Dy) + fabs(c[3]) / I.Dx + fabs(c[4]) / I.Dy + fabs(c[5]);
        if (!isfinite(rate)) rate = 0.0;
    }
    rate = warp_max(rate);
    if ((threadIdx.x & 31) == 0) atomic_max_pos(rate_max, rate);
}

__global__ void boundary_xy_kernel(const InstDev I, double2* xy)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= I.n_bnd) return;
    int2 ij = I.bnd_ij[k];
    Jet m = eval_map(I, I.xi0 + ij.x * I.Dx, I.eta0 + ij.y * I.Dy);
    xy[k] = make_double2(m.x, m.y);
}

template <typename real>
__global__ void get_coeffs_kernel(const InstDev I, const real* __restrict__ rec, double* __restrict__ out)
{
    long long n = (long long)I.n_patch * I.mx * I.my;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    int a = (int)(idx % I.mx);
    long long r1 = idx / I.mx;
    int ic = (int)(r1 % I.ncols);
    long long r2 = r1 / I.ncols;
    int b = (int)(r2 % I.my);
    int jr = (int)(r2 / I.my);
    long long p = (long long)jr * I.ncols + ic;
    double* o = out + ((p * I.my + b) * I.mx + a) * 8;
    for (int k = 0; k < 8; ++k) o[k] = (double)rec[idx * 8 + k];
}

struct InitParams {
    int kind, n_modes;
    double p[16];
    double mu[8];
};

__global__ void init_field_kernel(const InstDev I, const CoefDev C, const InitParams ip, double t, double* U)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= I.nxp * I.nyp) return;
    int i = k % I.nxp, j = k / I.nxp;
    double xi = I.xi0 + i * I.Dx, eta = I.eta0 + j * I.Dy;
    Jet m = eval_map(I, xi, eta);
    double v = 0.0;
    switch (ip.kind) {
    case PD_INIT_EXACT:
        v = exact_solution(C.sol, m.x, m.y, t);
        break;
    case PD_INIT_BESSEL: {
        double r = hypot(m.x, m.y), th = atan2(m.y, m.x), ra = ip.p[1];
        for (int q = 1; q <= ip.n_modes; ++q) {
            double mu = ip.mu[q - 1];
            double Z = jn(q, mu * ra) * yn(q, mu * r) - yn(q, mu * ra) * jn(q, mu * r);
            v += ip.p[2 + q] * Z * cos(q * th) * exp(-C.d0 * mu * mu * t);
        }
        break;
    }
    case PD_INIT_BUMP: {
        double zx = (xi - I.xi0) / (I.xi1 - I.xi0), zy = (eta - I.eta0) / (I.eta1 - I.eta0);
        double fx = I.periodic ? 1.0 + 0.5 * cos(xi) : sinpi(zx);
        v = fx * sinpi(zy);
        break;
    }
    case PD_INIT_ANNULUS_POLY: {
        double r = hypot(m.x, m.y), th = atan2(m.y, m.x);
        v = (r - ip.p[0]) * (ip.p[1] - r) * sin(th);
        break;
    }
    default:
        v = 0.0;
    }
    U[k] = v;
}

// 1-D metric tables of the table coefficient mode (FP64, plus FP32 copies)
__global__ void table_build_kernel(const InstDev I, double* col_tab, double* row_tab, float* col_f, float* row_f)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int ncol = I.ncols * I.mx, nrow = I.nrows * I.my;
    if (t < ncol) {
        int ic = t / I.mx, a = t % I.mx;
        double xi = (I.xi0 + (I.i0 + ic) * I.Dx) - 0.5 * I.hx + a * I.dx;
        double* o = col_tab + (size_t)t * 2;
        if (I.coef_mode == COEF_POLAR) {
            double s, c;
            sincos(xi, &s, &c);
            o[0] = s; o[1] = c;
        } else {
            Jet m = eval_map(I, xi, I.eta0);
            double ia = 1.0 / m.x_a;
            o[0] = ia; o[1] = m.x_aa * ia * ia * ia;
        }
        if (col_f) { col_f[(size_t)t * 2] = (float)o[0]; col_f[(size_t)t * 2 + 1] = (float)o[1]; }
    } else if (t < ncol + nrow) {
        int u = t - ncol;
        int jr = u / I.my, b = u % I.my;
        double eta = (I.eta0 + (1 + jr) * I.Dy) - 0.5 * I.hy + b * I.dy;
        double* o = row_tab + (size_t)u * 4;
        if (I.coef_mode == COEF_POLAR) {
            Jet m = eval_map(I, 0.0, eta);   // at xi = 0: x = R, x_eta = R', x_etaeta = R''
            double R = m.x, R1 = m.x_b, R2 = m.x_bb;
            o[0] = 1.0 / R; o[1] = 1.0 / R1; o[2] = R * R2 / (R1 * R1); o[3] = 0.0;
        } else {
            Jet m = eval_map(I, I.xi0, eta);
            double ib = 1.0 / m.y_b;
            o[0] = ib; o[1] = m.y_bb * ib * ib * ib; o[2] = 0.0; o[3] = 0.0;
        }
        if (row_f)
            for (int k = 0; k < 4; ++k) row_f[(size_t)u * 4 + k] = (float)o[k];
    }
}

// coefficients of a table-mode instance at every micro point, [p][b][a][8]
__global__ void table_get_coeffs_kernel(const InstDev I, double* __restrict__ out)
{
    long long n = (long long)I.n_patch * I.mx * I.my;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    int a = (int)(idx % I.mx);
    long long r1 = idx / I.mx;
    int ic = (int)(r1 % I.ncols);
    long long r2 = r1 / I.ncols;
    int b = (int)(r2 % I.my);
    int jr = (int)(r2 / I.my);
    double c[6];
    table_coeffs<double>(I, ic, a, jr, b, c);
    long long p = (long long)jr * I.ncols + ic;
    double* o = out + ((p * I.my + b) * I.mx + a) * 8;
    for (int k = 0; k < 6; ++k) o[k] = c[k];
    o[6] = 0.0; o[7] = 0.0;
}

// row s: ds_k = s(T + k dt) - s(T) (k < K), s(T), T, T_next with T = t0 + s dtm
// koff = 0: s(t_k) - s(T) at the start of forward-Euler step k; koff = 1/2:
// at the middle of ADI step k
__global__ void time_table_kernel(int K, int tkind, double tc, double dt, double koff, double t0, double dtm,
                                  int n_steps, double* tab)
{
    int stride = K + kTabExtra;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n_steps * stride) return;
    int s = (int)(idx / stride), k = (int)(idx % stride);
    double T = t0 + s * dtm;
    double v;
    if (k < K) v = time_factor(tkind, tc, T + (k + koff) * dt) - time_factor(tkind, tc, T);
    else if (k == K) v = time_factor(tkind, tc, T);
    else if (k == K + 1) v = T;
    else v = t0 + (s + 1) * dtm;
    tab[idx] = v;
}

__global__ void batch_time_table_kernel(const InstDev* __restrict__ insts, int n_inst, const double* __restrict__ dtm,
                                        double t0, int n_macro, const long long* __restrict__ tab_off, double* tab,
                                        long long total)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    // find the instance of this entry (tab_off is increasing; n_inst + 1 entries)
    int lo = 0, hi = n_inst;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (tab_off[mid] <= idx) lo = mid; else hi = mid;
    }
    const InstDev& I = insts[lo];
    int stride = I.K + kTabExtra;
    long long loc = idx - tab_off[lo];
    int s = (int)(loc / stride), k = (int)(loc % stride);
    double d = dtm[lo];
    double T = t0 + s * d;
    double v;
    if (k < I.K) v = time_factor(I.tkind, I.tc, T + k * I.dt) - time_factor(I.tkind, I.tc, T);
    else if (k == I.K) v = time_factor(I.tkind, I.tc, T);
    else if (k == I.K + 1) v = T;
    else v = t0 + (s + 1) * d;
    tab[idx] = v;
    (void)n_macro;
}

// Surrogate features of patch p that do not change with U: the four metric
// terms over the macro explicit rate R at the centre, half the trace of the
// diffusion tensor at the centre and its relative change at the edge
// midpoints E, W, N, S, and tau R.
__global__ void surrogate_static_kernel(const InstDev I, const CoefDev C, double tau, float* __restrict__ feat,
                                        double* __restrict__ Rout)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= I.n_patch) return;
    const int i = I.i0 + p % I.ncols, j = 1 + p / I.ncols;
    const double xi = I.xi0 + i * I.Dx, eta = I.eta0 + j * I.Dy;
    Jet m = eval_map(I, xi, eta);
    PhysPoint P = eval_phys(C, m.x, m.y);
    double c[6];
    transformed(m, P, c);
    const double R = 2.0 * c[0] / (I.Dx * I.Dx) + 2.0 * c[2] / (I.Dy * I.Dy) + fabs(c[1]) / (I.Dx * I.Dy)
                   + fabs(c[3]) / I.Dx + fabs(c[4]) / I.Dy + fabs(c[5]);
    auto dhalf = [&](double a, double b) {
        Jet q = eval_map(I, a, b);
        PhysPoint Q = eval_phys(C, q.x, q.y);
        return 0.5 * (Q.K.a + Q.K.c);
    };
    const double dc = 0.5 * (P.K.a + P.K.c);
    const double de[4] = { dhalf(xi + 0.5 * I.hx, eta), dhalf(xi - 0.5 * I.hx, eta),
                           dhalf(xi, eta + 0.5 * I.hy), dhalf(xi, eta - 0.5 * I.hy) };
    float* o = feat + (long long)p * 10;
    o[0] = (float)(2.0 * c[0] / (I.Dx * I.Dx * R));
    o[1] = (float)(2.0 * c[2] / (I.Dy * I.Dy * R));
    o[2] = (float)(c[3] / (I.Dx * R));
    o[3] = (float)(c[4] / (I.Dy * R));
    o[4] = (float)dc;
    for (int k = 0; k < 4; ++k) o[5 + k] = (float)((de[k] - dc) / dc);
    o[9] = (float)(tau * R);
    Rout[p] = R;
}

}  // namespace

cudaError_t launch_surrogate_static(const InstDev& I, const pd_coeff_desc& c, double tau, float* feat, double* R,
                                    cudaStream_t st)
{
    surrogate_static_kernel<<<(I.n_patch + 127) / 128, 128, 0, st>>>(I, to_dev(c), tau, feat, R);
    return cudaGetLastError();
}

cudaError_t launch_batch_time_tables(const InstDev* insts, int n_inst, const double* dtm, double t0, int n_macro,
                                     const long long* tab_off, double* tab, long long total, cudaStream_t st)
{
    if (total <= 0) return cudaSuccess;
    batch_time_table_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(insts, n_inst, dtm, t0, n_macro, tab_off, tab, total);
    return cudaGetLastError();
}

cudaError_t launch_precompute(const InstDev& I, const pd_coeff_desc& c, const double* amp_dev, void* rec,
                              int prec, unsigned long long* rate_max, unsigned long long* macro_rate_max,
                              cudaStream_t st)
{
    CoefDev C = to_dev(c);
    long long n = (long long)I.n_patch * I.mx * I.my;
    int bs = 256;
    unsigned nb = (unsigned)((n + bs - 1) / bs);
    if (prec == PD_FP32)
        precompute_kernel<float><<<nb, bs, 0, st>>>(I, C, amp_dev, (float*)rec, rate_max);
    else
        precompute_kernel<double><<<nb, bs, 0, st>>>(I, C, amp_dev, (double*)rec, rate_max);
    macro_rate_kernel<<<(I.n_patch + 127) / 128, 128, 0, st>>>(I, C, macro_rate_max);
    if (I.n_bnd > 0)
        boundary_xy_kernel<<<(I.n_bnd + 127) / 128, 128, 0, st>>>(I, const_cast<double2*>(I.bnd_xy));
    return cudaGetLastError();
}

cudaError_t launch_tables(const InstDev& I, double* col_tab, double* row_tab, float* col_tab_f, float* row_tab_f,
                          unsigned long long* rate_max, unsigned long long* macro_rate_max, cudaStream_t st)
{
    (void)rate_max; (void)macro_rate_max;
    int n = I.ncols * I.mx + I.nrows * I.my;
    table_build_kernel<<<(n + 127) / 128, 128, 0, st>>>(I, col_tab, row_tab, col_tab_f, row_tab_f);
    return cudaGetLastError();
}

cudaError_t launch_table_get_coeffs(const InstDev& I, double* out, cudaStream_t st)
{
    long long n = (long long)I.n_patch * I.mx * I.my;
    table_get_coeffs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(I, out);
    return cudaGetLastError();
}

cudaError_t launch_get_coeffs(const InstDev& I, int prec, double* out, cudaStream_t st)
{
    long long n = (long long)I.n_patch * I.mx * I.my;
    unsigned nb = (unsigned)((n + 255) / 256);
    if (prec == PD_FP32)
        get_coeffs_kernel<float><<<nb, 256, 0, st>>>(I, (const float*)I.rec, out);
    else
        get_coeffs_kernel<double><<<nb, 256, 0, st>>>(I, (const double*)I.rec, out);
    return cudaGetLastError();
}

cudaError_t launch_init_field(const InstDev& I, const pd_coeff_desc& c, int kind, const double* prm,
                              int n_prm, const double* mu, double t, double* U, cudaStream_t st)
{
    InitParams ip = {};
    ip.kind = kind;
    for (int k = 0; k < n_prm && k < 16; ++k) ip.p[k] = prm[k];
    if (kind == PD_INIT_BESSEL) {
        ip.n_modes = (int)prm[0];
        for (int k = 0; k < ip.n_modes && k < 8; ++k) ip.mu[k] = mu[k];
    }
    int n = I.nxp * I.nyp;
    init_field_kernel<<<(n + 127) / 128, 128, 0, st>>>(I, to_dev(c), ip, t, U);
    return cudaGetLastError();
}

cudaError_t launch_time_table(const InstDev& I, double t0, double dtm, int n_steps, double* tab, cudaStream_t st)
{
    long long n = (long long)n_steps * (I.K + kTabExtra);
    time_table_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(I.K, I.tkind, I.tc, I.dt,
                                                                 I.micro == PD_MICRO_ADI ? 0.5 : 0.0, t0, dtm, n_steps, tab);
    return cudaGetLastError();
}

}  // namespace pd

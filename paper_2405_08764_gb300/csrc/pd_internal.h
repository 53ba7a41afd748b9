// Internal definitions of the GB300 patch-dynamics library.
//
// Device-side layout
//   * coefficient records: one 8-value record per micro point (alpha, beta,
//     gamma, nu, omega, phi, G * patch amplitude, 0), stored in "strip image"
//     order: for patch row jr and micro row b, the micro columns of all
//     patches of that row are contiguous:
//        rec[((jr * my + b) * ncols + ic) * mx + a]
//     so a warp whose lanes hold consecutive micro columns of consecutive
//     patches reads one contiguous run per micro row.
//   * macro field U: FP64, U[j * nxp + i] per instance.
//   * micro state (separate C-ABI passes): see include/pd.h.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "pd.h"

namespace pd {

constexpr int kMaxK = 4096;      // micro steps per burst
constexpr int kMaxM = 32;        // micro points per side (one warp spans a patch row)
constexpr int kTabExtra = 3;     // time table row: ds_0..ds_{K-1}, s(T), T, T_next

// Per-instance constants used by the kernels (FP64; kernels convert).
struct InstDev {
    int n_xi, n_eta, periodic, nxp, nyp, ncols, nrows, i0;
    int mx, my, K, conv, restrict_mode, tkind, sol, map;
    int n_patch, n_bnd;
    int has_cross, has_tsrc;
    double xi0, eta0, Dx, Dy, hx, hy, dx, dy;
    double dt, tau, tc;
    double map_p[4];
    double xi1, eta1;
    double lw[9][9];             // monomial coefficients of the 3x3 interpolant, see poly_weights
    // two-phase form of the same coefficients (micro sizes >= 9): coefficient k =
    // scale_k * (P + w1_k Q + w2_k R) over first/second macro differences, see macro_coeffs
    int c2slot[9][3];
    double c2w[9][3];
    long long u_off;             // offset of this instance in U (doubles)
    long long p_off;             // offset in patches (dU, bias)
    long long pt_off;            // offset in micro points (u0, r, w of the micro state)
    long long e_off;             // offset in edge entries (4 * edge_stride per patch)
    int edge_stride;             // max(mx, my) + 2
    const void* rec;             // coefficient records (float or double, 8 per point)
    const void* brec;            // burst records (16 per point, see burst_record_kernel)
    double inv_nn;               // 1 / ((m_xi - 1)(m_eta - 1))
    double inv_tau;              // 1 / tau
    const int2* bnd_ij;          // boundary nodes (i, j)
    const double2* bnd_xy;       // their physical coordinates
    int* err;                    // device error flags
    // coefficient storage: records (per micro point) or 1-D metric tables for
    // constant K, v, f on separable or polar maps (see table_coeffs)
    int coef_mode;
    const double* col_tab;       // [ncols][mx][2]
    const double* row_tab;       // [nrows][my][4]
    const float* col_tab_f;      // FP32 copies for the FP32 batched path
    const float* row_tab_f;
    double K11, K12, K22, v1, v2, f0;
    // reciprocals of the nano steps (division-free stencil weights)
    double inv_dx, inv_dy, inv_dx2, inv_dy2, inv_4dxdy;
    int ppw;                     // patches per warp in the batched kernel (<= 32 / mx)
    int micro;                   // pd_micro_solver
    // FP32 copies of the instance constants, converted once on the host (a
    // double -> float conversion issues on the slow FP64 pipe): K11, K12, K22,
    // v1, v2, f0, 1/dx, 1/dy, 1/dx^2, 1/dy^2, 1/(4 dx dy), dx, dy, hx, hy, dt
    float kf[16];
    float c2sf[9];               // FP32 copies of the interpolant scales c2w[k][2]
    const void* arec_c;          // ADI line records, eta lines (8 per point, see pd_adi.cu)
    const void* arec_r;          // ADI line records, xi lines (8 per point, patch-transposed)
};

enum CoefMode { COEF_RECORDS = 0, COEF_SEPARABLE = 1, COEF_POLAR = 2 };

// fill InstDev::kf from the FP64 constants (host side, after every change of them)
inline void fill_float_consts(InstDev& I)
{
    const double v[16] = { I.K11, I.K12, I.K22, I.v1, I.v2, I.f0, I.inv_dx, I.inv_dy, I.inv_dx2, I.inv_dy2,
                           I.inv_4dxdy, I.dx, I.dy, I.hx, I.hy, I.dt };
    for (int k = 0; k < 16; ++k) I.kf[k] = (float)v[k];
    for (int k = 0; k < 9; ++k) I.c2sf[k] = (float)I.c2w[k][2];
}

// Transformed coefficients (alpha, beta, gamma, nu, omega, phi) for constant K, v,
// f from 1-D metric tables (eq. Computational_Problem with the operator of the
// derived form used by precompute_kernel, specialised by hand):
//  separable maps x = X(xi), y = Y(eta): col = (1/X', X''/X'^3), row = (1/Y', Y''/Y'^3):
//    alpha = K11/X'^2, beta = 2 K12/(X'Y'), gamma = K22/Y'^2,
//    nu = v1/X' + K11 X''/X'^3, omega = v2/Y' + K22 Y''/Y'^3, phi = f;
//  polar map x = R cos xi, y = R sin xi: col = (sin xi, cos xi), row = (1/R, 1/R', R R''/R'^2):
//    A = s^2 K11 - 2sc K12 + c^2 K22, B = sc (K22 - K11) + (c^2 - s^2) K12,
//    C = c^2 K11 + 2sc K12 + s^2 K22, B' = (c^2 - s^2)(K22 - K11) - 4sc K12,
//    alpha = A/R^2, beta = 2B/(R R'), gamma = C/R'^2,
//    nu = (-s v1 + c v2)/R + 2B/R^2, omega = (c v1 + s v2)/R' - (B' + C (1 - R R''/R'^2))/(R R'),
//    phi = f.
template <typename real>
__device__ __forceinline__ void table_coeffs(const InstDev& I, int ic, int a, int jr, int b, real c[6])
{
    const double* ct = I.col_tab + ((size_t)ic * I.mx + a) * 2;
    const double* rt = I.row_tab + ((size_t)jr * I.my + b) * 4;
    const real K11 = (real)I.K11, K12 = (real)I.K12, K22 = (real)I.K22;
    const real v1 = (real)I.v1, v2 = (real)I.v2;
    if (I.coef_mode == COEF_SEPARABLE) {
        real ia = (real)ct[0], ia2 = (real)ct[1], ib = (real)rt[0], ib2 = (real)rt[1];
        c[0] = K11 * ia * ia;
        c[1] = real(2) * K12 * ia * ib;
        c[2] = K22 * ib * ib;
        c[3] = v1 * ia + K11 * ia2;
        c[4] = v2 * ib + K22 * ib2;
    } else {
        real s = (real)ct[0], co = (real)ct[1];
        real iR = (real)rt[0], iRp = (real)rt[1], q = (real)rt[2];
        real ss = s * s, cc = co * co, sc = s * co;
        real A = ss * K11 - real(2) * sc * K12 + cc * K22;
        real B = sc * (K22 - K11) + (cc - ss) * K12;
        real C = cc * K11 + real(2) * sc * K12 + ss * K22;
        real Bp = (cc - ss) * (K22 - K11) - real(4) * sc * K12;
        c[0] = A * iR * iR;
        c[1] = real(2) * B * iR * iRp;
        c[2] = C * iRp * iRp;
        c[3] = (-s * v1 + co * v2) * iR + real(2) * B * iR * iR;
        c[4] = (co * v1 + s * v2) * iRp - (Bp + C * (real(1) - q)) * iR * iRp;
    }
    c[5] = (real)I.f0;
}



// Monomial coefficients of the biquadratic interpolant P(s, t) of eq.
// (Lagrange_2D) around the patch centre, c_kl of s^k t^l, plus the lift
// constant C0 of eq. (C_0):
//   index 0: C0, 1: c10, 2: c01, 3: c20, 4: c11, 5: c02, 6: c21, 7: c12, 8: c22.
// The lift of eq. (Lifting) with central macro differences is
//   u0 = C0 + c10 s + c01 t + c20 s^2 + c11 s t + c02 t^2.
template <typename real>
struct Poly {
    real C0, c10, c01, c20, c11, c02, c21, c12, c22;
};

template <typename real>
struct PatchGeo {
    real hx, hy, dx, dy;
    int nx, ny;   // nano intervals (m - 1)
    __device__ __forceinline__ real s(int a) const { return real(-0.5) * hx + real(a) * dx; }
    __device__ __forceinline__ real t(int b) const { return real(-0.5) * hy + real(b) * dy; }
};

// The same geometry with the micro coordinates read from tables (s(a) at
// sv[a + 1], t(b) at tv[b + 1], a, b = -1 .. m): no integer -> float
// conversion per use, which matters in per-point loops (conversions issue on
// the slow FP64 pipe of this part).
template <typename real>
struct PatchGeoTab {
    real hx, hy, dx, dy;
    int nx, ny;
    const real* sv;
    const real* tv;
    __device__ __forceinline__ real s(int a) const { return sv[a + 1]; }
    __device__ __forceinline__ real t(int b) const { return tv[b + 1]; }
};

// d/dxi of (P - u0): the part of the Neumann data of eq. (edge) that the
// quadratic lift does not carry.
template <typename real>
__device__ __forceinline__ real edge_gap_xi(const Poly<real>& c, real s, real t)
{
    return t * (real(2) * c.c21 * s + c.c12 * t + real(2) * c.c22 * s * t);
}
// d/deta of (P - u0)
template <typename real>
__device__ __forceinline__ real edge_gap_eta(const Poly<real>& c, real s, real t)
{
    return s * (c.c21 * s + real(2) * c.c12 * t + real(2) * c.c22 * s * t);
}

// Ghost-point value minus the quadratic lift extended to the ghost position
// (a', b'), for the ghost rule: eta-ghost rows from the bottom/top Neumann data,
// then xi-ghost columns (corners included) from the left/right data.
template <typename real, typename Geo>
__device__ __forceinline__ real ghost_offset(const Poly<real>& c, const Geo& g, int ap, int bp)
{
    real v = real(0);
    int ain = ap;
    if (ap < 0) { v -= real(2) * g.dx * edge_gap_xi(c, real(-0.5) * g.hx, g.t(bp)); ain = 1; }
    else if (ap > g.nx) { v += real(2) * g.dx * edge_gap_xi(c, real(0.5) * g.hx, g.t(bp)); ain = g.nx - 1; }
    if (bp < 0) v -= real(2) * g.dy * edge_gap_eta(c, g.s(ain), real(-0.5) * g.hy);
    else if (bp > g.ny) v += real(2) * g.dy * edge_gap_eta(c, g.s(ain), real(0.5) * g.hy);
    return v;
}

// Micro operator weights at one point (not scaled by dt).
template <typename real>
struct PointW {
    real wE, wW, wN, wS, wX, wC;   // neighbour / centre weights of L_h
    real ox, oy;                   // offset of the first-difference point (upwind: -+d/2)
};

template <typename real>
__device__ __forceinline__ PointW<real> point_weights(real al, real be, real ga, real nu, real om, real ph,
                                                      real dx, real dy, int conv)
{
    PointW<real> w;
    real ax = al / (dx * dx), gy = ga / (dy * dy);
    w.wX = be / (real(4) * dx * dy);
    w.wC = -real(2) * ax - real(2) * gy + ph;
    if (conv == PD_CONV_CENTRAL) {
        w.wE = ax - nu / (real(2) * dx); w.wW = ax + nu / (real(2) * dx);
        w.wN = gy - om / (real(2) * dy); w.wS = gy + om / (real(2) * dy);
        w.ox = real(0); w.oy = real(0);
    } else {
        if (nu > real(0)) { w.wW = ax + nu / dx; w.wE = ax; w.wC -= nu / dx; w.ox = real(-0.5) * dx; }
        else              { w.wE = ax - nu / dx; w.wW = ax; w.wC += nu / dx; w.ox = real(0.5) * dx; }
        if (om > real(0)) { w.wS = gy + om / dy; w.wN = gy; w.wC -= om / dy; w.oy = real(-0.5) * dy; }
        else              { w.wN = gy - om / dy; w.wS = gy; w.wC += om / dy; w.oy = real(0.5) * dy; }
    }
    return w;
}

// The instance constants in the working precision, converted once per patch
// group: a double -> float conversion issues on the FP64 pipe, which on this
// part runs at a small fraction of the FP32 rate.
template <typename real>
struct RealConsts {
    real K11, K12, K22, v1, v2, f0;
    real idx, idy, idx2, idy2, i4dxdy, dx, dy;
    const real* col;             // 1-D metric tables in the working precision
    const real* row;
};

template <typename real>
__device__ __forceinline__ RealConsts<real> real_consts(const InstDev& I)
{
    RealConsts<real> k;
    if constexpr (sizeof(real) == 4) {
        k.K11 = I.kf[0]; k.K12 = I.kf[1]; k.K22 = I.kf[2];
        k.v1 = I.kf[3]; k.v2 = I.kf[4]; k.f0 = I.kf[5];
        k.idx = I.kf[6]; k.idy = I.kf[7]; k.idx2 = I.kf[8]; k.idy2 = I.kf[9];
        k.i4dxdy = I.kf[10]; k.dx = I.kf[11]; k.dy = I.kf[12];
        k.col = I.col_tab_f; k.row = I.row_tab_f;
    } else {
        k.K11 = I.K11; k.K12 = I.K12; k.K22 = I.K22;
        k.v1 = I.v1; k.v2 = I.v2; k.f0 = I.f0;
        k.idx = I.inv_dx; k.idy = I.inv_dy; k.idx2 = I.inv_dx2; k.idy2 = I.inv_dy2;
        k.i4dxdy = I.inv_4dxdy; k.dx = I.dx; k.dy = I.dy;
        k.col = I.col_tab; k.row = I.row_tab;
    }
    return k;
}

// table_coeffs with the constants and tables already in the working precision
template <typename real>
__device__ __forceinline__ void table_coeffs_k(const InstDev& I, const RealConsts<real>& k, int ic, int a, int jr, int b,
                                               real c[6])
{
    const real* ct = k.col + ((size_t)ic * I.mx + a) * 2;
    const real* rt = k.row + ((size_t)jr * I.my + b) * 4;
    if (I.coef_mode == COEF_SEPARABLE) {
        const real ia = ct[0], ia2 = ct[1], ib = rt[0], ib2 = rt[1];
        c[0] = k.K11 * ia * ia;
        c[1] = real(2) * k.K12 * ia * ib;
        c[2] = k.K22 * ib * ib;
        c[3] = k.v1 * ia + k.K11 * ia2;
        c[4] = k.v2 * ib + k.K22 * ib2;
    } else {
        const real s = ct[0], co = ct[1];
        const real iR = rt[0], iRp = rt[1], q = rt[2];
        const real ss = s * s, cc = co * co, sc = s * co;
        const real A = ss * k.K11 - real(2) * sc * k.K12 + cc * k.K22;
        const real B = sc * (k.K22 - k.K11) + (cc - ss) * k.K12;
        const real C = cc * k.K11 + real(2) * sc * k.K12 + ss * k.K22;
        const real Bp = (cc - ss) * (k.K22 - k.K11) - real(4) * sc * k.K12;
        c[0] = A * iR * iR;
        c[1] = real(2) * B * iR * iRp;
        c[2] = C * iRp * iRp;
        c[3] = (-s * k.v1 + co * k.v2) * iR + real(2) * B * iR * iR;
        c[4] = (co * k.v1 + s * k.v2) * iRp - (Bp + C * (real(1) - q)) * iR * iRp;
    }
    c[5] = k.f0;
}

// point_weights_fast with the constants already in the working precision
template <typename real>
__device__ __forceinline__ PointW<real> point_weights_k(const InstDev& I, const RealConsts<real>& k, real al, real be,
                                                        real ga, real nu, real om, real ph)
{
    PointW<real> w;
    real ax = al * k.idx2, gy = ga * k.idy2;
    w.wX = be * k.i4dxdy;
    w.wC = -real(2) * ax - real(2) * gy + ph;
    if (I.conv == PD_CONV_CENTRAL) {
        real hn = real(0.5) * nu * k.idx, ho = real(0.5) * om * k.idy;
        w.wE = ax - hn; w.wW = ax + hn;
        w.wN = gy - ho; w.wS = gy + ho;
        w.ox = real(0); w.oy = real(0);
    } else {
        real nx = nu * k.idx, oy = om * k.idy;
        if (nu > real(0)) { w.wW = ax + nx; w.wE = ax; w.wC -= nx; w.ox = real(-0.5) * k.dx; }
        else              { w.wE = ax - nx; w.wW = ax; w.wC += nx; w.ox = real(0.5) * k.dx; }
        if (om > real(0)) { w.wS = gy + oy; w.wN = gy; w.wC -= oy; w.oy = real(-0.5) * k.dy; }
        else              { w.wN = gy - oy; w.wS = gy; w.wC += oy; w.oy = real(0.5) * k.dy; }
    }
    return w;
}

// raw coefficients (alpha, beta, gamma, nu, omega, phi, G, 0) of micro point (a, b)
// of patch (ic, jr), from the tables or the per-point records
template <typename real>
__device__ __forceinline__ void point_coeffs(const InstDev& I, int jr, int ic, int a, int b, real v[8])
{
    if (I.coef_mode != COEF_RECORDS) {
        real c[6];
        table_coeffs<real>(I, ic, a, jr, b, c);
        for (int k = 0; k < 6; ++k) v[k] = c[k];
        v[6] = real(0); v[7] = real(0);
    } else {
        const real* r = static_cast<const real*>(I.rec) + ((((long long)jr * I.my + b) * I.ncols + ic) * I.mx + a) * 8;
        for (int k = 0; k < 8; ++k) v[k] = r[k];
    }
}

// stencil weights of L_h without divisions (reciprocal nano steps from InstDev)
template <typename real>
__device__ __forceinline__ PointW<real> point_weights_fast(const InstDev& I, real al, real be, real ga, real nu,
                                                           real om, real ph)
{
    PointW<real> w;
    const real idx = (real)I.inv_dx, idy = (real)I.inv_dy;
    real ax = al * (real)I.inv_dx2, gy = ga * (real)I.inv_dy2;
    w.wX = be * (real)I.inv_4dxdy;
    w.wC = -real(2) * ax - real(2) * gy + ph;
    if (I.conv == PD_CONV_CENTRAL) {
        real hn = real(0.5) * nu * idx, ho = real(0.5) * om * idy;
        w.wE = ax - hn; w.wW = ax + hn;
        w.wN = gy - ho; w.wS = gy + ho;
        w.ox = real(0); w.oy = real(0);
    } else {
        real nx = nu * idx, oy = om * idy;
        if (nu > real(0)) { w.wW = ax + nx; w.wE = ax; w.wC -= nx; w.ox = real(-0.5) * (real)I.dx; }
        else              { w.wE = ax - nx; w.wW = ax; w.wC += nx; w.ox = real(0.5) * (real)I.dx; }
        if (om > real(0)) { w.wS = gy + oy; w.wN = gy; w.wC -= oy; w.oy = real(-0.5) * (real)I.dy; }
        else              { w.wN = gy - oy; w.wS = gy; w.wC += oy; w.oy = real(0.5) * (real)I.dy; }
    }
    return w;
}

// Burst forcing r = L_h(u0 with its ghost points) + s(T) G at micro point (a, b),
// evaluated in closed form: the centred second and cross differences of the
// quadratic lift are exact, a two-point difference of it is its derivative at
// the midpoint, and every ghost neighbour adds weight * ghost_offset.  No
// difference of nearly equal lifted values is formed, so FP32 evaluation keeps
// full relative precision.
template <typename real, typename Geo>
__device__ __forceinline__ real burst_forcing(const Poly<real>& c, const Geo& g, int a, int b,
                                              real al, real be, real ga, real nu, real om, real ph,
                                              real G, real sT, const PointW<real>& w)
{
    real s = g.s(a), t = g.t(b);
    real u0 = c.C0 + s * (c.c10 + s * c.c20 + t * c.c11) + t * (c.c01 + t * c.c02);
    real ux = c.c10 + real(2) * c.c20 * (s + w.ox) + c.c11 * t;
    real uy = c.c01 + real(2) * c.c02 * (t + w.oy) + c.c11 * s;
    real r = real(2) * c.c20 * al + c.c11 * be + real(2) * c.c02 * ga - nu * ux - om * uy + ph * u0 + sT * G;
    if (a == 0) r += w.wW * ghost_offset(c, g, -1, b);
    if (a == g.nx) r += w.wE * ghost_offset(c, g, g.nx + 1, b);
    if (b == 0) r += w.wS * ghost_offset(c, g, a, -1);
    if (b == g.ny) r += w.wN * ghost_offset(c, g, a, g.ny + 1);
    if (be != real(0) && (a == 0 || a == g.nx || b == 0 || b == g.ny)) {
        auto out = [&](int ap, int bp) { return ap < 0 || ap > g.nx || bp < 0 || bp > g.ny; };
        if (out(a + 1, b + 1)) r += w.wX * ghost_offset(c, g, a + 1, b + 1);
        if (out(a - 1, b - 1)) r += w.wX * ghost_offset(c, g, a - 1, b - 1);
        if (out(a + 1, b - 1)) r -= w.wX * ghost_offset(c, g, a + 1, b - 1);
        if (out(a - 1, b + 1)) r -= w.wX * ghost_offset(c, g, a - 1, b + 1);
    }
    return r;
}

// burst_forcing without its ghost-neighbour terms: the closed form of
// L_h(u_lift) + s(T) G, for kernels that form the ghost terms their own way.
template <typename real, typename Geo>
__device__ __forceinline__ real burst_forcing_base(const Poly<real>& c, const Geo& g, int a, int b,
                                                   real al, real be, real ga, real nu, real om, real ph,
                                                   real G, real sT, const PointW<real>& w)
{
    real s = g.s(a), t = g.t(b);
    real u0 = c.C0 + s * (c.c10 + s * c.c20 + t * c.c11) + t * (c.c01 + t * c.c02);
    real ux = c.c10 + real(2) * c.c20 * (s + w.ox) + c.c11 * t;
    real uy = c.c01 + real(2) * c.c02 * (t + w.oy) + c.c11 * s;
    return real(2) * c.c20 * al + c.c11 * be + real(2) * c.c02 * ga - nu * ux - om * uy + ph * u0 + sT * G;
}


// time factor s(t) of the source
__device__ __forceinline__ double time_factor(int kind, double c, double t)
{
    if (kind == PD_TIME_EXP) return exp(c * t);
    if (kind == PD_TIME_SIN) return sin(c * t);
    return 1.0;
}

__device__ __forceinline__ double exact_solution(int sol, double x, double y, double t)
{
    if (sol == PD_SOL_EXP_XYT) return exp(x + y + t);
    if (sol == PD_SOL_SINPROD_DECAY) return exp(-t) * sinpi(x) * sinpi(y);
    return 0.0;
}

enum ErrBits { ERR_NONFINITE = 1, ERR_JACOBIAN = 2, ERR_COEF = 4, ERR_TIMEOUT = 8 };

// An NVTX range named after a C-ABI call for the lifetime of the object, so
// profilers show each call's kernels under it (header-only NVTX: inert when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Makes `dev` the calling thread's current device for the lifetime of the
// guard and restores the caller's device afterwards, so a host thread that
// drives several devices finds its current device unchanged after any call.
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) switched = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (switched) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// ---------------------------------------------------------------------------
// host-side launch helpers (defined in the .cu files)
struct StepLaunch {
    const InstDev* inst_dev;   // device copy
    const InstDev* inst_host;  // host copy
    const double* Uc;
    double* Un;
    const double* tab;         // time table row of this macro step
    double dtm;
};

cudaError_t launch_precompute(const InstDev& I, const pd_coeff_desc& c, const double* amp_dev,
                              void* rec, int prec, unsigned long long* rate_max,
                              unsigned long long* macro_rate_max, cudaStream_t st);
cudaError_t launch_burst_records(const InstDev& I, int prec, void* brec, cudaStream_t st);
cudaError_t launch_get_coeffs(const InstDev& I, int prec, double* out, cudaStream_t st);
cudaError_t launch_init_field(const InstDev& I, const pd_coeff_desc& c, int kind, const double* prm,
                              int n_prm, const double* mu, double t, double* U, cudaStream_t st);
cudaError_t launch_time_table(const InstDev& I, double t0, double dtm, int n_steps, double* tab,
                              cudaStream_t st);
cudaError_t launch_fused_step(const InstDev& I, const InstDev* I_dev, int prec, const double* Uc,
                              double* Un, const double* tab_row, double dtm, cudaStream_t st,
                              int* n_launch);
cudaError_t launch_lift(const InstDev& I, const InstDev* I_dev, int prec, const double* U, double t,
                        char* state, const pd_info& lay, cudaStream_t st);
cudaError_t launch_burst(const InstDev& I, const InstDev* I_dev, int prec, char* state,
                         const pd_info& lay, double t, int k_steps, cudaStream_t st);
// bias_override: per-patch reference offsets to add instead of the state's
// bias section (global patch index), e.g. zeros for the change of the departure
cudaError_t launch_restrict(const InstDev& I, int prec, const char* state, const pd_info& lay,
                            double* dU, cudaStream_t st, const double* bias_override = nullptr);
cudaError_t launch_project(const InstDev& I, double* U, const double* dU, double t, double dtm,
                           cudaStream_t st);
bool fused_supported(const InstDev& I);
// read access to one instance of a grid for the other parts of the library
struct GridAccess {
    InstDev I;                       // host copy; pointers are device pointers
    pd_coeff_desc coef;
    int prec = 0;
    int n_inst = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    double dtm_sugg = 0.0;
};
}  // namespace pd
struct pd_grid;
namespace pd {
// PD_ESTATE when the instance's coefficients are not set
pd_status grid_access(pd_grid* g, int inst, GridAccess& out);
void grid_message(pd_grid* g, const char* msg);
void grid_count_launches(pd_grid* g, long long n);

// restricted change of every patch (or of the *list_n patches of list) after
// k_steps micro steps from the lift of U; tab_row is a time-table row built
// for k_steps
// ADI micro solver (pd_adi.cu): line records once per pd_set_coeffs, and the
// fused macro step / restricted change with ADI bursts
cudaError_t launch_adi_records(const InstDev& I, int prec, void* arec_c, void* arec_r, cudaStream_t st);
cudaError_t launch_adi_fused(const InstDev& I, int prec, const double* Uc, double* Un, const double* tab_row,
                             double dtm, cudaStream_t st);
cudaError_t launch_adi_dU(const InstDev& I, int prec, const double* U, const double* tab_row, double* dU,
                          const int* list, const int* list_n, cudaStream_t st);
// edge-data refresh (pd_refresh.cu): D = V_q - V_{q-1} on the macro nodes, then
// r += e(D) at the edge points of every patch
cudaError_t launch_refresh(const InstDev& I, int prec, const double* U, const double* dR_cur, const double* dR_prev,
                           double t_prev, double t_cur, int first, double* D, void* r_state, cudaStream_t st);
cudaError_t launch_patch_dU(const InstDev& I, int prec, const double* U, const double* tab_row, int k_steps,
                            double* dU, const int* list, const int* list_n, cudaStream_t st);
// second-order outer integrators: Heun's combination and the AB2 update
cudaError_t launch_heun_combine(const InstDev& I, double* U, const double* S1, const double* S2, cudaStream_t st);
cudaError_t launch_ab2(const InstDev& I, double* U, const double* dUn, const double* dUp, double t, double dtm,
                       cudaStream_t st);
// per-patch basis T[p][10] of the one-micro-step restricted change over dt
cudaError_t launch_one_step_basis(const InstDev& I, int prec, double* T, cudaStream_t st);
// per-patch surrogate features that do not depend on U (10 per patch) and the
// macro explicit rate R at the patch centre
cudaError_t launch_surrogate_static(const InstDev& I, const pd_coeff_desc& c, double tau, float* feat, double* R,
                                    cudaStream_t st);
bool batch_supported(const InstDev& I);

// Persistent dataflow launch of n_steps macro steps (see pd_persist.cu).
struct PersistArgs {
    double* U0;            // buffer of even steps (the caller's field)
    double* U1;            // buffer of odd steps (library scratch)
    const double* tab;     // time table of the whole pd_step call
    int s0, n_steps;       // first step of this chunk, steps in this chunk
    double dtm;
    int* flags;            // one step counter per item warp (zeroed before the launch)
    const int* bnd_off;    // CSR: boundary nodes owned by each item warp
    const int* bnd_idx;
    long long wait_ns;     // give up a neighbour wait after this many ns
    int silent_warp;       // test hook: this item warp never publishes (-1: none)
};
// 1-D metric tables (table coefficient mode) and batched execution
cudaError_t launch_tables(const InstDev& I, double* col_tab, double* row_tab, float* col_tab_f, float* row_tab_f, unsigned long long* rate_max,
                          unsigned long long* macro_rate_max, cudaStream_t st);
cudaError_t launch_table_get_coeffs(const InstDev& I, double* out, cudaStream_t st);
struct BatchItem {
    int inst;      // instance index
    int kind;      // 0: patch group (row jr, warp column wc), 1: 32 boundary nodes (chunk jr)
    int jr, wc;
};
struct BatchArgs {
    const InstDev* insts;      // device array
    const BatchItem* items;
    int n_items;
    int* counter;              // work-queue counter of this macro step (zeroed)
    double* Ubase;             // caller's field (all instances)
    double* Sbase;             // scratch field
    int parity;                // step parity: reads Ubase if 0
    const double* dtm;         // per-instance macro step
    const double2* scale;      // per instance: (dtm / (tau (m_xi - 1)(m_eta - 1)), dtm / tau), formed on the host
    const double* tab;         // per-instance time tables (nullable)
    const long long* tab_off;  // per-instance offset of the table of this pd_step
    int step;                  // macro step index within the pd_step call
};
// one launch covers the items of the instances with micro size M (M x M patches)
// sep: the separable-map patch groups of one micro size (FP32 only), run by
// kernels whose burst keeps the column-only east/west weights per lane
cudaError_t launch_batch(int prec, bool tsrc, int M, bool sep, const BatchArgs& a, int block, int grid,
                         cudaStream_t st);
int batch_blocks_per_sm(int prec, bool tsrc, int M, bool sep, int block);
cudaError_t launch_batch_time_tables(const InstDev* insts, int n_inst, const double* dtm, double t0, int n_macro,
                                     const long long* tab_off, double* tab, long long total, cudaStream_t st);
int persist_item_warps(const InstDev& I);
size_t persist_smem_bytes(const InstDev& I, size_t es, int n_steps);
int persist_max_steps(const InstDev& I, int prec);
bool persist_fits(const InstDev& I, int prec);
cudaError_t launch_persist(const InstDev& I, int prec, const PersistArgs& a, cudaStream_t st);

}  // namespace pd

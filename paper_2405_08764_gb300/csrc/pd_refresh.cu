// Edge-data refresh during the burst (Q > 1).  Section 3 keeps the Neumann
// data of eq. (edge) fixed over the burst and names their refresh as the more
// accurate alternative.  The burst is cut into Q sub-bursts of K/Q steps;
// before sub-burst q the edge data are rebuilt from the macro estimate
// V_q = U + (restricted change of the departure so far) on interior nodes and
// the Dirichlet data at the sub-burst start time on boundary nodes.
//
// In the split form u = u_lift + w the lift keeps the lifted edge data, so
// the departure's ghost points carry the difference of the edge data; in the
// micro operator that difference acts only through the ghost neighbours of
// the edge points, as an added forcing e at those points.  e is linear in the
// macro field, so the forcing of the micro state is updated by e(V_q - V_{q-1})
// before each sub-burst: refresh_field_kernel forms the increment field
// D = V_q - V_{q-1} on the macro nodes and refresh_kernel adds e(D) to r at
// the edge points (any m <= 32, both precisions).
#include "pd_device.cuh"

#include <math.h>

namespace pd {

namespace {

// D = V_q - V_{q-1}: on the node of patch k the change of its restricted change
// (dR_cur - dR_prev); on boundary nodes the change of the Dirichlet data, from
// the field U itself for the first refresh.
__global__ void refresh_field_kernel(const InstDev I, const double* __restrict__ U, const double* __restrict__ dR_cur,
                                     const double* __restrict__ dR_prev, double t_prev, double t_cur, int first,
                                     double* __restrict__ D)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < I.n_patch) {
        const int jr = k / I.ncols, ic = k - jr * I.ncols;
        const long long node = (long long)(1 + jr) * I.nxp + I.i0 + ic;
        const long long pg = (long long)I.p_off + k;
        D[node] = dR_cur[pg] - dR_prev[pg];
    } else if (k < I.n_patch + I.n_bnd) {
        const int b = k - I.n_patch;
        const int2 ij = I.bnd_ij[b];
        const double2 xy = I.bnd_xy[b];
        const long long node = (long long)ij.y * I.nxp + ij.x;
        const double prev = first ? U[node] : exact_solution(I.sol, xy.x, xy.y, t_prev);
        D[node] = exact_solution(I.sol, xy.x, xy.y, t_cur) - prev;
    }
}

// derivatives of the biquadratic interpolant with monomial coefficients c
__device__ __forceinline__ double dxi_poly(const double c[9], double s, double t)
{
    return c[1] + 2.0 * c[3] * s + c[4] * t + 2.0 * c[6] * s * t + c[7] * t * t + 2.0 * c[8] * s * t * t;
}

__device__ __forceinline__ double deta_poly(const double c[9], double s, double t)
{
    return c[2] + 2.0 * c[5] * t + c[4] * s + c[6] * s * s + 2.0 * c[7] * s * t + 2.0 * c[8] * s * s * t;
}

// change of the ghost value at (ap, bp) (outside the patch) for the edge-data
// change of the interpolant c, in the ghost order of the explicit scheme:
// eta-ghost rows from the bottom/top data, then xi-ghost columns (corners
// included) from the left/right data
__device__ __forceinline__ double ghost_delta(const double c[9], const PatchGeo<double>& g, int ap, int bp)
{
    double v = 0.0;
    int ain = ap;
    if (ap < 0) { v -= 2.0 * g.dx * dxi_poly(c, -0.5 * g.hx, g.t(bp)); ain = 1; }
    else if (ap > g.nx) { v += 2.0 * g.dx * dxi_poly(c, 0.5 * g.hx, g.t(bp)); ain = g.nx - 1; }
    if (bp < 0) v -= 2.0 * g.dy * deta_poly(c, g.s(ain), -0.5 * g.hy);
    else if (bp > g.ny) v += 2.0 * g.dy * deta_poly(c, g.s(ain), 0.5 * g.hy);
    return v;
}

// one thread per micro point; interior points return at once
template <typename real>
__global__ void refresh_kernel(const InstDev I, const double* __restrict__ D, const real* __restrict__ rec,
                               real* __restrict__ r)
{
    const long long n = (long long)I.n_patch * I.mx * I.my;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int mm = I.mx * I.my;
    const int p = (int)(idx / mm);
    const int rem = (int)(idx - (long long)p * mm);
    const int b = rem / I.mx, a = rem - b * I.mx;
    const int nx = I.mx - 1, ny = I.my - 1;
    if (a != 0 && a != nx && b != 0 && b != ny) return;
    const int jr = p / I.ncols, ic = p - jr * I.ncols;
    const int i = I.i0 + ic, j = 1 + jr;
    // monomial coefficients of the interpolant of D (the constant term is not needed)
    double st[9];
    for (int pp = 0; pp < 3; ++pp)
        for (int qq = 0; qq < 3; ++qq)
            st[pp * 3 + qq] = D[(long long)(j + qq - 1) * I.nxp + wrap_col(I, i + pp - 1)];
    double c[9];
    c[0] = 0.0;
    for (int k = 1; k < 9; ++k) {
        double v = 0.0;
        for (int q = 0; q < 9; ++q) v = fma(I.lw[k][q], st[q], v);
        c[k] = v;
    }
    const long long pt = (((long long)jr * I.my + b) * I.ncols + ic) * I.mx + a;
    const real* cr = rec + pt * 8;
    PointW<double> w = point_weights<double>((double)cr[0], (double)cr[1], (double)cr[2], (double)cr[3],
                                             (double)cr[4], (double)cr[5], I.dx, I.dy, I.conv);
    PatchGeo<double> g = { I.hx, I.hy, I.dx, I.dy, nx, ny };
    double e = 0.0;
    if (a == 0) e += w.wW * ghost_delta(c, g, -1, b);
    if (a == nx) e += w.wE * ghost_delta(c, g, nx + 1, b);
    if (b == 0) e += w.wS * ghost_delta(c, g, a, -1);
    if (b == ny) e += w.wN * ghost_delta(c, g, a, ny + 1);
    if ((double)cr[1] != 0.0) {
        auto out = [&](int ap, int bp) { return ap < 0 || ap > nx || bp < 0 || bp > ny; };
        if (out(a + 1, b + 1)) e += w.wX * ghost_delta(c, g, a + 1, b + 1);
        if (out(a - 1, b - 1)) e += w.wX * ghost_delta(c, g, a - 1, b - 1);
        if (out(a + 1, b - 1)) e -= w.wX * ghost_delta(c, g, a + 1, b - 1);
        if (out(a - 1, b + 1)) e -= w.wX * ghost_delta(c, g, a - 1, b + 1);
    }
    real* rp = r + I.pt_off + idx;
    *rp = (real)((double)*rp + e);
}

}  // namespace

cudaError_t launch_refresh(const InstDev& I, int prec, const double* U, const double* dR_cur, const double* dR_prev,
                           double t_prev, double t_cur, int first, double* D, void* r_state, cudaStream_t st)
{
    const int nn = I.n_patch + I.n_bnd;
    refresh_field_kernel<<<(nn + 127) / 128, 128, 0, st>>>(I, U, dR_cur, dR_prev, t_prev, t_cur, first, D);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = (long long)I.n_patch * I.mx * I.my;
    const unsigned nb = (unsigned)((n + 127) / 128);
    if (prec == PD_FP32)
        refresh_kernel<float><<<nb, 128, 0, st>>>(I, D, static_cast<const float*>(I.rec), static_cast<float*>(r_state));
    else
        refresh_kernel<double><<<nb, 128, 0, st>>>(I, D, static_cast<const double*>(I.rec), static_cast<double*>(r_state));
    return cudaGetLastError();
}

}  // namespace pd

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
// the edge points (any m <= 32, both precisions, in the grid's working
// precision).
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
template <typename real>
__device__ __forceinline__ real dxi_poly(const real (&c)[9], real s, real t)
{
    return c[1] + real(2) * c[3] * s + c[4] * t + real(2) * c[6] * s * t + c[7] * t * t + real(2) * c[8] * s * t * t;
}

template <typename real>
__device__ __forceinline__ real deta_poly(const real (&c)[9], real s, real t)
{
    return c[2] + real(2) * c[5] * t + c[4] * s + c[6] * s * s + real(2) * c[7] * s * t + real(2) * c[8] * s * s * t;
}

// change of the ghost value at (ap, bp) (outside the patch) for the edge-data
// change of the interpolant c, in the ghost order of the explicit scheme:
// eta-ghost rows from the bottom/top data, then xi-ghost columns (corners
// included) from the left/right data
template <typename real>
__device__ __forceinline__ real ghost_delta(const real (&c)[9], const PatchGeo<real>& g, int ap, int bp)
{
    real v = real(0);
    int ain = ap;
    if (ap < 0) { v -= real(2) * g.dx * dxi_poly(c, real(-0.5) * g.hx, g.t(bp)); ain = 1; }
    else if (ap > g.nx) { v += real(2) * g.dx * dxi_poly(c, real(0.5) * g.hx, g.t(bp)); ain = g.nx - 1; }
    if (bp < 0) v -= real(2) * g.dy * deta_poly(c, g.s(ain), real(-0.5) * g.hy);
    else if (bp > g.ny) v += real(2) * g.dy * deta_poly(c, g.s(ain), real(0.5) * g.hy);
    return v;
}

// One warp per patch.  Lane s < 9 forms stencil difference s of D in FP64
// (the slots of the fused kernel: second and first differences and the
// centre value), converts it once, and coefficient k of the interpolant
// combines up to three slots in the working precision, so that no difference
// of nearly equal values is formed after the conversion.  The lanes then share
// out the 2 m_xi + 2 (m_eta - 2) edge points and add e(D) to r there, in the
// working precision; instance constants and slot weights are converted once
// per block (a double -> float conversion issues on the FP64 pipe, a small
// fraction of the FP32 rate on this part).
// FP32: eight blocks (64 warps) per SM at 32 registers.  The kernel is a chain
// of dependent latencies per warp, so more warps in flight pay more than the
// few values the tighter register budget moves to local memory (measured).
template <typename real>
__global__ void __launch_bounds__(256, (sizeof(real) == 4 ? 8 : 1))
refresh_kernel(const InstDev I, const double* __restrict__ D, const real* __restrict__ rec, real* __restrict__ r)
{
    __shared__ real cw_s[9][3];
    __shared__ int slot_s[9][3];
    __shared__ RealConsts<real> kc_s;
    __shared__ PatchGeo<real> g_s;
    for (int t = threadIdx.x; t < 27; t += blockDim.x) {
        cw_s[t / 3][t % 3] = (real)I.c2w[t / 3][t % 3];
        slot_s[t / 3][t % 3] = I.c2slot[t / 3][t % 3];
    }
    if (threadIdx.x == 0) {
        kc_s = real_consts<real>(I);
        g_s = PatchGeo<real>{ (real)I.hx, (real)I.hy, (real)I.dx, (real)I.dy, I.mx - 1, I.my - 1 };
    }
    __syncthreads();
    const int p = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (p >= I.n_patch) return;                      // whole warp
    const int jr = p / I.ncols, ic = p - jr * I.ncols;
    const int i = I.i0 + ic, j = 1 + jr;
    const int n_edge = 2 * I.mx + 2 * (I.my - 2);
    const int nx = I.mx - 1, ny = I.my - 1;
    auto edge_point = [&](int e, int& a, int& b) {
        if (e < I.mx) { a = e; b = 0; }
        else if (e < 2 * I.mx) { a = e - I.mx; b = ny; }
        else { const int t = e - 2 * I.mx; b = 1 + (t >> 1); a = (t & 1) ? nx : 0; }
    };
    // the first edge point's record and forcing do not depend on D: load them
    // before the stencil so that the memory latencies overlap
    int a0 = 0, b0 = 0;
    real rc0[6] = { real(0), real(0), real(0), real(0), real(0), real(0) }, r0v = real(0);
    real* const rbase = r + I.pt_off + (long long)p * I.mx * I.my;
    if (lane < n_edge) {
        edge_point(lane, a0, b0);
        const real* cr = rec + ((((long long)jr * I.my + b0) * I.ncols + ic) * I.mx + a0) * 8;
        real c6, c7;
        load_vec4<real>(cr, rc0[0], rc0[1], rc0[2], rc0[3]);
        load_vec4<real>(cr + 4, rc0[4], rc0[5], c6, c7);
        (void)c6; (void)c7;
        r0v = rbase[b0 * I.mx + a0];
    }
    const real sv = lane < 9 ? (real)stencil_slot<false>(I, D, i, j, lane) : real(0);
    real ck = real(0);                               // lane k: coefficient k (the constant term is not needed)
    {
        const int k = lane < 9 ? lane : 0;
        const real P0 = __shfl_sync(kFull, sv, slot_s[k][0]);
        const real P1 = __shfl_sync(kFull, sv, slot_s[k][1]);
        const real P2 = __shfl_sync(kFull, sv, slot_s[k][2]);
        if (lane >= 1 && lane < 9) ck = cw_s[k][2] * fma(cw_s[k][1], P2, fma(cw_s[k][0], P1, P0));
    }
    real c[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) c[k] = __shfl_sync(kFull, ck, k);
    const RealConsts<real> kc = kc_s;
    const PatchGeo<real> g = g_s;
    for (int e = lane; e < n_edge; e += 32) {
        int a, b;
        real cc[6], rv;
        if (e == lane) {
            a = a0; b = b0;
            for (int k = 0; k < 6; ++k) cc[k] = rc0[k];
            rv = r0v;
        } else {
            edge_point(e, a, b);
            const real* cr = rec + ((((long long)jr * I.my + b) * I.ncols + ic) * I.mx + a) * 8;
            for (int k = 0; k < 6; ++k) cc[k] = cr[k];
            rv = rbase[b * I.mx + a];
        }
        const real be = cc[1];
        const PointW<real> w = point_weights_k<real>(I, kc, cc[0], be, cc[2], cc[3], cc[4], cc[5]);
        // W/E and S/N ghosts without branches: the W/E ghost changes by -+2 dx d/dxi
        // at the left/right edge s, the S/N ghost by -+2 dy d/deta at the bottom/top
        // edge t (zero weight on the sides the point is not on)
        const real se = a == 0 ? real(-0.5) * g.hx : real(0.5) * g.hx;
        const real te = b == 0 ? real(-0.5) * g.hy : real(0.5) * g.hy;
        const real wx = a == 0 ? -w.wW : (a == nx ? w.wE : real(0));
        const real wy = b == 0 ? -w.wS : (b == ny ? w.wN : real(0));
        real v = wx * (real(2) * g.dx * dxi_poly(c, se, g.t(b))) + wy * (real(2) * g.dy * deta_poly(c, g.s(a), te));
        if (be != real(0)) {
            auto out = [&](int ap, int bp) { return ap < 0 || ap > nx || bp < 0 || bp > ny; };
            if (out(a + 1, b + 1)) v += w.wX * ghost_delta(c, g, a + 1, b + 1);
            if (out(a - 1, b - 1)) v += w.wX * ghost_delta(c, g, a - 1, b - 1);
            if (out(a + 1, b - 1)) v -= w.wX * ghost_delta(c, g, a + 1, b - 1);
            if (out(a - 1, b + 1)) v -= w.wX * ghost_delta(c, g, a - 1, b + 1);
        }
        rbase[b * I.mx + a] = rv + v;
    }
}

}  // namespace

cudaError_t launch_refresh(const InstDev& I, int prec, const double* U, const double* dR_cur, const double* dR_prev,
                           double t_prev, double t_cur, int first, double* D, void* r_state, cudaStream_t st)
{
    const int nn = I.n_patch + I.n_bnd;
    refresh_field_kernel<<<(nn + 127) / 128, 128, 0, st>>>(I, U, dR_cur, dR_prev, t_prev, t_cur, first, D);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)(((long long)I.n_patch * 32 + 255) / 256);
    if (prec == PD_FP32)
        refresh_kernel<float><<<nb, 256, 0, st>>>(I, D, static_cast<const float*>(I.rec), static_cast<float*>(r_state));
    else
        refresh_kernel<double><<<nb, 256, 0, st>>>(I, D, static_cast<const double*>(I.rec), static_cast<double*>(r_state));
    return cudaGetLastError();
}

}  // namespace pd

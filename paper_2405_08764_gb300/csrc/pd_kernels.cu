// Hot path of one macro step (Section 3.3): edge data + lift, micro burst,
// restriction and projective forward Euler.
//
// Resident micro burst.  A patch of M x M micro points lives in the registers of
// M consecutive lanes of one warp: lane a holds micro column a (M values), and
// P = 32 / M patches share a warp.  Neighbouring columns are exchanged with
// warp shuffles, neighbouring rows are in the same thread, so a micro step needs
// no shared memory and no barrier.  The Neumann ghost points of the departure
// w = u - u_lift are mirrors (their edge data is carried by the lift, see
// burst_forcing), so they are folded into the stencil weights once per burst.
// The stencil weights, the per-point forcing and the source factor stay in
// registers for all K micro steps.
//
// Precision: the monomial coefficients of the interpolant come from the FP64
// macro field with FP64 dot products (one coefficient per lane); the burst runs
// in `real` (float for PD_FP32, double for PD_FP64); the restricted change is
// divided by tau and accumulated into U in FP64.
#include "pd_device.cuh"

#include <math.h>

namespace pd {

namespace {

constexpr unsigned FULL = kFull;

enum { MODE_FUSED = 0, MODE_BURST = 1, MODE_DU = 2 };

// Burst record of one micro point (16 values, dt-scaled):
//   0..5  stencil weights cE, cW, cN, cS, cX, cC with the mirror ghosts of the
//         departure folded in (edge columns/rows take the outer weight on the
//         inner neighbour; the cross weight vanishes on the patch boundary),
//   6     Gs = dt G,
//   7..15 B_k = dt * d r / d c_k, the forcing r = L_h(u_lift) + s(T) G being
//         linear in the 9 monomial coefficients c_k of the interpolant;
//         B_k is obtained by evaluating burst_forcing at the unit vector e_k.
// Then per macro step R = dt r = sum_k B_k c_k + s(T) Gs.
template <typename real>
__global__ void burst_record_kernel(const InstDev I, const real* __restrict__ rec, real* __restrict__ brec)
{
    long long n = (long long)I.n_patch * I.mx * I.my;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    int a = (int)(idx % I.mx);
    long long r1 = idx / I.mx;
    int b = (int)((r1 / I.ncols) % I.my);
    double v[8];
    for (int k = 0; k < 8; ++k) v[k] = (double)rec[idx * 8 + k];
    PatchGeo<double> g = { I.hx, I.hy, I.dx, I.dy, I.mx - 1, I.my - 1 };
    PointW<double> pw = point_weights<double>(v[0], v[1], v[2], v[3], v[4], v[5], I.dx, I.dy, I.conv);
    double dt = I.dt;
    double e = dt * pw.wE, ww = dt * pw.wW, nn = dt * pw.wN, s = dt * pw.wS, x = dt * pw.wX;
    double cc = 1.0 + dt * pw.wC;
    if (a == 0) { e += ww; ww = 0.0; }
    if (a == I.mx - 1) { ww += e; e = 0.0; }
    if (b == 0) { nn += s; s = 0.0; }
    if (b == I.my - 1) { s += nn; nn = 0.0; }
    if (a == 0 || a == I.mx - 1 || b == 0 || b == I.my - 1) x = 0.0;
    real* o = brec + idx * 16;
    o[0] = (real)e; o[1] = (real)ww; o[2] = (real)nn; o[3] = (real)s; o[4] = (real)x; o[5] = (real)cc;
    o[6] = (real)(dt * v[6]);
    for (int k = 0; k < 9; ++k) {
        double u[9] = { 0, 0, 0, 0, 0, 0, 0, 0, 0 };
        u[k] = 1.0;
        Poly<double> ek = { u[0], u[1], u[2], u[3], u[4], u[5], u[6], u[7], u[8] };
        o[7 + k] = (real)(dt * burst_forcing<double>(ek, g, a, b, v[0], v[1], v[2], v[3], v[4], v[5], 0.0, 0.0, pw));
    }
}

// One warp = P patches of one patch row.  MODE_FUSED: lift -> burst -> restrict
// -> project for one macro step, writing U at T_next into Un.  MODE_BURST: load
// (w, r) from the micro state, run k_steps, store w.  MODE_DU: lift -> k_steps
// micro steps -> restrict, writing the restricted change of patch p into
// dU_out[p]; with a patch list, warp w takes list entries w P .. w P + P - 1
// (*list_n entries in all) instead of P neighbouring patches of one row.
template <int M, bool CROSS, bool TSRC, typename real, int MODE>
__global__ void __launch_bounds__(128, (sizeof(real) == 4 ? 4 : 1))
patch_warp_kernel(const InstDev I, const double* __restrict__ Uc, double* __restrict__ Un,
                  const double* __restrict__ tab, double upd_scale, double bias_scale, int k_steps,
                  real* __restrict__ st_w, const real* __restrict__ st_r, int n_item_warps,
                  double* __restrict__ dU_out, const int* __restrict__ list, const int* __restrict__ list_n)
{
    constexpr int P = 32 / M;
    constexpr bool LIFT = (MODE != MODE_BURST);
    constexpr int NC = (9 + M - 1) / M;
    __shared__ double lw_s[9][9];
    __shared__ int slot_s[9][3];
    __shared__ double cw_s[9][3];
    __shared__ double tinfo[3];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    real* ds_s = reinterpret_cast<real*>(dyn_smem);   // TSRC: K entries

    const int K = (MODE == MODE_FUSED) ? I.K : k_steps;
    // list-driven restricted changes: the grid covers every patch, the list only
    // some; blocks past the list's end leave before the shared-memory prologue
    if (MODE == MODE_DU && list && (int)(blockIdx.x * (blockDim.x >> 5)) * P >= *list_n) return;
    if (LIFT) {
        for (int t = threadIdx.x; t < 81; t += blockDim.x) lw_s[t / 9][t % 9] = I.lw[t / 9][t % 9];
        for (int t = threadIdx.x; t < 27; t += blockDim.x) { slot_s[t / 3][t % 3] = I.c2slot[t / 3][t % 3]; cw_s[t / 3][t % 3] = I.c2w[t / 3][t % 3]; }
    }
    if (TSRC)
        for (int t = threadIdx.x; t < K; t += blockDim.x) ds_s[t] = (real)tab[t];
    if (LIFT && threadIdx.x < 3) tinfo[threadIdx.x] = tab[K + threadIdx.x];
    __syncthreads();

    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;

    if (warp >= n_item_warps) {
        if (MODE != MODE_FUSED) return;
        // boundary nodes: Dirichlet data at T_next
        int k = (warp - n_item_warps) * 32 + lane;
        if (k < I.n_bnd) {
            int2 ij = I.bnd_ij[k];
            double2 xy = I.bnd_xy[k];
            Un[(long long)ij.y * I.nxp + ij.x] = exact_solution(I.sol, xy.x, xy.y, tinfo[2]);
        }
        return;
    }

    const int q = lane / M;
    const int a = lane - q * M;
    int jr, icl;
    bool active;
    if (MODE == MODE_DU && list) {
        const int n_list = *list_n;
        if (warp * P >= n_list) return;            // whole warp
        const int e = warp * P + q;
        active = (q < P) && (e < n_list);
        const int pid = list[active ? e : warp * P];
        jr = pid / I.ncols;
        icl = pid - jr * I.ncols;
    } else {
        const int wpr = (I.ncols + P - 1) / P;
        jr = warp / wpr;
        const int ic = (warp - jr * wpr) * P + q;
        active = (q < P) && (ic < I.ncols);
        icl = active ? ic : (I.ncols - 1);
    }
    const int i = I.i0 + icl, j = 1 + jr;
    const int qbase = (q < P ? q : P - 1) * M;
    const int pidx = jr * I.ncols + icl;

    real cv[9];
    double bias = 0.0, u00 = 0.0;
    if (LIFT) {
        double c20, c02;
        macro_coeffs<M, real, false>(I, Uc, i, j, a, qbase, lw_s, slot_s, cw_s, cv, c20, c02, u00);
        if (I.restrict_mode == PD_RESTRICT_MACRO) {
            // trapezoid average of the lift minus U_ij = (dxi^2 c20 + deta^2 c02) / 6
            bias = (I.dx * I.dx * c20 + I.dy * I.dy * c02) * (1.0 / 6.0);
        }
    }

    // per-point stencil weights, forcing and source from the burst records
    real w[M], Rr[M];
    real cE[M], cW[M], cN[M], cS[M], cC[M], cX[M], Gs[M];
    const real sT = LIFT ? (real)tinfo[0] : real(0);
    const real dt = (real)I.dt;
    const real* brec = static_cast<const real*>(I.brec);
    const long long rowstride = (long long)I.ncols * M;
    const long long base = (long long)jr * M * rowstride + (long long)icl * M + a;
    const long long sbase = I.pt_off + ((long long)jr * I.ncols + icl) * (M * M) + a;
#pragma unroll
    for (int b = 0; b < M; ++b) {
        const real* p = brec + (base + b * rowstride) * 16;
        real e, ww, n, s, x, cc, g, B0, B1, B2, B3, B4, B5, B6, B7, B8;
        load_vec4<real>(p, e, ww, n, s);
        load_vec4<real>(p + 4, x, cc, g, B0);
        real r;
        if (LIFT) {
            load_vec4<real>(p + 8, B1, B2, B3, B4);
            r = sT * g;
            r = fma(B0, cv[0], r); r = fma(B1, cv[1], r); r = fma(B2, cv[2], r);
            r = fma(B3, cv[3], r); r = fma(B4, cv[4], r);
            // B5..B8: c02 and the edge-gap terms; B6..B8 vanish away from the ghosts
            if (b == 0 || b == M - 1 || a == 0 || a == M - 1) {
                load_vec4<real>(p + 12, B5, B6, B7, B8);
                r = fma(B5, cv[5], r); r = fma(B6, cv[6], r); r = fma(B7, cv[7], r); r = fma(B8, cv[8], r);
            } else {
                B5 = p[12];
                r = fma(B5, cv[5], r);
            }
            w[b] = real(0);
        } else {
            r = dt * st_r[sbase + b * M];
            w[b] = st_w[sbase + b * M];
        }
        if (!active) { e = ww = n = s = x = cc = g = r = real(0); w[b] = real(0); }
        cE[b] = e; cW[b] = ww; cN[b] = n; cS[b] = s; cX[b] = x; cC[b] = cc;
        Gs[b] = g;
        Rr[b] = r;
    }

    burst_steps<M, CROSS, TSRC, real>(w, cE, cW, cN, cS, cC, cX, Gs, Rr, ds_s, K);

    if (MODE == MODE_BURST) {
        if (active) {
#pragma unroll
            for (int b = 0; b < M; ++b) st_w[sbase + b * M] = w[b];
        }
        return;
    }

    // trapezoid restriction of the departure, then eq. (Time_Derivative) and
    // eq. (Extrapolation) in FP64:  U_next = U + dt_macro (sum / n^2 + bias) / tau
    real col = real(0.5) * (w[0] + w[M - 1]);
#pragma unroll
    for (int b = 1; b < M - 1; ++b) col += w[b];
    if (a == 0 || a == M - 1) col *= real(0.5);
    if (!active) col = real(0);
#pragma unroll
    for (int off = 1; off < M; off <<= 1) {
        real o = __shfl_down_sync(FULL, col, off);
        if (a + off < M) col += o;
    }
    if (active && a == 0) {
        double inc = fma((double)col, upd_scale, bias * bias_scale);
        if (!isfinite(inc)) atomicOr(I.err, ERR_NONFINITE);
        if (MODE == MODE_DU) {
            dU_out[pidx] = inc;
        } else {
            long long node = (long long)j * I.nxp + i;
            Un[node] = u00 + inc;
        }
    }
}

// ---------------------------------------------------------------------------
// Generic kernels for the separate C-ABI passes (any m_xi, m_eta <= 32):
// one block per patch.

__device__ __forceinline__ void patch_ij(const InstDev& I, int p, int& i, int& j, int& ic, int& jr)
{
    ic = p % I.ncols; jr = p / I.ncols;
    i = I.i0 + ic; j = 1 + jr;
}

__device__ __forceinline__ long long rec_index(const InstDev& I, int jr, int ic, int a, int b)
{
    return ((long long)(jr * I.my + b) * I.ncols + ic) * I.mx + a;
}

// Ghost-neighbour terms of the burst forcing at micro point (a, b): weight *
// (ghost value - lift there), non-zero at edge points only.  The W/E/S/N ghosts
// are formed for every point without branches (zero weights inside the patch):
// the W/E ghost offset is -+2 dx gap_xi at the left/right edge s, the S/N one
// -+2 dy gap_eta at the bottom/top edge t; the diagonal ghosts of the cross
// term (beta != 0, edge points only) as ghost_offset.
template <typename real, typename Geo>
__device__ __forceinline__ real lift_ghost_terms(const Poly<real>& c, const Geo& g, int a, int b, real be,
                                                 const PointW<real>& w)
{
    const real sa = g.s(a), tb = g.t(b);
    const real se = a == 0 ? real(-0.5) * g.hx : real(0.5) * g.hx;
    const real te = b == 0 ? real(-0.5) * g.hy : real(0.5) * g.hy;
    const real wx = a == 0 ? -w.wW : (a == g.nx ? w.wE : real(0));
    const real wy = b == 0 ? -w.wS : (b == g.ny ? w.wN : real(0));
    real r = wx * (real(2) * g.dx * edge_gap_xi(c, se, tb)) + wy * (real(2) * g.dy * edge_gap_eta(c, sa, te));
    if (be != real(0) && (a == 0 || a == g.nx || b == 0 || b == g.ny)) {
        auto out = [&](int ap, int bp) { return ap < 0 || ap > g.nx || bp < 0 || bp > g.ny; };
        if (out(a + 1, b + 1)) r += w.wX * ghost_offset(c, g, a + 1, b + 1);
        if (out(a - 1, b - 1)) r += w.wX * ghost_offset(c, g, a - 1, b - 1);
        if (out(a + 1, b - 1)) r -= w.wX * ghost_offset(c, g, a + 1, b - 1);
        if (out(a - 1, b + 1)) r -= w.wX * ghost_offset(c, g, a - 1, b + 1);
    }
    return r;
}

// lift of several patches per block (ppb <= 32, so that every phase keeps the
// block's threads busy): interpolant coefficients
// (FP64, nine threads per patch), then per micro point the lifted value u0
// (FP64), the forcing r and w = 0, the edge data and the bias.  The quadratic
// lift is evaluated as u0(a, b) = A(a) + t_b B(a) + Q(b) with per-patch tables
// A = C0 + c10 s + c20 s^2, B = c01 + c11 s, Q = c02 t^2 (one FP64 fma and one
// add per point).
// FP32: five blocks per SM (48 registers, its 40 KB of shared memory each);
// more warps in flight pay more than the few values moved to local memory
// (measured: 1.57 against 1.64 ms at four blocks on the 512 x 2048 annulus).
template <typename real>
__global__ void __launch_bounds__(256, (sizeof(real) == 4 ? 5 : 2))
lift_kernel(const InstDev I, const double* __restrict__ U, const double* __restrict__ tab, double* u0,
            real* r_out, real* w_out, double* edge, double* bias_out, int edge_stride, int ppb)
{
    constexpr int PPB = 32;
    __shared__ double sl[PPB][9];            // stencil slots
    __shared__ double cs[PPB][9];
    __shared__ double tabA[PPB][32], tabB[PPB][32], tabQ[PPB][32];
    __shared__ double ecoef[PPB][4][3];      // edge data as a quadratic along each edge
    __shared__ __align__(16) real csr[PPB][12];   // coefficients in the working precision (padded)
    __shared__ double gs[34], gt[34];        // micro coordinates s_a, t_b for a, b = -1 .. m
    __shared__ real gsr[34], gtr[34];        // the same in the working precision
    __shared__ int4 pij_s[PPB];              // (i, j, ic, jr) of every patch of the block
    __shared__ long long recb_s[PPB];        // record index of point (0, 0) of every patch
    __shared__ long long ob_s[PPB];          // micro-state index of point (0, 0)
    __shared__ int ab_s[1024];               // (b << 16) | a of in-patch point tl
    __shared__ int se_s[4 * 34];             // (side << 8) | e of edge entry tl
    const int p0 = blockIdx.x * ppb;
    const int mm = I.mx * I.my;
    // instance constants in the working precision, converted once per block
    __shared__ RealConsts<real> kc_s;
    __shared__ PatchGeo<real> grc_s;
    __shared__ real sT_s;
    if (threadIdx.x == 0) {
        kc_s = real_consts<real>(I);
        grc_s = PatchGeo<real>{ (real)I.hx, (real)I.hy, (real)I.dx, (real)I.dy, I.mx - 1, I.my - 1 };
        sT_s = (real)tab[0];
    }
    PatchGeo<double> gd = { I.hx, I.hy, I.dx, I.dy, I.mx - 1, I.my - 1 };
    for (int t = threadIdx.x; t < 34; t += blockDim.x) {
        gs[t] = gd.s(t - 1);
        gt[t] = gd.t(t - 1);
    }
    for (int t = threadIdx.x; t < mm; t += blockDim.x) {
        const int b = t / I.mx;
        ab_s[t] = (b << 16) | (t - b * I.mx);
    }
    for (int t = threadIdx.x; t < 4 * edge_stride; t += blockDim.x) {
        const int side = t / edge_stride;
        se_s[t] = (side << 8) | (t - side * edge_stride);
    }
    for (int t = threadIdx.x; t < ppb; t += blockDim.x) {
        int i = 0, j = 0, ic = 0, jr = 0;
        if (p0 + t < I.n_patch) patch_ij(I, p0 + t, i, j, ic, jr);
        pij_s[t] = make_int4(i, j, ic, jr);
        recb_s[t] = (((long long)jr * I.my) * I.ncols + ic) * I.mx;
        ob_s[t] = I.pt_off + (long long)(p0 + t) * mm;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ppb * 9; t += blockDim.x) {
        const int q = t / 9, k = t - q * 9;
        double v = 0.0;
        if (p0 + q < I.n_patch) {
            const int4 pq = pij_s[q];
            v = stencil_slot<false>(I, U, pq.x, pq.y, k);
        }
        sl[q][k] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ppb * 9; t += blockDim.x) {
        const int q = t / 9, k = t - q * 9;
        const double* x = sl[q];
        const double c = fma(I.c2w[k][1], x[I.c2slot[k][2]], fma(I.c2w[k][0], x[I.c2slot[k][1]], x[I.c2slot[k][0]])) * I.c2w[k][2];
        cs[q][k] = c;
        csr[q][k] = (real)c;
    }
    __syncthreads();
    // per-patch tables, every phase dense over (patch, entry) so that the FP64
    // pipe (a small fraction of the FP32 rate on this part) runs full warps
    for (int t = threadIdx.x; t < ppb * I.mx; t += blockDim.x) {
        const int q = t / I.mx, k = t - q * I.mx;
        const double* c = cs[q];
        const double sa = gs[k + 1];
        tabA[q][k] = c[0] + sa * (c[1] + sa * c[3]);
        tabB[q][k] = c[2] + c[4] * sa;
    }
    for (int t = threadIdx.x; t < ppb * I.my; t += blockDim.x) {
        const int q = t / I.my, k = t - q * I.my;
        const double tb = gt[k + 1];
        tabQ[q][k] = cs[q][5] * tb * tb;
    }
    for (int t = threadIdx.x; t < ppb * 4; t += blockDim.x) {
        const int q = t >> 2, k = t & 3;
        const double* c = cs[q];
        // d/dxi of P on xi = -+hx/2 as a quadratic in t; d/deta on eta = -+hy/2 in s
        if (k < 2) {
            const double s0 = (k == 0 ? -0.5 : 0.5) * I.hx;
            ecoef[q][k][0] = c[1] + 2.0 * c[3] * s0;
            ecoef[q][k][1] = c[4] + 2.0 * c[6] * s0;
            ecoef[q][k][2] = c[7] + 2.0 * c[8] * s0;
        } else {
            const double t0 = (k == 2 ? -0.5 : 0.5) * I.hy;
            ecoef[q][k][0] = c[2] + 2.0 * c[5] * t0;
            ecoef[q][k][1] = c[4] + 2.0 * c[7] * t0;
            ecoef[q][k][2] = c[6] + 2.0 * c[8] * t0;
        }
    }
    for (int t = threadIdx.x; t < 34; t += blockDim.x) {
        gsr[t] = grc_s.s(t - 1);
        gtr[t] = grc_s.t(t - 1);
    }
    __syncthreads();
    const RealConsts<real> kc = kc_s;
    const PatchGeoTab<real> gr = { grc_s.hx, grc_s.hy, grc_s.dx, grc_s.dy, I.mx - 1, I.my - 1, gsr, gtr };
    const real* rec = static_cast<const real*>(I.rec);
    const real sT = sT_s;
    // points t = threadIdx.x + k blockDim.x of the block's ppb * mm, patch q and
    // in-patch index tl advanced without division; (a, b) from the table
    int q = 0, tl = threadIdx.x;
    while (tl >= mm) { tl -= mm; ++q; }
    const int rowstride = I.ncols * I.mx;
    for (; q < ppb; ) {
        const int p = p0 + q;
        if (p < I.n_patch) {
            const real* cq = csr[q];
            real c0, c1, c2, c3, c4, c5, c6, c7, c8, c9, c10, c11;
            load_vec4_shared(cq, c0, c1, c2, c3);
            load_vec4_shared(cq + 4, c4, c5, c6, c7);
            load_vec4_shared(cq + 8, c8, c9, c10, c11);
            (void)c9; (void)c10; (void)c11;
            Poly<real> cr = { c0, c1, c2, c3, c4, c5, c6, c7, c8 };
            const int ab = ab_s[tl];
            const int b = ab >> 16, a = ab & 0xffff;
            real v[8];
            if (I.coef_mode != COEF_RECORDS) {
                const int4 pq = pij_s[q];
                table_coeffs_k<real>(I, kc, pq.z, a, pq.w, b, v);
                v[6] = real(0);
            } else {
                const real* rr = rec + (recb_s[q] + b * rowstride + a) * 8;
                load_vec4<real>(rr, v[0], v[1], v[2], v[3]);
                load_vec4<real>(rr + 4, v[4], v[5], v[6], v[7]);
            }
            const long long o = ob_s[q] + tl;
            u0[o] = fma(gt[b + 1], tabB[q][a], tabA[q][a] + tabQ[q][b]);
            PointW<real> pw = point_weights_k<real>(I, kc, v[0], v[1], v[2], v[3], v[4], v[5]);
            r_out[o] = burst_forcing_base<real>(cr, gr, a, b, v[0], v[1], v[2], v[3], v[4], v[5], v[6], sT, pw) +
                       lift_ghost_terms<real>(cr, gr, a, b, v[1], pw);
            w_out[o] = real(0);
        }
        tl += blockDim.x;
        while (tl >= mm) { tl -= mm; ++q; }
    }
    // edge data of eq. (edge) = d/dxi, d/deta of the interpolant P at the edges
    // (dense over (patch, side, entry))
    {
        const int ne = 4 * edge_stride;
        int qq = 0, tle = threadIdx.x;
        while (tle >= ne) { tle -= ne; ++qq; }
        for (; qq < ppb; ) {
            const int p = p0 + qq;
            if (p < I.n_patch) {
                const int se = se_s[tle];
                const int side = se >> 8, e = se & 0xff;
                const double* ec = ecoef[qq][side];
                double val = 0.0;
                if ((side < 2 && e < I.my + 2) || (side >= 2 && e < I.mx + 2)) {
                    const double x = side < 2 ? gt[e] : gs[e];
                    val = fma(fma(ec[2], x, ec[1]), x, ec[0]);
                }
                edge[I.e_off + ((long long)p * 4 + side) * edge_stride + e] = val;
            }
            tle += blockDim.x;
            while (tle >= ne) { tle -= ne; ++qq; }
        }
    }
    for (int q = threadIdx.x; q < ppb; q += blockDim.x) {
        const int p = p0 + q;
        if (p >= I.n_patch) continue;
        const double* c = cs[q];
        bias_out[(long long)I.p_off + p] = (I.restrict_mode == PD_RESTRICT_MACRO) ? (I.dx * I.dx * c[3] + I.dy * I.dy * c[5]) / 6.0 : 0.0;
    }
}

// generic burst: whole patch in shared memory, one thread per micro point
template <typename real>
__global__ void __launch_bounds__(256)
burst_kernel(const InstDev I, const double* __restrict__ tab, int k_steps, real* w_io, const real* __restrict__ r_in)
{
    extern __shared__ unsigned char smem_raw[];
    real* ws = reinterpret_cast<real*>(smem_raw);
    real* ds = ws + 2 * I.mx * I.my;
    const int p = blockIdx.x;
    int i, j, ic, jr;
    patch_ij(I, p, i, j, ic, jr);
    const int mm = I.mx * I.my;
    const long long pp0 = I.pt_off + (long long)p * mm;
    const real* rec = static_cast<const real*>(I.rec);
    const real dt = (real)I.dt;
    for (int t = threadIdx.x; t < k_steps; t += blockDim.x) ds[t] = (real)tab[t];
    // this thread's point (mm <= 1024 not needed: loop)
    for (int t = threadIdx.x; t < mm; t += blockDim.x) ws[t] = w_io[pp0 + t];
    __syncthreads();
    real* cur = ws;
    real* nxt = ws + mm;
    for (int k = 0; k < k_steps; ++k) {
        for (int t = threadIdx.x; t < mm; t += blockDim.x) {
            int a = t % I.mx, b = t / I.mx;
            real v[8];
            point_coeffs<real>(I, jr, ic, a, b, v);
            PointW<real> pw = point_weights<real>(v[0], v[1], v[2], v[3], v[4], v[5], (real)I.dx, (real)I.dy, I.conv);
            // homogeneous mirrors for the departure
            int aE = a + 1 > I.mx - 1 ? I.mx - 2 : a + 1;
            int aW = a - 1 < 0 ? 1 : a - 1;
            int bN = b + 1 > I.my - 1 ? I.my - 2 : b + 1;
            int bS = b - 1 < 0 ? 1 : b - 1;
            real L = pw.wC * cur[t] + pw.wE * cur[b * I.mx + aE] + pw.wW * cur[b * I.mx + aW]
                   + pw.wN * cur[bN * I.mx + a] + pw.wS * cur[bS * I.mx + a]
                   + pw.wX * (cur[bN * I.mx + aE] - cur[bS * I.mx + aE] - cur[bN * I.mx + aW] + cur[bS * I.mx + aW]);
            nxt[t] = cur[t] + dt * (L + r_in[pp0 + t] + ds[k] * v[6]);
        }
        __syncthreads();
        real* tmp = cur; cur = nxt; nxt = tmp;
    }
    for (int t = threadIdx.x; t < mm; t += blockDim.x) w_io[pp0 + t] = cur[t];
}

// trapezoid restriction of the departure: ppb (<= 64) patches per block, their
// contiguous w staged into shared memory with 16-byte cp.async copies (plain
// loads where the block's start is not 16-byte aligned), four threads per patch
// summing against a table of the trapezoid weights (accumulation in the grid's
// precision, like the fused kernels' column sums), dU in FP64
constexpr int kRestrictPatches = 64;
constexpr size_t kRestrictStage = 96 * 1024;

template <typename real>
__global__ void __launch_bounds__(256)
restrict_kernel(const InstDev I, const real* __restrict__ w, const double* __restrict__ bias, double* __restrict__ dU,
                int ppb)
{
    extern __shared__ __align__(16) unsigned char rsm[];
    const int mm = I.mx * I.my;
    real* tile = reinterpret_cast<real*>(rsm);                // [ppb * mm]
    real* tw = tile + (size_t)ppb * mm;                       // [mm] weights
    for (int t = threadIdx.x; t < mm; t += blockDim.x) {
        const int b = t / I.mx, a = t - b * I.mx;
        const real wa = (a == 0 || a == I.mx - 1) ? real(0.5) : real(1);
        tw[t] = (b == 0 || b == I.my - 1) ? real(0.5) * wa : wa;
    }
    const int p0 = blockIdx.x * ppb;
    const int np = min(ppb, I.n_patch - p0);
    // the bias of this thread's patch, requested before the staging loads
    const int q = threadIdx.x >> 2, sub = threadIdx.x & 3;
    const long long pg = (long long)I.p_off + p0 + q;
    const double bq = (q < np && sub == 0) ? __ldg(bias + pg) : 0.0;
    const real* src = w + I.pt_off + (long long)p0 * mm;
    const int n = np * mm;
    constexpr int V = 16 / sizeof(real);
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (reinterpret_cast<uintptr_t>(tile) & 15) == 0) {
        // every 16-byte piece of the block's patches requested at once, straight
        // into shared memory (no registers held while the loads are in flight)
        const int nv = n / V;
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* t4 = reinterpret_cast<uint4*>(tile);
        for (int e = threadIdx.x; e < nv; e += blockDim.x) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(t4 + e);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(s4 + e) : "memory");
        }
        for (int e = nv * V + threadIdx.x; e < n; e += blockDim.x) tile[e] = src[e];
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else {
#pragma unroll 4
        for (int e = threadIdx.x; e < n; e += blockDim.x) tile[e] = src[e];
    }
    __syncthreads();
    real acc = real(0);
    if (q < np) {
        const real* x = tile + q * mm;
        for (int t = sub; t < mm; t += 4) acc = fma(tw[t], x[t], acc);
    }
    acc += __shfl_xor_sync(FULL, acc, 1);
    acc += __shfl_xor_sync(FULL, acc, 2);
    if (q < np && sub == 0) {
        double v = fma((double)acc, I.inv_nn, bq);
        if (!isfinite(v)) atomicOr(I.err, ERR_NONFINITE);
        dU[pg] = v;
    }
}

// Dirichlet data at one boundary node, out of line: inlined, the FP64 solution
// code tripled the instructions every warp of the projection issued, interior
// warps included (measured)
__device__ __noinline__ void project_boundary_node(const InstDev& I, double* __restrict__ U, int q, double t_next)
{
    const int2 ij = I.bnd_ij[q];
    const double2 xy = I.bnd_xy[q];
    U[(long long)ij.y * I.nxp + ij.x] = exact_solution(I.sol, xy.x, xy.y, t_next);
}

// eq. (Extrapolation) on interior nodes + Dirichlet data at t + dt_macro
// (scale = dt_macro / tau, formed on the host: no FP64 division per node).
// Grid rows y (strided by gridDim.y): y < nrows is patch row jr = y, blockIdx.x a
// chunk of kProjectPer * blockDim.x of its columns; the rows after those hold
// chunks of the boundary nodes.  Each thread issues the loads of all its nodes
// before the first update, so it keeps kProjectPer loads of U and dU in flight.
constexpr int kProjectPer = 4;
constexpr int kProjectBlock = 128;

__global__ void __launch_bounds__(kProjectBlock)
project_kernel(const InstDev I, double* __restrict__ U, const double* __restrict__ dU, double t_next, double scale,
               int n_rows_total)
{
    for (int jr = blockIdx.y; jr < n_rows_total; jr += gridDim.y) {
        if (jr < I.nrows) {
            const int c0 = blockIdx.x * (kProjectPer * kProjectBlock) + threadIdx.x;
            double* row = U + (long long)(1 + jr) * I.nxp + I.i0;
            const double* drow = dU + (long long)I.p_off + (long long)jr * I.ncols;
            double u[kProjectPer], d[kProjectPer];
#pragma unroll
            for (int k = 0; k < kProjectPer; ++k) {
                const int ic = c0 + k * kProjectBlock;
                if (ic < I.ncols) { u[k] = row[ic]; d[k] = __ldg(drow + ic); }
            }
#pragma unroll
            for (int k = 0; k < kProjectPer; ++k) {
                const int ic = c0 + k * kProjectBlock;
                if (ic < I.ncols) row[ic] = fma(scale, d[k], u[k]);
            }
        } else {
            const int q = ((jr - I.nrows) * gridDim.x + blockIdx.x) * kProjectBlock + threadIdx.x;
            if (q < I.n_bnd) project_boundary_node(I, U, q, t_next);
        }
    }
}

// ds table for a standalone burst: ds_k = s(t + k dt) - s(t_lift)
__global__ void burst_table_kernel(int K, int tkind, double tc, double dt, double t, const double* t_lift,
                                   double* tab)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) tab[k] = time_factor(tkind, tc, t + k * dt) - time_factor(tkind, tc, *t_lift);
}

__global__ void lift_table_kernel(int tkind, double tc, double t, double* tab, double* t_lift)
{
    tab[0] = time_factor(tkind, tc, t);
    *t_lift = t;
}

// ---------------------------------------------------------------------------
// dispatch of the templated warp kernel

template <int M, typename real, int MODE>
cudaError_t launch_warp(const InstDev& I, const double* Uc, double* Un, const double* tab, double dtm,
                        int k_steps, real* st_w, const real* st_r, cudaStream_t st,
                        double* dU_out = nullptr, const int* list = nullptr, const int* list_n = nullptr)
{
    // dt_macro / tau scales the restricted change; the trapezoid sum also carries 1 / n^2
    // (MODE_DU writes the restricted change itself)
    double bias_scale = (MODE == MODE_DU) ? 1.0 : dtm * I.inv_tau;
    double upd_scale = (MODE == MODE_DU) ? I.inv_nn : bias_scale * I.inv_nn;
    constexpr int P = 32 / M;
    int wpr = (I.ncols + P - 1) / P;
    int n_item_warps = wpr * I.nrows;
    int n_bnd_warps = (MODE == MODE_FUSED) ? (I.n_bnd + 31) / 32 : 0;
    int n_warps = n_item_warps + n_bnd_warps;
    const int bs = 128;
    unsigned nb = (unsigned)((n_warps * 32 + bs - 1) / bs);
    bool cross = I.has_cross != 0, tsrc = I.has_tsrc != 0;
    int K = (MODE == MODE_FUSED) ? I.K : k_steps;
    size_t smem = tsrc ? sizeof(real) * (size_t)K : 0;
#define PD_LAUNCH(CR, TS) patch_warp_kernel<M, CR, TS, real, MODE><<<nb, bs, smem, st>>>(I, Uc, Un, tab, upd_scale, bias_scale, k_steps, st_w, st_r, n_item_warps, dU_out, list, list_n)
    if (cross && tsrc) PD_LAUNCH(true, true);
    else if (cross) PD_LAUNCH(true, false);
    else if (tsrc) PD_LAUNCH(false, true);
    else PD_LAUNCH(false, false);
#undef PD_LAUNCH
    return cudaGetLastError();
}

template <typename real, int MODE>
cudaError_t dispatch_m(const InstDev& I, const double* Uc, double* Un, const double* tab, double dtm,
                       int k_steps, real* st_w, const real* st_r, cudaStream_t st,
                       double* dU_out = nullptr, const int* list = nullptr, const int* list_n = nullptr)
{
    switch (I.mx) {
    case 3: return launch_warp<3, real, MODE>(I, Uc, Un, tab, dtm, k_steps, st_w, st_r, st, dU_out, list, list_n);
    case 5: return launch_warp<5, real, MODE>(I, Uc, Un, tab, dtm, k_steps, st_w, st_r, st, dU_out, list, list_n);
    case 7: return launch_warp<7, real, MODE>(I, Uc, Un, tab, dtm, k_steps, st_w, st_r, st, dU_out, list, list_n);
    case 9: return launch_warp<9, real, MODE>(I, Uc, Un, tab, dtm, k_steps, st_w, st_r, st, dU_out, list, list_n);
    case 11: return launch_warp<11, real, MODE>(I, Uc, Un, tab, dtm, k_steps, st_w, st_r, st, dU_out, list, list_n);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_burst_records(const InstDev& I, int prec, void* brec, cudaStream_t st)
{
    long long n = (long long)I.n_patch * I.mx * I.my;
    unsigned nb = (unsigned)((n + 127) / 128);
    if (prec == PD_FP32)
        burst_record_kernel<float><<<nb, 128, 0, st>>>(I, (const float*)I.rec, (float*)brec);
    else
        burst_record_kernel<double><<<nb, 128, 0, st>>>(I, (const double*)I.rec, (double*)brec);
    return cudaGetLastError();
}

bool batch_supported(const InstDev& I)
{
    return I.mx == I.my && (I.mx == 3 || I.mx == 5 || I.mx == 7 || I.mx == 9 || I.mx == 11) && I.K <= kMaxK;
}

bool fused_supported(const InstDev& I)
{
    return I.mx == I.my && (I.mx == 3 || I.mx == 5 || I.mx == 7 || I.mx == 9 || I.mx == 11) && I.K <= kMaxK;
}

cudaError_t launch_patch_dU(const InstDev& I, int prec, const double* U, const double* tab_row, int k_steps,
                            double* dU, const int* list, const int* list_n, cudaStream_t st)
{
    if (I.micro == PD_MICRO_ADI) {
        if (k_steps != I.K) return cudaErrorInvalidValue;   // ADI bursts always run the instance's K steps
        return launch_adi_dU(I, prec, U, tab_row, dU, list, list_n, st);
    }
    if (prec == PD_FP32)
        return dispatch_m<float, MODE_DU>(I, U, nullptr, tab_row, 0.0, k_steps, nullptr, nullptr, st, dU, list, list_n);
    return dispatch_m<double, MODE_DU>(I, U, nullptr, tab_row, 0.0, k_steps, nullptr, nullptr, st, dU, list, list_n);
}

// Per patch, the trapezoid-weighted sums over its micro points of the burst
// record's forcing basis B_0..B_8 and of dt G, times 1/(n^2 dt): after one
// micro step from w = 0 the departure is the forcing, so the restricted
// change over dt is F1 = sum_k c_k S_k + s(T) S_9 exactly.  The interpolant
// coefficients are c_k = sum_q lw[k][q] U_q over the 3x3 stencil, so the
// stored basis is T_q = sum_k S_k lw[k][q] (q = 0..8) and T_9 = S_9:
// F1 = sum_q T_q U_q + s(T) T_9.
template <typename real>
__global__ void one_step_basis_kernel(const InstDev I, const real* __restrict__ brec, double* __restrict__ T)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= I.n_patch) return;
    const int jr = p / I.ncols, ic = p - jr * I.ncols;
    const int M = I.mx;
    double acc[10] = { 0, 0, 0, 0, 0, 0, 0, 0, 0, 0 };
    for (int b = 0; b < M; ++b) {
        const double wb = (b == 0 || b == M - 1) ? 0.5 : 1.0;
        for (int a = 0; a < M; ++a) {
            const double w = wb * ((a == 0 || a == M - 1) ? 0.5 : 1.0);
            const real* r = brec + (((long long)(jr * M + b) * I.ncols + ic) * M + a) * 16;
            for (int k = 0; k < 9; ++k) acc[k] += w * (double)r[7 + k];
            acc[9] += w * (double)r[6];
        }
    }
    const double f = I.inv_nn / I.dt;
    for (int q = 0; q < 9; ++q) {
        double t = 0.0;
        for (int k = 0; k < 9; ++k) t = fma(acc[k], I.lw[k][q], t);
        T[(long long)p * 10 + q] = t * f;
    }
    T[(long long)p * 10 + 9] = acc[9] * f;
}

cudaError_t launch_one_step_basis(const InstDev& I, int prec, double* T, cudaStream_t st)
{
    const unsigned nb = (unsigned)((I.n_patch + 127) / 128);
    if (prec == PD_FP32) one_step_basis_kernel<float><<<nb, 128, 0, st>>>(I, static_cast<const float*>(I.brec), T);
    else one_step_basis_kernel<double><<<nb, 128, 0, st>>>(I, static_cast<const double*>(I.brec), T);
    return cudaGetLastError();
}

cudaError_t launch_fused_step(const InstDev& I, const InstDev*, int prec, const double* Uc, double* Un,
                              const double* tab_row, double dtm, cudaStream_t st, int* n_launch)
{
    if (n_launch) ++*n_launch;
    if (I.micro == PD_MICRO_ADI) return launch_adi_fused(I, prec, Uc, Un, tab_row, dtm, st);
    if (prec == PD_FP32)
        return dispatch_m<float, MODE_FUSED>(I, Uc, Un, tab_row, dtm, 0, nullptr, nullptr, st);
    return dispatch_m<double, MODE_FUSED>(I, Uc, Un, tab_row, dtm, 0, nullptr, nullptr, st);
}

cudaError_t launch_lift(const InstDev& I, const InstDev*, int prec, const double* U, double t, char* state,
                        const pd_info& lay, cudaStream_t st)
{
    // header of the state buffer: [0] lift time, [1] scratch s(t)
    double* hdr = reinterpret_cast<double*>(state);
    lift_table_kernel<<<1, 1, 0, st>>>(I.tkind, I.tc, t, hdr + 1, hdr);
    double* u0 = reinterpret_cast<double*>(state + lay.off_u0);
    double* edge = reinterpret_cast<double*>(state + lay.off_edge);
    double* bias = reinterpret_cast<double*>(state + lay.off_bias);
    const int ppb = std::max(1, std::min(32, 2592 / (I.mx * I.my)));
    const unsigned nb = (unsigned)((I.n_patch + ppb - 1) / ppb);
    if (prec == PD_FP32)
        lift_kernel<float><<<nb, 256, 0, st>>>(I, U, hdr + 1, u0, reinterpret_cast<float*>(state + lay.off_r),
                                               reinterpret_cast<float*>(state + lay.off_w), edge, bias, lay.edge_stride, ppb);
    else
        lift_kernel<double><<<nb, 256, 0, st>>>(I, U, hdr + 1, u0, reinterpret_cast<double*>(state + lay.off_r),
                                                reinterpret_cast<double*>(state + lay.off_w), edge, bias, lay.edge_stride, ppb);
    return cudaGetLastError();
}

cudaError_t launch_burst(const InstDev& I, const InstDev*, int prec, char* state, const pd_info& lay, double t,
                         int k_steps, cudaStream_t st)
{
    double* hdr = reinterpret_cast<double*>(state);
    double* tab = hdr + 2;  // up to kMaxK entries live in the header block
    burst_table_kernel<<<(k_steps + 127) / 128, 128, 0, st>>>(k_steps, I.tkind, I.tc, I.dt, t, hdr, tab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (fused_supported(I) && I.coef_mode == COEF_RECORDS) {
        if (prec == PD_FP32)
            return dispatch_m<float, MODE_BURST>(I, nullptr, nullptr, tab, 0.0, k_steps,
                                                 reinterpret_cast<float*>(state + lay.off_w),
                                                 reinterpret_cast<const float*>(state + lay.off_r), st);
        return dispatch_m<double, MODE_BURST>(I, nullptr, nullptr, tab, 0.0, k_steps,
                                              reinterpret_cast<double*>(state + lay.off_w),
                                              reinterpret_cast<const double*>(state + lay.off_r), st);
    }
    size_t es = prec == PD_FP32 ? sizeof(float) : sizeof(double);
    size_t smem = (2 * (size_t)I.mx * I.my + k_steps) * es;
    if (smem > 48 * 1024) {
        cudaError_t a = prec == PD_FP32
            ? cudaFuncSetAttribute(burst_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(burst_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (a != cudaSuccess) return a;
    }
    if (prec == PD_FP32)
        burst_kernel<float><<<I.n_patch, 256, smem, st>>>(I, tab, k_steps, reinterpret_cast<float*>(state + lay.off_w),
                                                           reinterpret_cast<const float*>(state + lay.off_r));
    else
        burst_kernel<double><<<I.n_patch, 256, smem, st>>>(I, tab, k_steps, reinterpret_cast<double*>(state + lay.off_w),
                                                            reinterpret_cast<const double*>(state + lay.off_r));
    return cudaGetLastError();
}

cudaError_t launch_restrict(const InstDev& I, int prec, const char* state, const pd_info& lay, double* dU,
                            cudaStream_t st, const double* bias_override)
{
    const double* bias = bias_override ? bias_override : reinterpret_cast<const double*>(state + lay.off_bias);
    const size_t es = prec == PD_FP32 ? sizeof(float) : sizeof(double);
    const size_t per = es * (size_t)I.mx * I.my;
    const int ppb = (int)std::max<size_t>(1, std::min<size_t>(kRestrictPatches, kRestrictStage / per - 1));
    const unsigned nb = (unsigned)((I.n_patch + ppb - 1) / ppb);
    const size_t smem = per * (size_t)(ppb + 1);
    cudaError_t e;
    if (prec == PD_FP32) {
        e = cudaFuncSetAttribute(restrict_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            restrict_kernel<float><<<nb, 256, smem, st>>>(I, reinterpret_cast<const float*>(state + lay.off_w), bias, dU, ppb);
    } else {
        e = cudaFuncSetAttribute(restrict_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            restrict_kernel<double><<<nb, 256, smem, st>>>(I, reinterpret_cast<const double*>(state + lay.off_w), bias, dU, ppb);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Heun's combination: U_{n+1} = (U_n + S2)/2 on the interior nodes, with
// S1 = U_n + dt F(U_n, T_n) (boundary data at T_{n+1}) and S2 = S1 + dt F(S1, T_{n+1});
// the boundary nodes take S1's data at T_{n+1}.
__global__ void heun_combine_kernel(const InstDev I, double* __restrict__ U, const double* __restrict__ S1,
                                    const double* __restrict__ S2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < I.n_patch) {
        int i, j, ic, jr;
        patch_ij(I, k, i, j, ic, jr);
        const long long node = (long long)j * I.nxp + i;
        U[node] = 0.5 * (U[node] + S2[node]);
    } else if (k < I.n_patch + I.n_bnd) {
        const int2 ij = I.bnd_ij[k - I.n_patch];
        const long long node = (long long)ij.y * I.nxp + ij.x;
        U[node] = S1[node];
    }
}

// Adams-Bashforth-2: U += dt (3/2 dU_n - 1/2 dU_{n-1}) / tau on the interior,
// Dirichlet data at t + dt on the boundary.
__global__ void ab2_kernel(const InstDev I, double* __restrict__ U, const double* __restrict__ dUn,
                           const double* __restrict__ dUp, double t_next, double dtm)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < I.n_patch) {
        int i, j, ic, jr;
        patch_ij(I, k, i, j, ic, jr);
        const long long node = (long long)j * I.nxp + i;
        const double d = 1.5 * dUn[(long long)I.p_off + k] - 0.5 * dUp[(long long)I.p_off + k];
        if (!isfinite(d)) atomicOr(I.err, ERR_NONFINITE);
        U[node] = U[node] + dtm * (d / I.tau);
    } else if (k < I.n_patch + I.n_bnd) {
        const int q = k - I.n_patch;
        const int2 ij = I.bnd_ij[q];
        const double2 xy = I.bnd_xy[q];
        U[(long long)ij.y * I.nxp + ij.x] = exact_solution(I.sol, xy.x, xy.y, t_next);
    }
}

cudaError_t launch_heun_combine(const InstDev& I, double* U, const double* S1, const double* S2, cudaStream_t st)
{
    const int n = I.n_patch + I.n_bnd;
    heun_combine_kernel<<<(n + 127) / 128, 128, 0, st>>>(I, U, S1, S2);
    return cudaGetLastError();
}

cudaError_t launch_ab2(const InstDev& I, double* U, const double* dUn, const double* dUp, double t, double dtm,
                       cudaStream_t st)
{
    const int n = I.n_patch + I.n_bnd;
    ab2_kernel<<<(n + 127) / 128, 128, 0, st>>>(I, U, dUn, dUp, t + dtm, dtm);
    return cudaGetLastError();
}

cudaError_t launch_project(const InstDev& I, double* U, const double* dU, double t, double dtm, cudaStream_t st)
{
    const unsigned gx = (unsigned)((I.ncols + kProjectPer * kProjectBlock - 1) / (kProjectPer * kProjectBlock));
    const unsigned bnd_rows = (unsigned)(((long long)I.n_bnd + (long long)gx * kProjectBlock - 1) / ((long long)gx * kProjectBlock));
    const int rows = I.nrows + (int)bnd_rows;
    if (rows == 0) return cudaSuccess;
    project_kernel<<<dim3(gx, (unsigned)std::min(rows, 65535)), kProjectBlock, 0, st>>>(I, U, dU, t + dtm,
                                                                                      dtm * I.inv_tau, rows);
    return cudaGetLastError();
}

}  // namespace pd

// Batched macro step over many independent instances of uneven sizes.
//
// One launch per macro step covers every instance of the grid.  The work is a
// list of items (a patch group = up to 32 / m patches of one patch row of one
// instance, or a chunk of 32 boundary nodes), sorted by cost on the host; the
// warps of a persistent-size grid pull items from a device counter (one atomic
// per item), so instances of different micro sizes and macro grids balance
// across the GPU.  A patch group runs the whole macro step in registers: lift,
// K forward-Euler micro steps, trapezoid restriction, projective update.  The
// transformed coefficients come from the instance's 1-D metric tables (constant
// K, v, f on separable or polar maps) or from its per-point records, and the
// stencil weights and closed-form forcing are formed on the fly.
#include "pd_device.cuh"

#include <math.h>

namespace pd {

namespace {

template <int M, bool TSRC, typename real>
__device__ __forceinline__ void patch_item(const InstDev& I, const BatchItem& it, const BatchArgs& A, int lane)
{
    const int P = I.ppw;                      // patches per warp chosen for this instance
    const int jr = it.jr;
    const int ic0 = it.wc * P;
    const int q = lane / M;
    const int a = lane - q * M;
    const int ic = ic0 + q;
    const bool active = (q < P) && (ic < I.ncols);
    const int icl = active ? ic : (I.ncols - 1);
    const int i = I.i0 + icl, j = 1 + jr;
    const int qbase = (q < P ? q : P - 1) * M;

    const double* Uc = (A.parity ? A.Sbase : A.Ubase) + I.u_off;
    double* Un = (A.parity ? A.Ubase : A.Sbase) + I.u_off;

    real cv[9];
    double c20, c02, u00;
    macro_coeffs<M, real, false>(I, Uc, i, j, a, qbase, I.lw, I.c2slot, I.c2w, cv, c20, c02, u00);
    double bias = 0.0;
    if (I.restrict_mode == PD_RESTRICT_MACRO) bias = (I.dx * I.dx * c20 + I.dy * I.dy * c02) * (1.0 / 6.0);
    Poly<real> c = { cv[0], cv[1], cv[2], cv[3], cv[4], cv[5], cv[6], cv[7], cv[8] };

    const double* trow = (A.tab && (TSRC || I.sol != PD_SOL_NONE)) ? A.tab + A.tab_off[it.inst] + (long long)A.step * (I.K + kTabExtra) : nullptr;
    const real sT = (TSRC && trow) ? (real)trow[I.K] : real(0);

    const RealConsts<real> kc = real_consts<real>(I);
    PatchGeo<real> g;
    if constexpr (sizeof(real) == 4) { g.hx = I.kf[13]; g.hy = I.kf[14]; }
    else { g.hx = I.hx; g.hy = I.hy; }
    g.dx = kc.dx; g.dy = kc.dy;
    g.nx = M - 1; g.ny = M - 1;
    const real dt = sizeof(real) == 4 ? (real)I.kf[15] : (real)I.dt;
    const real* rec = static_cast<const real*>(I.rec);
    const long long rowstride = (long long)I.ncols * M;
    const long long base = (long long)jr * M * rowstride + (long long)icl * M + a;

    real w[M], Rr[M], cE[M], cW[M], cN[M], cS[M], cC[M], cX[M], Gs[M];
#pragma unroll
    for (int b = 0; b < M; ++b) {
        real co[6], G = real(0);
        if (I.coef_mode != COEF_RECORDS) {
            table_coeffs_k<real>(I, kc, icl, a, jr, b, co);
        } else {
            const real* pr = rec + (base + b * rowstride) * 8;
            for (int k = 0; k < 6; ++k) co[k] = pr[k];
            G = pr[6];
        }
        PointW<real> pw = point_weights_k<real>(I, kc, co[0], co[1], co[2], co[3], co[4], co[5]);
        real r = burst_forcing<real>(c, g, a, b, co[0], co[1], co[2], co[3], co[4], co[5], G, sT, pw);
        real e = dt * pw.wE, ww = dt * pw.wW, n = dt * pw.wN, s = dt * pw.wS, x = dt * pw.wX;
        real cc = real(1) + dt * pw.wC;
        if (a == 0) { e += ww; ww = real(0); }
        if (a == M - 1) { ww += e; e = real(0); }
        if (b == 0) { n += s; s = real(0); }
        if (b == M - 1) { s += n; n = real(0); }
        if (a == 0 || a == M - 1 || b == 0 || b == M - 1) x = real(0);
        if (!active) { e = ww = n = s = x = cc = r = G = real(0); }
        cE[b] = e; cW[b] = ww; cN[b] = n; cS[b] = s; cX[b] = x; cC[b] = cc;
        Rr[b] = dt * r;
        Gs[b] = dt * G;
        w[b] = real(0);
    }

    // time-dependent source: ds_k read straight from the instance's time table (L1)
    if (TSRC && trow) burst_steps<M, true, true, real>(w, cE, cW, cN, cS, cC, cX, Gs, Rr, trow, I.K);
    else burst_steps<M, true, false, real>(w, cE, cW, cN, cS, cC, cX, Gs, Rr, trow, I.K);

    real col = real(0.5) * (w[0] + w[M - 1]);
#pragma unroll
    for (int b = 1; b < M - 1; ++b) col += w[b];
    if (a == 0 || a == M - 1) col *= real(0.5);
    if (!active) col = real(0);
#pragma unroll
    for (int off = 1; off < M; off <<= 1) {
        real o = __shfl_down_sync(kFull, col, off);
        if (a + off < M) col += o;
    }
    if (active && a == 0) {
        double bias_scale = A.dtm[it.inst] * I.inv_tau;
        double inc = fma((double)col, bias_scale * I.inv_nn, bias * bias_scale);
        if (!isfinite(inc)) atomicOr(I.err, ERR_NONFINITE);
        Un[(long long)j * I.nxp + i] = u00 + inc;
    }
}

__device__ __forceinline__ void boundary_item(const InstDev& I, const BatchItem& it, const BatchArgs& A, int lane)
{
    double* Un = (A.parity ? A.Ubase : A.Sbase) + I.u_off;
    int k = it.jr * 32 + lane;
    if (k >= I.n_bnd) return;
    int2 ij = I.bnd_ij[k];
    double v = 0.0;
    if (I.sol != PD_SOL_NONE && A.tab) {
        const double* trow = A.tab + A.tab_off[it.inst] + (long long)A.step * (I.K + kTabExtra);
        double2 xy = I.bnd_xy[k];
        v = exact_solution(I.sol, xy.x, xy.y, trow[I.K + 2]);
    }
    Un[(long long)ij.y * I.nxp + ij.x] = v;
}

// at most 128 threads per block and 170 registers per thread: three blocks per SM
template <bool TSRC, typename real>
__global__ void __launch_bounds__(128, 3) batch_kernel(const BatchArgs A)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(A.counter, 1);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= A.n_items) break;
        const BatchItem it = A.items[idx];
        const InstDev& I = A.insts[it.inst];
        if (it.kind == 1) { boundary_item(I, it, A, lane); continue; }
        switch (I.mx) {
        case 3: patch_item<3, TSRC, real>(I, it, A, lane); break;
        case 5: patch_item<5, TSRC, real>(I, it, A, lane); break;
        case 7: patch_item<7, TSRC, real>(I, it, A, lane); break;
        case 9: patch_item<9, TSRC, real>(I, it, A, lane); break;
        case 11: patch_item<11, TSRC, real>(I, it, A, lane); break;
        default: break;
        }
    }
}

template <bool TSRC, typename real>
int occupancy(int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<TSRC, real>, block, 0) != cudaSuccess) return 0;
    return nb;
}

}  // namespace

cudaError_t launch_batch(int prec, bool tsrc, const BatchArgs& a, int block, int grid, cudaStream_t st)
{
    if (prec == PD_FP32) {
        if (tsrc) batch_kernel<true, float><<<grid, block, 0, st>>>(a);
        else batch_kernel<false, float><<<grid, block, 0, st>>>(a);
    } else {
        if (tsrc) batch_kernel<true, double><<<grid, block, 0, st>>>(a);
        else batch_kernel<false, double><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

int batch_blocks_per_sm(int prec, bool tsrc, int block)
{
    if (prec == PD_FP32) return tsrc ? occupancy<true, float>(block) : occupancy<false, float>(block);
    return tsrc ? occupancy<true, double>(block) : occupancy<false, double>(block);
}

}  // namespace pd

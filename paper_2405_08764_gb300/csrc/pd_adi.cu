// ADI micro solver (Section 4.1 runs the micro simulations with an
// alternating direction implicit scheme, two nano steps per burst), read as
// the Peaceman-Rachford splitting of the micro operator L_h = Lx + Ly + Lc:
//   Lx = alpha d_xixi - nu d_xi + phi/2   (along xi),
//   Ly = gamma d_etaeta - omega d_eta + phi/2   (along eta),
//   Lc = beta d_xieta   (explicit),
// with h = dt/2 and the source at the middle of the step:
//   (I - h Lx) w*      = w + h (Ly w + Lc w + f),
//   (I - h Ly) w^{k+1} = w* + h (Lx w* + Lc w* + f).
// The burst runs on the departure w = u - u_lift, whose ghost points are
// mirrors (the edge data is carried by the lift), so every line system is a
// constant tridiagonal matrix; its Thomas factors are computed once per
// pd_set_coeffs in FP64 and stored with the explicit line weights.  The
// forcing f = r0 + (s(t + h) - s(T)) G is the explicit scheme's forcing
// (burst records) at the half step.
//
// Layout in the kernel: a patch of M x M micro points lives in M lanes of one
// warp, lane a holding micro column a (M values) as in the explicit kernel.
// The eta lines are then in-thread: the explicit eta part and the eta Thomas
// sweep need no communication.  The xi lines go through a per-warp shared
// tile: the right-hand side is transposed so that lane b holds micro row b,
// the xi Thomas sweep and the explicit xi part of the second half step run
// in-thread, and the result is transposed back.  The mixed part takes the
// neighbouring column (row) by shuffles in either layout.
#include "pd_device.cuh"

#include <math.h>

namespace pd {

namespace {

constexpr unsigned FULL = kFull;
enum { AMODE_FUSED = 0, AMODE_DU = 1 };

__device__ __forceinline__ long long point_index(const InstDev& I, int jr, int ic, int a, int b)
{
    return (((long long)jr * I.my + b) * I.ncols + ic) * I.mx + a;
}

// One thread per (patch, direction, line).  Record of point (a, b) (8 values,
// all scaled by h = dt/2, mirror ghosts folded into the edge weights):
//   arec_c[point (a, b)]              = S, C, N, X, inv, cp, 0, 0 of the eta line a
//   arec_r[point (b, a) of the patch] = W, C, E, X, inv, cp, 0, 0 of the xi line b
// with X = h beta / (4 dxi deta) (zero on the patch boundary, where the mixed
// difference of a mirrored departure vanishes), inv the reciprocal pivot and
// cp the eliminated super-diagonal of the Thomas factorisation of I - h L_line.
template <typename real>
__global__ void adi_record_kernel(const InstDev I, const real* __restrict__ rec, real* __restrict__ arec_c,
                                  real* __restrict__ arec_r)
{
    const int M = I.mx;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)I.n_patch * 2 * M) return;
    const int line = (int)(t % M);
    const int dir = (int)((t / M) % 2);
    const int p = (int)(t / (2 * M));
    const int jr = p / I.ncols, ic = p - jr * I.ncols;
    const double h = 0.5 * I.dt;
    const double cx = 1.0 / (4.0 * I.dx * I.dy);
    double cp_prev = 0.0;
    for (int q = 0; q < M; ++q) {
        const int a = dir == 0 ? q : line, b = dir == 0 ? line : q;
        const long long pt = point_index(I, jr, ic, a, b);
        const real* c = rec + pt * 8;
        const double al = (double)c[0], be = (double)c[1], ga = (double)c[2];
        const double nu = (double)c[3], om = (double)c[4], ph = (double)c[5];
        // lower / centre / upper weights of the line operator (unscaled)
        double lo, ce, up;
        const double d = dir == 0 ? I.dx : I.dy;
        const double k2 = (dir == 0 ? al : ga) / (d * d);
        const double v = dir == 0 ? nu : om;
        ce = -2.0 * k2 + 0.5 * ph;
        if (I.conv == PD_CONV_CENTRAL) {
            lo = k2 + v / (2.0 * d);
            up = k2 - v / (2.0 * d);
        } else if (v > 0.0) {
            lo = k2 + v / d; up = k2; ce -= v / d;
        } else {
            lo = k2; up = k2 - v / d; ce += v / d;
        }
        if (q == 0) { up += lo; lo = 0.0; }
        if (q == M - 1) { lo += up; up = 0.0; }
        lo *= h; ce *= h; up *= h;
        const bool edge = a == 0 || a == M - 1 || b == 0 || b == M - 1;
        const double X = edge ? 0.0 : h * be * cx;
        // Thomas factorisation of (I - h L): sub = -lo, diag = 1 - ce, sup = -up
        const double piv = (1.0 - ce) - (-lo) * cp_prev;
        const double inv = 1.0 / piv;
        const double cp = -up * inv;
        cp_prev = cp;
        real* o = dir == 0 ? arec_r + point_index(I, jr, ic, b, a) * 8 : arec_c + pt * 8;
        o[0] = (real)lo; o[1] = (real)ce; o[2] = (real)up; o[3] = (real)X;
        o[4] = (real)inv; o[5] = (real)cp; o[6] = real(0); o[7] = real(0);
    }
}

template <typename real>
__device__ __forceinline__ void load_vec2(const real* __restrict__ p, real& x, real& y)
{
    if constexpr (sizeof(real) == 4) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        x = v.x; y = v.y;
    } else {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        x = v.x; y = v.y;
    }
}

// v (column layout, lane a holds v[b] = value at (a, b)) -> out (row layout,
// lane b holds out[a] = value at (a, b)); the same exchange maps the row
// layout back to the column layout.  tile: this warp's P M M entries; lanes of
// the unused tail (q >= P) neither write nor read and return zeros.
template <int M, typename real>
__device__ __forceinline__ void transpose(real* tile, bool own, int q, int l, const real (&v)[M], real (&out)[M])
{
    real* t = tile + q * M * M;
    __syncwarp();
    if (own) {
#pragma unroll
        for (int k = 0; k < M; ++k) t[k * M + l] = v[k];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = own ? t[l * M + k] : real(0);
}

// One warp = P patches; MODE FUSED writes U at T_next (lift -> K ADI steps ->
// restriction -> projective Euler), MODE DU writes the restricted change of
// each patch (optionally of the patches of a list).
template <int M, bool CROSS, bool TSRC, typename real, int MODE>
__global__ void __launch_bounds__(128)
patch_adi_kernel(const InstDev I, const double* __restrict__ Uc, double* __restrict__ Un,
                 const double* __restrict__ tab, double upd_scale, double bias_scale, int n_item_warps,
                 double* __restrict__ dU_out, const int* __restrict__ list, const int* __restrict__ list_n)
{
    constexpr int P = 32 / M;
    constexpr int TILE = P * M * M;
    __shared__ int slot_s[9][3];
    __shared__ double cw_s[9][3];
    __shared__ double tinfo[3];
    __shared__ real tile_s[4][TILE];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    real* ds_s = reinterpret_cast<real*>(dyn_smem);   // TSRC: K entries, s(t_k + h) - s(T)

    const int K = I.K;
    for (int t = threadIdx.x; t < 27; t += blockDim.x) {
        slot_s[t / 3][t % 3] = I.c2slot[t / 3][t % 3];
        cw_s[t / 3][t % 3] = I.c2w[t / 3][t % 3];
    }
    if (TSRC)
        for (int t = threadIdx.x; t < K; t += blockDim.x) ds_s[t] = (real)tab[t];
    if (threadIdx.x < 3) tinfo[threadIdx.x] = tab[K + threadIdx.x];
    __syncthreads();

    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;

    if (warp >= n_item_warps) {
        if (MODE != AMODE_FUSED) return;
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
    const bool own = q < P;
    int jr, icl;
    bool active;
    if (MODE == AMODE_DU && list) {
        const int n_list = *list_n;
        if (warp * P >= n_list) return;            // whole warp
        const int e = warp * P + q;
        active = own && (e < n_list);
        const int pid = list[active ? e : warp * P];
        jr = pid / I.ncols;
        icl = pid - jr * I.ncols;
    } else {
        const int wpr = (I.ncols + P - 1) / P;
        jr = warp / wpr;
        const int ic = (warp - jr * wpr) * P + q;
        active = own && (ic < I.ncols);
        icl = active ? ic : (I.ncols - 1);
    }
    const int i = I.i0 + icl, j = 1 + jr;
    const int qbase = (own ? q : P - 1) * M;
    const int pidx = jr * I.ncols + icl;
    real* tile = tile_s[threadIdx.x >> 5];

    real cv[9];
    double c20, c02, u00 = 0.0, bias = 0.0;
    macro_coeffs<M, real, false>(I, Uc, i, j, a, qbase, nullptr, slot_s, cw_s, cv, c20, c02, u00);
    if (I.restrict_mode == PD_RESTRICT_MACRO) bias = (I.dx * I.dx * c20 + I.dy * I.dy * c02) * (1.0 / 6.0);

    // forcing of the half steps, h r0 = (dt r0) / 2 from the burst records, and
    // h G for the time-dependent source; column layout, then transposed
    const real sT = (real)tinfo[0];
    const real* brec = static_cast<const real*>(I.brec);
    const real* arc = static_cast<const real*>(I.arec_c);
    const real* arr = static_cast<const real*>(I.arec_r);
    const long long rowstride = (long long)I.ncols * M;
    const long long base = (long long)jr * M * rowstride + (long long)icl * M + a;
    real w[M], Rc[M], Rr[M], Gc[M], Gr[M];
#pragma unroll
    for (int b = 0; b < M; ++b) {
        const real* p = brec + (base + b * rowstride) * 16;
        real g, B0, B1, B2, B3, B4, B5, B6, B7, B8, x0, x1;
        load_vec4<real>(p + 4, x0, x1, g, B0);      // 4, 5: explicit weights, unused here
        load_vec4<real>(p + 8, B1, B2, B3, B4);
        load_vec4<real>(p + 12, B5, B6, B7, B8);
        (void)x0; (void)x1;
        real r = sT * g;
        r = fma(B0, cv[0], r); r = fma(B1, cv[1], r); r = fma(B2, cv[2], r);
        r = fma(B3, cv[3], r); r = fma(B4, cv[4], r); r = fma(B5, cv[5], r);
        r = fma(B6, cv[6], r); r = fma(B7, cv[7], r); r = fma(B8, cv[8], r);
        Rc[b] = active ? real(0.5) * r : real(0);
        Gc[b] = active ? real(0.5) * g : real(0);
        w[b] = real(0);
    }
    transpose<M, real>(tile, own, q, a, Rc, Rr);
    if (TSRC) transpose<M, real>(tile, own, q, a, Gc, Gr);

    for (int k = 0; k < K; ++k) {
        const real dsk = TSRC ? ds_s[k] : real(0);
        real v[M], d[M];
        // first half step, column layout: explicit eta part and mixed part
        if (CROSS) {
#pragma unroll
            for (int b = 0; b < M; ++b) d[b] = __shfl_down_sync(FULL, w[b], 1) - __shfl_up_sync(FULL, w[b], 1);
        }
#pragma unroll
        for (int b = 0; b < M; ++b) {
            real S, C, N, X;
            load_vec4<real>(arc + (base + b * rowstride) * 8, S, C, N, X);
            real acc = w[b] + Rc[b];
            if (TSRC) acc = fma(dsk, Gc[b], acc);
            acc = fma(C, w[b], acc);
            if (b > 0) acc = fma(S, w[b - 1], acc);
            if (b + 1 < M) acc = fma(N, w[b + 1], acc);
            if (CROSS && b > 0 && b + 1 < M) acc = fma(X, d[b + 1] - d[b - 1], acc);
            v[b] = acc;
        }
        // xi lines: transpose, Thomas sweep along the row
        real x[M];
        transpose<M, real>(tile, own, q, a, v, x);
        real cp[M];
#pragma unroll
        for (int c = 0; c < M; ++c) {
            const real* rp = arr + (base + c * rowstride) * 8;
            real inv;
            load_vec2<real>(rp + 4, inv, cp[c]);
            if (c > 0) x[c] = fma(__ldg(rp), x[c - 1], x[c]);
            x[c] *= inv;
        }
#pragma unroll
        for (int c = M - 2; c >= 0; --c) x[c] = fma(-cp[c], x[c + 1], x[c]);
        // second half step, row layout: explicit xi part and mixed part
        if (CROSS) {
#pragma unroll
            for (int c = 0; c < M; ++c) d[c] = __shfl_down_sync(FULL, x[c], 1) - __shfl_up_sync(FULL, x[c], 1);
        }
#pragma unroll
        for (int c = 0; c < M; ++c) {
            real W, C, E, X;
            load_vec4<real>(arr + (base + c * rowstride) * 8, W, C, E, X);
            real acc = x[c] + Rr[c];
            if (TSRC) acc = fma(dsk, Gr[c], acc);
            acc = fma(C, x[c], acc);
            if (c > 0) acc = fma(W, x[c - 1], acc);
            if (c + 1 < M) acc = fma(E, x[c + 1], acc);
            if (CROSS && c > 0 && c + 1 < M) acc = fma(X, d[c + 1] - d[c - 1], acc);
            v[c] = acc;
        }
        // eta lines: transpose back, Thomas sweep along the column
        transpose<M, real>(tile, own, q, a, v, w);
        real cq[M];
#pragma unroll
        for (int b = 0; b < M; ++b) {
            const real* rp = arc + (base + b * rowstride) * 8;
            real inv;
            load_vec2<real>(rp + 4, inv, cq[b]);
            if (b > 0) w[b] = fma(__ldg(rp), w[b - 1], w[b]);
            w[b] *= inv;
        }
#pragma unroll
        for (int b = M - 2; b >= 0; --b) w[b] = fma(-cq[b], w[b + 1], w[b]);
        if (!active) {
#pragma unroll
            for (int b = 0; b < M; ++b) w[b] = real(0);
        }
    }

    // trapezoid restriction of the departure, eqs. (Time_Derivative) and
    // (Extrapolation) in FP64
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
        if (MODE == AMODE_DU) {
            dU_out[pidx] = inc;
        } else {
            long long node = (long long)j * I.nxp + i;
            Un[node] = u00 + inc;
        }
    }
}

template <int M, typename real, int MODE>
cudaError_t launch_m(const InstDev& I, const double* Uc, double* Un, const double* tab, double dtm,
                     cudaStream_t st, double* dU_out, const int* list, const int* list_n)
{
    double bias_scale = (MODE == AMODE_DU) ? 1.0 : dtm * I.inv_tau;
    double upd_scale = (MODE == AMODE_DU) ? I.inv_nn : bias_scale * I.inv_nn;
    constexpr int P = 32 / M;
    int wpr = (I.ncols + P - 1) / P;
    int n_item_warps = wpr * I.nrows;
    int n_bnd_warps = (MODE == AMODE_FUSED) ? (I.n_bnd + 31) / 32 : 0;
    int n_warps = n_item_warps + n_bnd_warps;
    const int bs = 128;
    unsigned nb = (unsigned)((n_warps * 32 + bs - 1) / bs);
    bool cross = I.has_cross != 0, tsrc = I.has_tsrc != 0;
    size_t smem = tsrc ? sizeof(real) * (size_t)I.K : 0;
#define PD_ADI_LAUNCH(CR, TS) patch_adi_kernel<M, CR, TS, real, MODE><<<nb, bs, smem, st>>>(I, Uc, Un, tab, upd_scale, bias_scale, n_item_warps, dU_out, list, list_n)
    if (cross && tsrc) PD_ADI_LAUNCH(true, true);
    else if (cross) PD_ADI_LAUNCH(true, false);
    else if (tsrc) PD_ADI_LAUNCH(false, true);
    else PD_ADI_LAUNCH(false, false);
#undef PD_ADI_LAUNCH
    return cudaGetLastError();
}

template <typename real, int MODE>
cudaError_t dispatch(const InstDev& I, const double* Uc, double* Un, const double* tab, double dtm,
                     cudaStream_t st, double* dU_out = nullptr, const int* list = nullptr,
                     const int* list_n = nullptr)
{
    if (!I.arec_c || !I.arec_r || !I.brec || I.mx != I.my) return cudaErrorInvalidValue;
    switch (I.mx) {
    case 3: return launch_m<3, real, MODE>(I, Uc, Un, tab, dtm, st, dU_out, list, list_n);
    case 5: return launch_m<5, real, MODE>(I, Uc, Un, tab, dtm, st, dU_out, list, list_n);
    case 7: return launch_m<7, real, MODE>(I, Uc, Un, tab, dtm, st, dU_out, list, list_n);
    case 9: return launch_m<9, real, MODE>(I, Uc, Un, tab, dtm, st, dU_out, list, list_n);
    case 11: return launch_m<11, real, MODE>(I, Uc, Un, tab, dtm, st, dU_out, list, list_n);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_adi_records(const InstDev& I, int prec, void* arec_c, void* arec_r, cudaStream_t st)
{
    if (I.mx != I.my) return cudaErrorInvalidValue;
    long long n = (long long)I.n_patch * 2 * I.mx;
    unsigned nb = (unsigned)((n + 127) / 128);
    if (prec == PD_FP32)
        adi_record_kernel<float><<<nb, 128, 0, st>>>(I, (const float*)I.rec, (float*)arec_c, (float*)arec_r);
    else
        adi_record_kernel<double><<<nb, 128, 0, st>>>(I, (const double*)I.rec, (double*)arec_c, (double*)arec_r);
    return cudaGetLastError();
}

cudaError_t launch_adi_fused(const InstDev& I, int prec, const double* Uc, double* Un, const double* tab_row,
                             double dtm, cudaStream_t st)
{
    if (prec == PD_FP32) return dispatch<float, AMODE_FUSED>(I, Uc, Un, tab_row, dtm, st);
    return dispatch<double, AMODE_FUSED>(I, Uc, Un, tab_row, dtm, st);
}

cudaError_t launch_adi_dU(const InstDev& I, int prec, const double* U, const double* tab_row, double* dU,
                          const int* list, const int* list_n, cudaStream_t st)
{
    if (prec == PD_FP32) return dispatch<float, AMODE_DU>(I, U, nullptr, tab_row, 0.0, st, dU, list, list_n);
    return dispatch<double, AMODE_DU>(I, U, nullptr, tab_row, 0.0, st, dU, list, list_n);
}

}  // namespace pd

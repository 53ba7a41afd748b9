// Device helpers shared by the fused and the persistent macro-step kernels.
#pragma once

#include "pd_internal.h"

namespace pd {

constexpr unsigned kFull = 0xffffffffu;

template <typename real>
__device__ __forceinline__ void load_vec4(const real* __restrict__ p, real& x, real& y, real& z, real& w)
{
    if constexpr (sizeof(real) == 4) {
        float4 q = __ldg(reinterpret_cast<const float4*>(p));
        x = q.x; y = q.y; z = q.z; w = q.w;
    } else {
        double2 q0 = __ldg(reinterpret_cast<const double2*>(p));
        double2 q1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
        x = q0.x; y = q0.y; z = q1.x; w = q1.y;
    }
}

// four consecutive values of a 16-byte aligned shared array
template <typename real>
__device__ __forceinline__ void load_vec4_shared(const real* p, real& x, real& y, real& z, real& w)
{
    if constexpr (sizeof(real) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        x = q.x; y = q.y; z = q.z; w = q.w;
    } else {
        const double2 q0 = *reinterpret_cast<const double2*>(p);
        const double2 q1 = *(reinterpret_cast<const double2*>(p) + 1);
        x = q0.x; y = q0.y; z = q1.x; w = q1.y;
    }
}

__device__ __forceinline__ int wrap_col(const InstDev& I, int i)
{
    if (!I.periodic) return i;
    return i < 0 ? i + I.nxp : (i >= I.nxp ? i - I.nxp : i);
}

// K forward-Euler micro steps of the departure w, everything in registers.
// Lane a holds micro column a; east/west neighbours come from the adjacent lanes
// by shuffles, north/south from the same thread.  Rows are swept upwards with a
// rolling window: the neighbours of row b+1 are fetched (shuffles of the old
// values) before row b is overwritten, and the old value of row b-1 is kept in
// w_prev.  ds[k] = s(t_k) - s(T) for the time-dependent source.
template <int M, bool CROSS, bool TSRC, typename real, typename Tds>
__device__ __forceinline__ void burst_steps(real (&w)[M], const real (&cE)[M], const real (&cW)[M],
                                            const real (&cN)[M], const real (&cS)[M], const real (&cC)[M],
                                            const real (&cX)[M], const real (&Gs)[M], const real (&Rr)[M],
                                            const Tds* __restrict__ ds, int K)
{
    for (int k = 0; k < K; ++k) {
        const real dsk = TSRC ? (real)ds[k] : real(0);
        real e_n = __shfl_down_sync(kFull, w[0], 1);
        real v_n = __shfl_up_sync(kFull, w[0], 1);
        real d_n = e_n - v_n, d_c = d_n, d_p = d_n;
        real w_prev = real(0);
#pragma unroll
        for (int b = 0; b < M; ++b) {
            const real e_c = e_n, v_c = v_n;
            d_p = d_c;
            d_c = d_n;
            if (b + 1 < M) {
                e_n = __shfl_down_sync(kFull, w[b + 1], 1);
                v_n = __shfl_up_sync(kFull, w[b + 1], 1);
                if (CROSS) d_n = e_n - v_n;
            }
            real acc = fma(cC[b], w[b], Rr[b]);
            acc = fma(cE[b], e_c, acc);
            acc = fma(cW[b], v_c, acc);
            if (b + 1 < M) acc = fma(cN[b], w[b + 1], acc);
            if (b > 0) acc = fma(cS[b], w_prev, acc);
            if (CROSS && b > 0 && b + 1 < M) acc = fma(cX[b], d_n - d_p, acc);
            if (TSRC) acc = fma(dsk, Gs[b], acc);
            w_prev = w[b];
            w[b] = acc;
        }
    }
}

// Slot s (0..8) of the 3x3 stencil around node (i, j): one FP64 difference
// (three loads, one add, one fma).  Slots 0..2: second xi-differences at eta
// offsets -1, 0, 1; 3..5: first xi-differences; 6: first eta-difference at
// xi = 0; 7: second eta-difference at xi = 0; 8: U(0, 0).  The interpolant's
// coefficient k combines slots c2slot[k][0..2] with weights c2w[k].
template <bool L2LOAD>
__device__ __forceinline__ double stencil_slot(const InstDev& I, const double* __restrict__ Uc, int i, int j, int k)
{
    auto ld = [&](int di, int dj) -> double {
        const double* p = Uc + (long long)(j + dj) * I.nxp + wrap_col(I, i + di);
        return L2LOAD ? __ldcg(p) : __ldg(p);
    };
    int ai = 0, aj = 0, bi = 0, bj = 0, ci = 0, cj = 0;
    double wB = 0.0;
    bool neg = false, zeroC = false;
    switch (k) {
    case 0: ai = -1; aj = -1; bi = 0; bj = -1; ci = 1; cj = -1; wB = -2.0; break;
    case 1: ai = -1; aj = 0;  bi = 0; bj = 0;  ci = 1; cj = 0;  wB = -2.0; break;
    case 2: ai = -1; aj = 1;  bi = 0; bj = 1;  ci = 1; cj = 1;  wB = -2.0; break;
    case 3: ai = 1;  aj = -1; ci = -1; cj = -1; neg = true; break;
    case 4: ai = 1;  aj = 0;  ci = -1; cj = 0;  neg = true; break;
    case 5: ai = 1;  aj = 1;  ci = -1; cj = 1;  neg = true; break;
    case 6: ai = 0;  aj = 1;  ci = 0;  cj = -1; neg = true; break;
    case 7: ai = 0;  aj = -1; bi = 0; bj = 0;  ci = 0; cj = 1;  wB = -2.0; break;
    default: zeroC = true; break;   // slot 8: U(0,0)
    }
    double A = ld(ai, aj), B = ld(bi, bj), Cv = ld(ci, cj);
    if (neg) Cv = -Cv;
    if (zeroC) Cv = 0.0;
    return fma(wB, B, A + Cv);
}

// Monomial coefficients of the patch's interpolant from the FP64 macro field,
// in two FP64 phases:
//   phase 1: slot s (0..8) is one difference of the 3x3 stencil (three loads,
//            one add and one fma); lane a of a patch forms slots a, a + M, ...;
//   phase 2: coefficient k combines up to three slots (two fma, one multiply),
//            gathered by shuffles from the lanes that formed them.
// Broadcasts the FP32/FP64 copies cv[0..8] to every lane of the patch.
template <int M, typename real, bool L2LOAD>
__device__ __forceinline__ void macro_coeffs(const InstDev& I, const double* __restrict__ Uc, int i, int j, int a,
                                             int qbase, const double (*lw)[9], const int (*slot)[3],
                                             const double (*cw)[3], real cv[9], double& c20, double& c02,
                                             double& u00)
{
    (void)lw;
    auto slot_value = [&](int k) -> double { return stencil_slot<L2LOAD>(I, Uc, i, j, k); };
    if constexpr (M >= 9) {
        double x1 = slot_value(a < 9 ? a : 8);
        int k = a < 9 ? a : 8;
        double P = __shfl_sync(kFull, x1, (qbase + slot[k][0]) & 31);
        double Q = __shfl_sync(kFull, x1, (qbase + slot[k][1]) & 31);
        double R = __shfl_sync(kFull, x1, (qbase + slot[k][2]) & 31);
        double ck = fma(cw[k][1], R, fma(cw[k][0], Q, P)) * cw[k][2];
        real ckr = (real)ck;
#pragma unroll
        for (int kk = 0; kk < 9; ++kk) cv[kk] = __shfl_sync(kFull, ckr, (qbase + kk) & 31);
        c20 = __shfl_sync(kFull, ck, (qbase + 3) & 31);
        c02 = __shfl_sync(kFull, ck, (qbase + 5) & 31);
        u00 = __shfl_sync(kFull, x1, (qbase + 8) & 31);
    } else {
        constexpr int NC = (9 + M - 1) / M;
        double x1[NC];
#pragma unroll
        for (int r = 0; r < NC; ++r) x1[r] = slot_value(min(a + r * M, 8));
        // slot s lives in register s / M of lane qbase + s % M
        auto gather = [&](int s) -> double {
            const int ln = (qbase + s % M) & 31;
            double v = __shfl_sync(kFull, x1[0], ln);
#pragma unroll
            for (int rr = 1; rr < NC; ++rr) {
                const double w = __shfl_sync(kFull, x1[rr], ln);
                if (s / M == rr) v = w;
            }
            return v;
        };
        double ck[NC];
        real ckr[NC];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const int k = min(a + r * M, 8);
            const double P = gather(slot[k][0]), Q = gather(slot[k][1]), R = gather(slot[k][2]);
            ck[r] = fma(cw[k][1], R, fma(cw[k][0], Q, P)) * cw[k][2];
            ckr[r] = (real)ck[r];
        }
#pragma unroll
        for (int kk = 0; kk < 9; ++kk) cv[kk] = __shfl_sync(kFull, ckr[kk / M], (qbase + kk % M) & 31);
        c20 = __shfl_sync(kFull, ck[3 / M], (qbase + 3 % M) & 31);
        c02 = __shfl_sync(kFull, ck[5 / M], (qbase + 5 % M) & 31);
        u00 = gather(8);
    }
}

}  // namespace pd

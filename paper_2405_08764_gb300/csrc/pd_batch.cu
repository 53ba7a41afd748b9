// Batched macro step over many independent instances of uneven sizes.
//
// Every macro step launches one kernel per micro size m over the instances
// with that size.  The work is a list of items (a patch group = up to 32 / m
// patches of one patch row of one instance, or a chunk of 32 boundary nodes);
// the warps of a persistent-size grid pull items from a device counter (one
// atomic per item), so instances of different macro grids balance across the
// GPU.  A patch group runs the whole macro step of eq. (Time_Derivative) and
// eq. (Extrapolation): lift, K forward-Euler micro steps, trapezoid
// restriction, projective update.
//
// Each item runs in four phases:
//   1. the nine monomial coefficients of each patch's interpolant from the
//      FP64 macro field (FP64 stencil differences), staged in shared memory;
//   2. the burst record of every micro point of the group -- the six
//      dt-scaled stencil weights with the mirror ghosts of the departure folded
//      in, the forcing dt r of the lifted field (burst_forcing) and dt G --
//      computed by all 32 lanes over the group's points in a rolled loop and
//      written to shared memory.  The transformed coefficients come from the
//      instance's 1-D metric tables (constant K, v, f on separable or polar
//      maps) or from its per-point records;
//   3. the K micro steps with lane a of patch q holding micro column a in
//      registers (records loaded from shared memory once);
//   4. the trapezoid sum (FP32 column sums and a segmented shuffle tree) and
//      the FP64 increment dt_macro / tau * dU.
// Staging the records keeps the register footprint of the per-point set-up out
// of the burst, so each micro size runs at the occupancy its burst allows, and
// spreads the set-up of the larger sizes over lanes the burst leaves idle.
#include "pd_device.cuh"

#include <math.h>

#include <type_traits>

namespace pd {

namespace {

// Shared-memory stage of one warp: per patch the FP64 values c20, c02, U(0,0)
// (4 doubles, one pad) and the nine interpolant coefficients in the working
// precision (12, three pads); per micro point two 4-vectors of the record:
// plane 0 = (cE, cW, cN, cS), plane 1 = (cX, cC, dt r, dt G), both in point
// order ((q M + b) M + a) so that lanes of consecutive columns read
// consecutive 16-byte entries; per patch edge point the weights its ghost
// terms need.
template <int M, typename real>
struct WarpStage {
    static constexpr int P = 32 / M;
    static constexpr int NPT = P * M * M;
    static constexpr size_t fp64_off = 0;
    static constexpr size_t cv_off = fp64_off + (size_t)P * 4 * sizeof(double);
    static constexpr size_t rec0_off = cv_off + (size_t)P * 12 * sizeof(real);
    static constexpr size_t rec1_off = rec0_off + (size_t)NPT * 4 * sizeof(real);
    // table instances (separable, polar): per patch and micro row the row factors
    // of the record (12 values; polar: 8 per lane);
    static constexpr size_t row_off = rec1_off + (size_t)NPT * 4 * sizeof(real);
    // per-point-record instances instead, in the same place: per patch, side
    // (W, E, S, N) and position along it the dt-scaled stencil weight toward the
    // ghost and the cross weight, before the mirror folding
    static constexpr size_t side_off = row_off;
    static_assert(P * 4 * M * 2 <= P * M * 12 && 32 * 8 <= P * M * 12, "row region holds either use");
    // a record of zeros (8 values) for the lanes that hold no micro column
    static constexpr size_t zero_off = row_off + (size_t)P * M * 12 * sizeof(real);
    static constexpr size_t bytes = zero_off + 8 * sizeof(real);
    static_assert(cv_off % 16 == 0 && rec0_off % 16 == 0 && rec1_off % 16 == 0 && side_off % 16 == 0 &&
                  row_off % 16 == 0 && zero_off % 16 == 0, "16-byte aligned planes");
};

// The stage of a warp that runs only separable-map items (FP32): the
// east/west weights of such a point depend on its column only and stay in the
// lane's registers, the north/south weights on its row only and stay in the row
// factors, so the stage keeps one plane per point, (cX, cC, dt r, 0), besides
// the row factors, the coefficients and the zero record.
template <int M, typename real>
struct WarpStageSep {
    static constexpr int P = 32 / M;
    static constexpr int NPT = P * M * M;
    static constexpr size_t fp64_off = 0;
    static constexpr size_t cv_off = fp64_off + (size_t)P * 4 * sizeof(double);
    static constexpr size_t rec1_off = cv_off + (size_t)P * 12 * sizeof(real);
    static constexpr size_t rec0_off = rec1_off;        // no per-point weight plane
    static constexpr size_t row_off = rec1_off + (size_t)NPT * 4 * sizeof(real);
    static constexpr size_t side_off = row_off;
    static constexpr size_t zero_off = row_off + (size_t)P * M * 12 * sizeof(real);
    static constexpr size_t bytes = zero_off + 16 * sizeof(real);
    static_assert(cv_off % 16 == 0 && rec1_off % 16 == 0 && row_off % 16 == 0 && zero_off % 16 == 0,
                  "16-byte aligned planes");
};

template <int M, typename real, bool SEP>
using StageOf = typename std::conditional<SEP, WarpStageSep<M, real>, WarpStage<M, real>>::type;

template <typename real>
__device__ __forceinline__ void store_vec4_shared(real* p, real x, real y, real z, real w)
{
    if constexpr (sizeof(real) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(x, y, z, w);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(x, y);
        reinterpret_cast<double2*>(p)[1] = make_double2(z, w);
    }
}

// Slot k (0..8) of the 3x3 stencil around node (i, j) as in stencil_slot, with
// the three stencil points and weights formed by selects instead of a switch,
// so lanes forming different slots do not diverge: v = wB U_B + (U_A + sC U_C).
__device__ __forceinline__ double stencil_slot_sel(const InstDev& I, const double* __restrict__ Uc, int i, int j,
                                                   int k)
{
    const bool x2 = k < 3;                    // second xi-differences at eta offsets -1, 0, 1
    const bool x1 = (k >= 3) && (k < 6);      // first xi-differences at eta offsets -1, 0, 1
    const int eo = x2 ? k - 1 : (x1 ? k - 4 : 0);
    const int ia = x2 ? -1 : (x1 ? 1 : 0);
    const int ja = (x2 || x1) ? eo : (k == 6 ? 1 : (k == 7 ? -1 : 0));
    const int ic = -ia;
    const int jc = (x2 || x1) ? eo : -ja;
    const int jb = x2 ? eo : 0;
    const double wB = (x2 || k == 7) ? -2.0 : 0.0;
    const double sC = (x1 || k == 6) ? -1.0 : (k == 8 ? 0.0 : 1.0);
    const double A = __ldg(Uc + (long long)(j + ja) * I.nxp + wrap_col(I, i + ia));
    const double B = __ldg(Uc + (long long)(j + jb) * I.nxp + i);
    const double C = __ldg(Uc + (long long)(j + jc) * I.nxp + wrap_col(I, i + ic));
    return fma(wB, B, fma(sC, C, A));
}

// Phase 1: slot s of the 3x3 stencil (one FP64 difference) by lane qbase + s % M
// in register s / M, the coefficient k combined from three slots (two fma, one
// multiply) by lane qbase + k % M, then written to the patch's shared entry.
template <int M, typename real>
__device__ __forceinline__ void stage_coeffs(const InstDev& I, const double* __restrict__ Uc, int i, int j, int a,
                                             int qbase, bool writer, real* cvq, double* dq)
{
    constexpr int NC = (9 + M - 1) / M;
    double x1[NC];
#pragma unroll
    for (int r = 0; r < NC; ++r) x1[r] = stencil_slot_sel(I, Uc, i, j, min(a + r * M, 8));
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
#pragma unroll
    for (int r = 0; r < NC; ++r) {
        const int k = min(a + r * M, 8);
        const double P = gather(I.c2slot[k][0]), Q = gather(I.c2slot[k][1]), R = gather(I.c2slot[k][2]);
        // the combination of differences needs FP64 (it cancels); its scale is
        // applied in the working precision (one FP64 multiply less per round on
        // the FP32 path), in FP64 only where the MACRO reference bias reads c20, c02
        const double cp = fma(I.c2w[k][1], R, fma(I.c2w[k][0], Q, P));
        const bool writes = writer && a + r * M < 9;
        if constexpr (sizeof(real) == 4) {
            if (writes) cvq[k] = (real)cp * I.c2sf[k];
        } else {
            if (writes) cvq[k] = cp * I.c2w[k][2];
        }
        if (writes) {
            if (I.restrict_mode == PD_RESTRICT_MACRO) {
                if (k == 3) dq[0] = cp * I.c2w[k][2];
                if (k == 5) dq[1] = cp * I.c2w[k][2];
            }
            if (k == 8) dq[2] = x1[r];     // slot 8 is U(0, 0)
        }
    }
}

// d/dxi and d/deta of (P - u0) at an edge, the parts of the Neumann data of
// eq. (edge) that the quadratic lift does not carry (see edge_gap_xi/_eta)
template <typename real>
__device__ __forceinline__ real gap_xi(real c21, real c12, real c22, real s, real t)
{
    return t * (real(2) * c21 * s + c12 * t + real(2) * c22 * s * t);
}
template <typename real>
__device__ __forceinline__ real gap_eta(real c21, real c12, real c22, real s, real t)
{
    return s * (c21 * s + real(2) * c12 * t + real(2) * c22 * s * t);
}

// Ghost-neighbour terms (dt-scaled) of micro point (a, b), the part of
// burst_forcing that only edge points have, from the point's unfolded
// dt-scaled weights toward the ghosts (dW at a = 0, dE at a = M - 1, dS at
// b = 0, dN at b = M - 1) and dX.  A ghost neighbour (a', b') adds
// weight * (ghost value - lift there); the diagonal ghosts of the cross term go
// with the W/E side when a' is outside the patch, else with the S/N side.  The
// Neumann gaps are polynomials along each edge: on xi = se, gap_xi = A1 t + A2
// t^2 with A1 = 2 c21 se, A2 = c12 + 2 c22 se, so the W/E terms of row t need
// only gap(t) and gap(t + dy) - gap(t - dy) = 2 dy (A1 + 2 A2 t).
template <int M, typename real>
__device__ __forceinline__ real ghost_terms(int a, int b, real dW, real dE, real dS, real dN, real dX, real c21,
                                            real c12, real c22, real s0, real t0, real dx, real dy)
{
    real g = real(0);
    const bool aw = a == 0, ae = a == M - 1, bs = b == 0, bn = b == M - 1;
    if (aw || ae) {
        const real tb = t0 + real(b) * dy;
        const real sgx = aw ? real(-1) : real(1);
        const real se = aw ? s0 : -s0;
        const real sin_ = aw ? s0 + dx : -s0 - dx;          // s of the column next to the edge
        const real Kx = sgx * real(2) * dx;
        const real A1 = real(2) * c21 * se, A2 = c12 + real(2) * c22 * se;
        real dif = Kx * real(2) * dy * (A1 + real(2) * A2 * tb);
        if (bs) dif += real(2) * dy * gap_eta(c21, c12, c22, sin_, t0);
        if (bn) dif += real(2) * dy * gap_eta(c21, c12, c22, sin_, -t0);
        g += (aw ? dW : dE) * (Kx * tb * (A1 + A2 * tb)) + sgx * dX * dif;
    }
    if (bs || bn) {
        const real sa = s0 + real(a) * dx;
        const real sgy = bs ? real(-1) : real(1);
        const real te = bs ? t0 : -t0;
        const real Ky = sgy * real(2) * dy;
        const real gm = Ky * gap_eta(c21, c12, c22, sa, te);
        const real gl = a >= 1 ? Ky * gap_eta(c21, c12, c22, sa - dx, te) : real(0);
        const real gr = a <= M - 2 ? Ky * gap_eta(c21, c12, c22, sa + dx, te) : real(0);
        g += (bs ? dS : dN) * gm + sgy * dX * (gr - gl);
    }
    return g;
}

// Burst records of a patch group whose instance has per-point coefficient
// records (heterogeneous coefficients): out of line, so that the table-mode
// set-up the uniform instances run is compiled without this path's registers.
template <typename real>
struct RecSetup {
    const real* cv_s;
    real* rec0;
    real* rec1;
    real* side;
    const real* rect;
    real idx, idy, idx2, idy2, i4dxdy, hdx, hdy, s0, t0, dx, dy, sT, dt;
    int recrow, nvalid;
    bool central;
};

template <int M, typename real>
__device__ __noinline__ void records_setup(const RecSetup<real> k, int lane)
{
    constexpr int P = 32 / M;
    constexpr int npt = P * M * M;
    const real* cv_s = k.cv_s;
    real* rec0 = k.rec0;
    real* rec1 = k.rec1;
    real* side = k.side;
    const real* rect = k.rect;
    const real idx = k.idx, idy = k.idy, idx2 = k.idx2, idy2 = k.idy2, i4dxdy = k.i4dxdy;
    const real hdx = k.hdx, hdy = k.hdy, s0 = k.s0, t0 = k.t0, dx = k.dx, dy = k.dy, sT = k.sT, dt = k.dt;
    const int recrow = k.recrow, nvalid = k.nvalid;
    const bool central = k.central;
    // general point: record of micro point (pa, pb) of patch pq from its
    // transformed coefficients, written at pt; weights and the forcing of
    // the quadratic lift as point_weights_k and burst_forcing (without its
    // ghost terms), the upwind choice by selects
    auto emit = [&](int pt, int pq, int pa, int pb, real al, real be, real ga, real nu, real om, real ph,
                    real G) {
        const real* c9 = cv_s + pq * 12;
        real C0, c10, c01, c20, c11, c02, c21_, c12_;
        load_vec4_shared<real>(c9, C0, c10, c01, c20);
        load_vec4_shared<real>(c9 + 4, c11, c02, c21_, c12_);
        const real ax = al * idx2, gy = ga * idy2;
        real wE, wW, wN, wS, ox, oy;
        real wC = -real(2) * ax - real(2) * gy + ph;
        const real wX = be * i4dxdy;
        if (central) {
            const real hn = real(0.5) * nu * idx, ho = real(0.5) * om * idy;
            wE = ax - hn; wW = ax + hn; wN = gy - ho; wS = gy + ho;
            ox = real(0); oy = real(0);
        } else {
            const real nx = nu * idx, oyv = om * idy;
            const bool pn = nu > real(0), po = om > real(0);
            wW = pn ? ax + nx : ax;
            wE = pn ? ax : ax - nx;
            wC = pn ? wC - nx : wC + nx;
            ox = pn ? -hdx : hdx;
            wS = po ? gy + oyv : gy;
            wN = po ? gy : gy - oyv;
            wC = po ? wC - oyv : wC + oyv;
            oy = po ? -hdy : hdy;
        }
        const real sa = s0 + real(pa) * dx, tb = t0 + real(pb) * dy;
        const real u0 = C0 + sa * (c10 + sa * c20 + tb * c11) + tb * (c01 + tb * c02);
        const real ux = c10 + real(2) * c20 * (sa + ox) + c11 * tb;
        const real uy = c01 + real(2) * c02 * (tb + oy) + c11 * sa;
        const real r = real(2) * c20 * al + c11 * be + real(2) * c02 * ga - nu * ux - om * uy + ph * u0 + sT * G;
        const real dE = dt * wE, dW = dt * wW, dN = dt * wN, dS = dt * wS, dX = dt * wX;
        const bool aw = pa == 0, ae = pa == M - 1, bs = pb == 0, bn = pb == M - 1;
        const real e = aw ? dE + dW : (ae ? real(0) : dE);
        const real ww = ae ? dW + dE : (aw ? real(0) : dW);
        const real n = bs ? dN + dS : (bn ? real(0) : dN);
        const real sw = bn ? dS + dN : (bs ? real(0) : dS);
        const real x = (aw || ae || bs || bn) ? real(0) : dX;
        store_vec4_shared<real>(rec0 + pt * 4, e, ww, n, sw);
        store_vec4_shared<real>(rec1 + pt * 4, x, real(1) + dt * wC, dt * r, dt * G);
        real* sq = side + pq * 8 * M;
        if (aw) { sq[2 * pb] = dW; sq[2 * pb + 1] = dX; }
        if (ae) { sq[2 * (M + pb)] = dE; sq[2 * (M + pb) + 1] = dX; }
        if (bs) { sq[2 * (2 * M + pa)] = dS; sq[2 * (2 * M + pa) + 1] = dX; }
        if (bn) { sq[2 * (3 * M + pa)] = dN; sq[2 * (3 * M + pa) + 1] = dX; }
    };
    {
        // per-point coefficient records: every lane takes points of the group in turn
#pragma unroll 1
        for (int pt = lane; pt < npt; pt += 32) {
            const int pq = pt / (M * M);
            const int rem = pt - pq * (M * M);
            const int pb = rem / M;
            const int pa = rem - pb * M;
            if (pq < nvalid) {
                const real* pr = rect + pb * recrow + (pq * M + pa) * 8;
                emit(pt, pq, pa, pb, pr[0], pr[1], pr[2], pr[3], pr[4], pr[5], pr[6]);
            } else {
                store_vec4_shared<real>(rec0 + pt * 4, real(0), real(0), real(0), real(0));
                store_vec4_shared<real>(rec1 + pt * 4, real(0), real(0), real(0), real(0));
            }
        }
    }
    __syncwarp();
    // ghost terms: a ghost neighbour (a', b') outside the patch adds
    // weight * (ghost value - lift there) (ghost_offset); the diagonal
    // ghosts of the cross term are taken by the W/E pass when a' is outside,
    // else by the S/N pass.
    const real sL = s0, sR = -s0, tB = t0, tT = -t0;
    const real s1 = s0 + dx, sM2 = -s0 - dx;              // s(1), s(M - 2)
#pragma unroll 1
    for (int sd = 0; sd < 4; ++sd) {
#pragma unroll 1
        for (int e = lane; e < P * M; e += 32) {
            const int pq = e / M;
            const int p = e - pq * M;
            if (pq >= nvalid) continue;
            const real* c9 = cv_s + pq * 12;
            const real c21 = c9[6], c12 = c9[7], c22 = c9[8];
            const real* sq = side + (size_t)pq * 8 * M + 2 * (sd * M + p);
            const real wg = sq[0], wx = sq[1];
            const real lo = p >= 1 ? real(1) : real(0), hi = p <= M - 2 ? real(1) : real(0);
            real g;
            int pt;
            if (sd < 2) {
                // W (a = 0) / E (a = M - 1): ghosts at a' = -1 / M, rows b - 1, b, b + 1
                const real sg = sd == 0 ? real(-1) : real(1);
                const real se = sd == 0 ? sL : sR;
                const real sin_ = sd == 0 ? s1 : sM2;          // s(a_in) for the eta part of a corner ghost
                const real tb = t0 + real(p) * dy;
                const real gm = sg * real(2) * dx * gap_xi(c21, c12, c22, se, tb);
                const real gdn = sg * real(2) * dx * gap_xi(c21, c12, c22, se, tb - dy) -
                                 (real(1) - lo) * real(2) * dy * gap_eta(c21, c12, c22, sin_, tB);
                const real gup = sg * real(2) * dx * gap_xi(c21, c12, c22, se, tb + dy) +
                                 (real(1) - hi) * real(2) * dy * gap_eta(c21, c12, c22, sin_, tT);
                // W: +wX go(-1, b-1) - wX go(-1, b+1); E: +wX go(M, b+1) - wX go(M, b-1)
                g = wg * gm + sg * wx * (gup - gdn);
                pt = (pq * M + p) * M + (sd == 0 ? 0 : M - 1);
            } else {
                // S (b = 0) / N (b = M - 1): ghosts at b' = -1 / M, columns a - 1, a, a + 1 inside the patch
                const real sg = sd == 2 ? real(-1) : real(1);
                const real te = sd == 2 ? tB : tT;
                const real sa = s0 + real(p) * dx;
                const real gm = sg * real(2) * dy * gap_eta(c21, c12, c22, sa, te);
                const real gl = sg * real(2) * dy * gap_eta(c21, c12, c22, sa - dx, te);
                const real gr = sg * real(2) * dy * gap_eta(c21, c12, c22, sa + dx, te);
                // S: +wX go(a-1, -1) - wX go(a+1, -1); N: +wX go(a+1, M) - wX go(a-1, M)
                g = wg * gm + sg * wx * (hi * gr - lo * gl);
                pt = (pq * M + (sd == 2 ? 0 : M - 1)) * M + p;
            }
            rec1[(size_t)pt * 4 + 2] += g;
        }
        __syncwarp();
    }
}

// K micro steps of a separable-map patch group: burst_steps with the cross
// term and without the time-dependent source (table instances carry none), the
// east/west weights one value per lane.  The same operations in the same order.
template <int M, typename real>
__device__ __forceinline__ void burst_steps_sep(real (&w)[M], const real cE, const real cW, const real (&cN)[M],
                                                const real (&cS)[M], const real (&cC)[M], const real (&cX)[M],
                                                const real (&Rr)[M], int K)
{
    for (int k = 0; k < K; ++k) {
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
                d_n = e_n - v_n;
            }
            real acc = fma(cC[b], w[b], Rr[b]);
            acc = fma(cE, e_c, acc);
            acc = fma(cW, v_c, acc);
            if (b + 1 < M) acc = fma(cN[b], w[b + 1], acc);
            if (b > 0) acc = fma(cS[b], w_prev, acc);
            if (b > 0 && b + 1 < M) acc = fma(cX[b], d_n - d_p, acc);
            w_prev = w[b];
            w[b] = acc;
        }
    }
}

template <int M, bool TSRC, typename real, bool SEP>
__device__ __forceinline__ void patch_item(const InstDev& I, const BatchItem& it, const BatchArgs& A, int lane,
                                           unsigned char* stage)
{
    using S = StageOf<M, real, SEP>;
    const int P = I.ppw;                      // patches per warp chosen for this instance (<= 32 / M)
    const int jr = it.jr;
    const int ic0 = it.wc * P;
    const int q = lane / M;
    const int a = lane - q * M;
    const int ic = ic0 + q;
    const bool active = (q < P) && (ic < I.ncols);
    const int icl = active ? ic : (I.ncols - 1);
    const int i = I.i0 + icl, j = 1 + jr;
    const int qc = q < P ? q : P - 1;
    const int qbase = qc * M;

    double* fp64_s = reinterpret_cast<double*>(stage + S::fp64_off);
    real* cv_s = reinterpret_cast<real*>(stage + S::cv_off);
    real* rec0 = reinterpret_cast<real*>(stage + S::rec0_off);
    real* rec1 = reinterpret_cast<real*>(stage + S::rec1_off);

    const double* Uc = (A.parity ? A.Sbase : A.Ubase) + I.u_off;
    double* Un = (A.parity ? A.Ubase : A.Sbase) + I.u_off;

    // ---- phase 1: interpolant coefficients (FP64 stencil) -> shared
    __syncwarp();                             // the previous item's readers are done
    stage_coeffs<M, real>(I, Uc, i, j, a, qbase, q < P, cv_s + qc * 12, fp64_s + qc * 4);
    __syncwarp();

    // ---- phase 2: burst records of the group's points, all lanes.  (a) every
    // point: weights and the forcing of the lift without ghost terms; (b) one
    // pass per patch side (uniform across the warp): the ghost-point terms of
    // the points on that side added to their forcing.
    const double* trow = (A.tab && (TSRC || I.sol != PD_SOL_NONE))
                             ? A.tab + A.tab_off[it.inst] + (long long)A.step * (I.K + kTabExtra) : nullptr;
    real sep_ef = real(0), sep_wf = real(0);  // separable-only warps: the lane's east/west weights
    {
        // instance constants in registers for the whole item (read once from
        // the instance record, never inside the point loops)
        const real sT = (TSRC && trow) ? (real)trow[I.K] : real(0);
        const RealConsts<real> kc = real_consts<real>(I);
        real hx, hy;
        if constexpr (sizeof(real) == 4) { hx = I.kf[13]; hy = I.kf[14]; }
        else { hx = I.hx; hy = I.hy; }
        const real dx = kc.dx, dy = kc.dy;
        const real s0 = real(-0.5) * hx, t0 = real(-0.5) * hy;
        const real hdx = real(0.5) * dx, hdy = real(0.5) * dy;
        const real dt = sizeof(real) == 4 ? (real)I.kf[15] : (real)I.dt;
        const int mode = I.coef_mode;
        const bool central = I.conv == PD_CONV_CENTRAL;
        const int nvalid = min(P, I.ncols - ic0);             // patches of the group inside the row
        const real K11 = kc.K11, K12 = kc.K12, K22 = kc.K22, v1 = kc.v1, v2 = kc.v2, f0 = kc.f0;
        const real idx = kc.idx, idy = kc.idy, idx2 = kc.idx2, idy2 = kc.idy2, i4dxdy = kc.i4dxdy;
        // this item's entries of the 1-D tables: columns ic0 .. ic0 + P - 1, row jr
        const real* colt = mode != COEF_RECORDS ? kc.col + (size_t)ic0 * M * 2 : nullptr;
        const real* rowt = mode != COEF_RECORDS ? kc.row + (size_t)jr * M * 4 : nullptr;
        const real* rect = mode == COEF_RECORDS
                               ? static_cast<const real*>(I.rec) + ((size_t)jr * M * I.ncols + (size_t)ic0) * M * 8
                               : nullptr;
        const int recrow = I.ncols * M * 8;                   // one micro row of the patch row, in values
        real* side = reinterpret_cast<real*>(stage + S::side_off);
        if (SEP || mode == COEF_SEPARABLE) {
            // Separable map x = X(xi), y = Y(eta) with constant K, v, f: alpha, nu
            // and the xi-weights depend on the column only, gamma, omega and the
            // eta-weights on the row only, beta = 2 K12 X'^-1 Y'^-1 is a product,
            // and the forcing splits as r = X_a + Y_b + c11 Z_ab with
            //   X_a = 2 c20 alpha - nu (c10 + 2 c20 (s + ox)) + f (c10 s + c20 s^2),
            //   Y_b = 2 c02 gamma - omega (c01 + 2 c02 (t + oy)) + f (C0 + c01 t + c02 t^2),
            //   Z_ab = beta - nu t - omega s + f s t.
            // Row factors per (patch, micro row) first, one lane each:
            real* rowq = reinterpret_cast<real*>(stage + S::row_off);
            for (int e = lane; e < P * M; e += 32) {
                const int pq = e / M;
                const int pb = e - pq * M;
                const real* rt = rowt + pb * 4;
                const real ib = rt[0], ib2 = rt[1];
                const real ga = K22 * ib * ib;
                const real om = v2 * ib + K22 * ib2;
                const real gy = ga * idy2;
                real wN, wS, wCr, oy;
                if (central) {
                    const real ho = real(0.5) * om * idy;
                    wN = gy - ho; wS = gy + ho; wCr = -real(2) * gy; oy = real(0);
                } else {
                    const real oyv = om * idy;
                    const bool po = om > real(0);
                    wS = po ? gy + oyv : gy;
                    wN = po ? gy : gy - oyv;
                    wCr = po ? -real(2) * gy - oyv : -real(2) * gy + oyv;
                    oy = po ? -hdy : hdy;
                }
                const real nu_ = dt * wN, su = dt * wS;
                const real nf = pb == 0 ? nu_ + su : (pb == M - 1 ? real(0) : nu_);
                const real sf = pb == M - 1 ? su + nu_ : (pb == 0 ? real(0) : su);
                const real crow = real(1) + dt * (wCr + f0);
                const real tb = t0 + real(pb) * dy;
                const real* c9 = cv_s + pq * 12;
                const real C0 = c9[0], c01 = c9[2], c02 = c9[5];
                const real Yb = real(2) * c02 * ga - om * (c01 + real(2) * c02 * (tb + oy)) +
                                f0 * (C0 + tb * (c01 + tb * c02));
                real* o = rowq + e * 12;
                // unfolded dt wS of the bottom row, dt wN of the top row (their ghost terms)
                const real wsn = pb == 0 ? su : (pb == M - 1 ? nu_ : real(0));
                store_vec4_shared<real>(o, nf, sf, crow, ib);
                store_vec4_shared<real>(o + 4, tb, om, Yb, wsn);
            }
            __syncwarp();
            // then each lane (q, a) holding a column walks down its micro rows
            if (q < nvalid) {
                const real* ct = colt + (q * M + a) * 2;
                const real ia = ct[0], ia2 = ct[1];
                const real al = K11 * ia * ia;
                const real nu = v1 * ia + K11 * ia2;
                const real ax = al * idx2;
                real wE, wW, wCc, ox;
                if (central) {
                    const real hn = real(0.5) * nu * idx;
                    wE = ax - hn; wW = ax + hn; wCc = -real(2) * ax; ox = real(0);
                } else {
                    const real nx = nu * idx;
                    const bool pn = nu > real(0);
                    wW = pn ? ax + nx : ax;
                    wE = pn ? ax : ax - nx;
                    wCc = pn ? -real(2) * ax - nx : -real(2) * ax + nx;
                    ox = pn ? -hdx : hdx;
                }
                const real eu = dt * wE, wu = dt * wW, ccol = dt * wCc;
                const real ef = a == 0 ? eu + wu : (a == M - 1 ? real(0) : eu);
                const real wf = a == M - 1 ? wu + eu : (a == 0 ? real(0) : wu);
                const real b2 = real(2) * K12 * ia;                   // beta / (1 / Y')
                const real xu = dt * b2 * i4dxdy;                     // unfolded cross weight / (1 / Y')
                const real xin = (a == 0 || a == M - 1) ? real(0) : xu;
                const real sa = s0 + real(a) * dx;
                const real* c9 = cv_s + q * 12;
                const real c10 = c9[1], c20 = c9[3], c11 = c9[4];
                const real Xa = real(2) * c20 * al - nu * (c10 + real(2) * c20 * (sa + ox)) + f0 * (sa * (c10 + sa * c20));
                const real fs = f0 * sa;
                const real c21 = c9[6], c12 = c9[7], c22 = c9[8];
                const real* rq = rowq + q * M * 12;
#pragma unroll 1
                for (int b = 0; b < M; ++b) {
                    real nf, sf, crow, ib, tb, om, Yb, wsn;
                    load_vec4_shared<real>(rq + b * 12, nf, sf, crow, ib);
                    load_vec4_shared<real>(rq + b * 12 + 4, tb, om, Yb, wsn);
                    real Z = b2 * ib;
                    Z = fma(-nu, tb, Z);
                    Z = fma(-om, sa, Z);
                    Z = fma(fs, tb, Z);
                    const real r = (Xa + Yb) + c11 * Z;
                    const bool redge = b == 0 || b == M - 1;
                    const real x = redge ? real(0) : xin * ib;
                    const int pt = (q * M + b) * M + a;
                    // unfolded dt wX at (a, b) = xu ib
                    const real g = ghost_terms<M, real>(a, b, wu, eu, wsn, wsn, xu * ib, c21, c12, c22, s0, t0, dx, dy);
                    if constexpr (!SEP) store_vec4_shared<real>(rec0 + pt * 4, ef, wf, nf, sf);
                    store_vec4_shared<real>(rec1 + pt * 4, x, ccol + crow, dt * r + g, real(0));
                }
                if constexpr (SEP) {
                    sep_ef = ef;
                    sep_wf = wf;
                }
            } else if (q < P) {
                // patches past the end of the row: zero records
#pragma unroll 1
                for (int b = 0; b < M; ++b) {
                    const int pt = (q * M + b) * M + a;
                    if constexpr (!SEP) store_vec4_shared<real>(rec0 + pt * 4, real(0), real(0), real(0), real(0));
                    store_vec4_shared<real>(rec1 + pt * 4, real(0), real(0), real(0), real(0));
                }
            }
        } else if constexpr (!SEP) {
          if (mode == COEF_POLAR) {
            // Polar map x = R cos xi, y = R sin xi with constant K, v, f: each
            // coefficient of table_coeffs is a sum of products of an angular factor
            // (the lane's micro column) and a radial factor (the micro row, shared by
            // all lanes), so the angular part is formed once per lane.  Radial factors
            // per micro row first, one lane each:
            real* rowq = reinterpret_cast<real*>(stage + S::row_off);
            if (lane < M) {
                const real* rt = rowt + lane * 4;
                const real iR = rt[0], iRp = rt[1], qq = rt[2];
                const real iRR = iR * iRp;
                real* o = rowq + lane * 8;
                store_vec4_shared<real>(o, iR, iRp, iR * iR, iRR);
                store_vec4_shared<real>(o + 4, iRp * iRp, (real(1) - qq) * iRR, t0 + real(lane) * dy, real(0));
            }
            __syncwarp();
            if (q < nvalid) {
                const real* ct = colt + (q * M + a) * 2;
                const real sn = ct[0], co = ct[1];
                const real ss = sn * sn, c2 = co * co, sc = sn * co;
                const real Av = ss * K11 - real(2) * sc * K12 + c2 * K22;
                const real Bv = sc * (K22 - K11) + (c2 - ss) * K12;
                const real Cv = c2 * K11 + real(2) * sc * K12 + ss * K22;
                const real Bp = (c2 - ss) * (K22 - K11) - real(4) * sc * K12;
                const real V1 = -sn * v1 + co * v2, V2 = co * v1 + sn * v2;
                const real Bv2 = real(2) * Bv;
                const real* c9 = cv_s + q * 12;
                real C0, c10, c01, c20, c11, c02, c21_, c12_;
                load_vec4_shared<real>(c9, C0, c10, c01, c20);
                load_vec4_shared<real>(c9 + 4, c11, c02, c21_, c12_);
                const real sa = s0 + real(a) * dx;
                const real uxa = c10 + real(2) * c20 * sa;               // d/dxi of the lift at (s, 0)
                const real U0a = C0 + sa * (c10 + sa * c20);
                const real c20dx = c20 * dx, c02dy = c02 * dy;
                const bool aw = a == 0, ae = a == M - 1;
                const real c22 = c9[8];
#pragma unroll 1
                for (int b = 0; b < M; ++b) {
                    real iR, iRp, iR2, iRR, iRp2, omq, tb, pad;
                    load_vec4_shared<real>(rowq + b * 8, iR, iRp, iR2, iRR);
                    load_vec4_shared<real>(rowq + b * 8 + 4, iRp2, omq, tb, pad);
                    const real al = Av * iR2, be = Bv2 * iRR, ga = Cv * iRp2;
                    const real nu = V1 * iR + Bv2 * iR2;
                    const real om = V2 * iRp - Bp * iRR - Cv * omq;
                    const real ax = al * idx2, gy = ga * idy2;
                    real wC = -real(2) * ax - real(2) * gy + f0;
                    const real wX = be * i4dxdy;
                    real wE, wW, wN, wS, ox2, oy2;                        // ox2 = 2 c20 ox, oy2 = 2 c02 oy
                    if (central) {
                        const real hn = real(0.5) * nu * idx, ho = real(0.5) * om * idy;
                        wE = ax - hn; wW = ax + hn; wN = gy - ho; wS = gy + ho;
                        ox2 = real(0); oy2 = real(0);
                    } else {
                        const real nx = nu * idx, oyv = om * idy;
                        const bool pn = nu > real(0), po = om > real(0);
                        wW = pn ? ax + nx : ax;
                        wE = pn ? ax : ax - nx;
                        wC = pn ? wC - nx : wC + nx;
                        ox2 = pn ? -c20dx : c20dx;
                        wS = po ? gy + oyv : gy;
                        wN = po ? gy : gy - oyv;
                        wC = po ? wC - oyv : wC + oyv;
                        oy2 = po ? -c02dy : c02dy;
                    }
                    const real ux = uxa + ox2 + c11 * tb;
                    const real uy = c01 + real(2) * c02 * tb + oy2 + c11 * sa;
                    const real u0 = U0a + tb * (c11 * sa + c01 + c02 * tb);
                    const real r = real(2) * c20 * al + c11 * be + real(2) * c02 * ga - nu * ux - om * uy + f0 * u0;
                    const real dE = dt * wE, dW = dt * wW, dN = dt * wN, dS = dt * wS, dX = dt * wX;
                    const bool bs = b == 0, bn = b == M - 1;
                    const int pt = (q * M + b) * M + a;
                    const real g = ghost_terms<M, real>(a, b, dW, dE, dS, dN, dX, c21_, c12_, c22, s0, t0, dx, dy);
                    store_vec4_shared<real>(rec0 + pt * 4, aw ? dE + dW : (ae ? real(0) : dE),
                                            ae ? dW + dE : (aw ? real(0) : dW), bs ? dN + dS : (bn ? real(0) : dN),
                                            bn ? dS + dN : (bs ? real(0) : dS));
                    store_vec4_shared<real>(rec1 + pt * 4, (aw || ae || bs || bn) ? real(0) : dX, real(1) + dt * wC,
                                            dt * r + g, real(0));
                }
            } else if (q < P) {
#pragma unroll 1
                for (int b = 0; b < M; ++b) {
                    const int pt = (q * M + b) * M + a;
                    store_vec4_shared<real>(rec0 + pt * 4, real(0), real(0), real(0), real(0));
                    store_vec4_shared<real>(rec1 + pt * 4, real(0), real(0), real(0), real(0));
                }
            }
          } else {
            records_setup<M, real>(RecSetup<real>{ cv_s, rec0, rec1, side, rect, idx, idy, idx2, idy2, i4dxdy, hdx, hdy,
                                                   s0, t0, dx, dy, sT, dt, recrow, nvalid, central }, lane);
          }
        }
        __syncwarp();
    }

    // ---- phase 3: K micro steps, lane (q, a) holding micro column a of patch q
    // a patch past the end of its row has zero records; a lane past the last
    // patch of the group reads the zero record for every row
    real w[M];
    const real* z = reinterpret_cast<const real*>(stage + S::zero_off);
    if constexpr (SEP) {
        // separable-only warps: per point (cX, cC, dt r) from the stage, the row's
        // north/south weights from the row factors, east/west from the lane
        real Rr[M], cN[M], cS[M], cC[M], cX[M];
        const real* r1p = q < P ? rec1 + ((size_t)(qc * M) * M + a) * 4 : z;
        const int rs = q < P ? M * 4 : 0;
        const real* rqp = q < P ? reinterpret_cast<const real*>(stage + S::row_off) + qc * M * 12 : z + 8;
        const int rqs = q < P ? 12 : 0;
#pragma unroll
        for (int b = 0; b < M; ++b) {
            real x, cc, R, Gd;
            load_vec4_shared<real>(r1p + b * rs, x, cc, R, Gd);
            (void)Gd;
            cN[b] = rqp[b * rqs];
            cS[b] = rqp[b * rqs + 1];
            cX[b] = x; cC[b] = cc;
            Rr[b] = R;
            w[b] = real(0);
        }
        burst_steps_sep<M, real>(w, sep_ef, sep_wf, cN, cS, cC, cX, Rr, I.K);
    } else {
        real Rr[M], cE[M], cW[M], cN[M], cS[M], cC[M], cX[M], Gs[M];
        const real* r0p = q < P ? rec0 + ((size_t)(qc * M) * M + a) * 4 : z;
        const real* r1p = q < P ? rec1 + ((size_t)(qc * M) * M + a) * 4 : z + 4;
        const int rs = q < P ? M * 4 : 0;
#pragma unroll
        for (int b = 0; b < M; ++b) {
            real e, ww, n, s, x, cc, R, Gd;
            load_vec4_shared<real>(r0p + b * rs, e, ww, n, s);
            load_vec4_shared<real>(r1p + b * rs, x, cc, R, Gd);
            cE[b] = e; cW[b] = ww; cN[b] = n; cS[b] = s; cX[b] = x; cC[b] = cc;
            Rr[b] = R;
            Gs[b] = Gd;
            w[b] = real(0);
        }

        // time-dependent source: ds_k read straight from the instance's time table (L1)
        if (TSRC && trow) burst_steps<M, true, true, real>(w, cE, cW, cN, cS, cC, cX, Gs, Rr, trow, I.K);
        else burst_steps<M, true, false, real>(w, cE, cW, cN, cS, cC, cX, Gs, Rr, trow, I.K);
    }

    // ---- phase 4: restriction and projective update
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
        const double* dq = fp64_s + qc * 4;
        const double2 sc = A.scale[it.inst];
        double bias = 0.0;
        if (I.restrict_mode == PD_RESTRICT_MACRO) bias = (I.dx * I.dx * dq[0] + I.dy * I.dy * dq[1]) * (1.0 / 6.0);
        double inc = fma((double)col, sc.x, bias * sc.y);
        // a non-finite restricted change shows in the working-precision sum already
        if (!isfinite(col) || !isfinite(bias)) atomicOr(I.err, ERR_NONFINITE);
        Un[(long long)j * I.nxp + i] = dq[2] + inc;
    }
}

// Out of line: inlined, the FP64 solution code of the boundary items cost the
// patch items' path 1 % on the uneven batch (measured).
__device__ __noinline__ void boundary_item(const InstDev& I, const BatchItem& it, const BatchArgs& A, int lane)
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

// Resident blocks per SM requested from the compiler for each micro size: the
// burst keeps about 9 M values per lane (departure, forcing, six weights, source
// factor), so the small micro sizes run at a higher occupancy than the largest.
template <int M, bool TSRC, typename real>
struct BatchBounds {
    // m = 11 (FP32, no time-dependent source) runs ten 64-thread blocks per SM
    // at 96 registers, which needs the shared-memory carveout at its maximum, and
    // m = 7 one block more than at 80 registers at 72 (its stage then limits it);
    // with the source term their bursts would spill there, so they keep the
    // larger budgets
    static constexpr bool max_shared = sizeof(real) == 4 && M >= 11 && !TSRC;
    static constexpr int min_blocks =
        sizeof(real) == 4 ? (M <= 5 ? 8 : M <= 7 ? (TSRC ? 6 : 7) : M <= 9 ? 5 : max_shared ? 5 : 4)
                          : (M <= 5 ? 4 : M <= 7 ? 3 : 2);
};

// Separable-only warps (FP32): their burst holds six values per micro row
// instead of eight, so they run more blocks per SM than BatchBounds allows.
template <int M>
struct SepBounds {
    static constexpr int min_blocks = M <= 5 ? 10 : M <= 7 ? 8 : M <= 9 ? 6 : 6;
};

template <int M, bool TSRC, typename real, bool SEP>
struct KernelBounds {
    static constexpr int min_blocks = SEP ? SepBounds<M>::min_blocks : BatchBounds<M, TSRC, real>::min_blocks;
    static constexpr bool max_shared = !SEP && BatchBounds<M, TSRC, real>::max_shared;
};

// One micro size per kernel: the items of this launch are the patch groups of
// the instances with m = M and those instances' boundary chunks; with SEP, the
// patch groups of the separable-map instances with m = M only (FP32).
template <int M, bool TSRC, typename real, bool SEP>
__global__ void __launch_bounds__(128, (KernelBounds<M, TSRC, real, SEP>::min_blocks)) batch_kernel(const BatchArgs A)
{
    using S = StageOf<M, real, SEP>;
    extern __shared__ __align__(16) unsigned char batch_smem[];
    unsigned char* stage = batch_smem + (size_t)(threadIdx.x >> 5) * S::bytes;
    const int lane = threadIdx.x & 31;
    if (lane < (SEP ? 16 : 8)) reinterpret_cast<real*>(stage + S::zero_off)[lane] = real(0);
    __syncwarp();
    // the next item's index, record and the head of its instance record are
    // requested while the current item runs
    auto fetch = [&]() -> int {
        int v = 0;
        if (lane == 0) v = atomicAdd(A.counter, 1);
        return __shfl_sync(kFull, v, 0);
    };
    int idx = fetch();
    BatchItem it = idx < A.n_items ? A.items[idx] : BatchItem{ 0, 0, 0, 0 };
    while (idx < A.n_items) {
        const int nidx = fetch();
        const BatchItem nit = nidx < A.n_items ? A.items[nidx] : BatchItem{ 0, 0, 0, 0 };
        if (nidx < A.n_items && lane < 4) {
            const char* p = reinterpret_cast<const char*>(A.insts + nit.inst) + lane * 128;
            asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
        }
        const InstDev& I = A.insts[it.inst];
        if (it.kind == 1) boundary_item(I, it, A, lane);
        else patch_item<M, TSRC, real, SEP>(I, it, A, lane, stage);
        idx = nidx;
        it = nit;
    }
}

template <int M, bool TSRC, typename real, bool SEP>
size_t smem_bytes(int block)
{
    return (size_t)(block / 32) * StageOf<M, real, SEP>::bytes;
}

template <int M, bool TSRC, typename real, bool SEP>
cudaError_t set_attributes(size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<M, TSRC, real, SEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (KernelBounds<M, TSRC, real, SEP>::max_shared)
        e = cudaFuncSetAttribute(batch_kernel<M, TSRC, real, SEP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int M, bool TSRC, typename real, bool SEP>
cudaError_t launch_m(const BatchArgs& a, int block, int grid, cudaStream_t st)
{
    const size_t smem = smem_bytes<M, TSRC, real, SEP>(block);
    cudaError_t e = set_attributes<M, TSRC, real, SEP>(smem);
    if (e != cudaSuccess) return e;
    batch_kernel<M, TSRC, real, SEP><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int M, bool TSRC, typename real, bool SEP>
int occupancy_m(int block)
{
    const size_t smem = smem_bytes<M, TSRC, real, SEP>(block);
    if (set_attributes<M, TSRC, real, SEP>(smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<M, TSRC, real, SEP>, block, smem) != cudaSuccess)
        return 0;
    return nb;
}

// separable-only kernels exist for FP32 and serve grids with and without a
// time-dependent source (their items carry none)
template <bool TSRC, typename real>
cudaError_t launch_tr(int M, bool sep, const BatchArgs& a, int block, int grid, cudaStream_t st)
{
    if (sep) {
        if constexpr (sizeof(real) == 4) {
            switch (M) {
            case 3: return launch_m<3, false, real, true>(a, block, grid, st);
            case 5: return launch_m<5, false, real, true>(a, block, grid, st);
            case 7: return launch_m<7, false, real, true>(a, block, grid, st);
            case 9: return launch_m<9, false, real, true>(a, block, grid, st);
            case 11: return launch_m<11, false, real, true>(a, block, grid, st);
            default: return cudaErrorInvalidValue;
            }
        }
        return cudaErrorInvalidValue;
    }
    switch (M) {
    case 3: return launch_m<3, TSRC, real, false>(a, block, grid, st);
    case 5: return launch_m<5, TSRC, real, false>(a, block, grid, st);
    case 7: return launch_m<7, TSRC, real, false>(a, block, grid, st);
    case 9: return launch_m<9, TSRC, real, false>(a, block, grid, st);
    case 11: return launch_m<11, TSRC, real, false>(a, block, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

template <bool TSRC, typename real>
int occupancy_tr(int M, bool sep, int block)
{
    if (sep) {
        if constexpr (sizeof(real) == 4) {
            switch (M) {
            case 3: return occupancy_m<3, false, real, true>(block);
            case 5: return occupancy_m<5, false, real, true>(block);
            case 7: return occupancy_m<7, false, real, true>(block);
            case 9: return occupancy_m<9, false, real, true>(block);
            case 11: return occupancy_m<11, false, real, true>(block);
            default: return 0;
            }
        }
        return 0;
    }
    switch (M) {
    case 3: return occupancy_m<3, TSRC, real, false>(block);
    case 5: return occupancy_m<5, TSRC, real, false>(block);
    case 7: return occupancy_m<7, TSRC, real, false>(block);
    case 9: return occupancy_m<9, TSRC, real, false>(block);
    case 11: return occupancy_m<11, TSRC, real, false>(block);
    default: return 0;
    }
}

}  // namespace

cudaError_t launch_batch(int prec, bool tsrc, int M, bool sep, const BatchArgs& a, int block, int grid,
                         cudaStream_t st)
{
    if (prec == PD_FP32)
        return tsrc ? launch_tr<true, float>(M, sep, a, block, grid, st) : launch_tr<false, float>(M, sep, a, block, grid, st);
    if (sep) return cudaErrorInvalidValue;
    return tsrc ? launch_tr<true, double>(M, false, a, block, grid, st) : launch_tr<false, double>(M, false, a, block, grid, st);
}

int batch_blocks_per_sm(int prec, bool tsrc, int M, bool sep, int block)
{
    if (prec == PD_FP32) return tsrc ? occupancy_tr<true, float>(M, sep, block) : occupancy_tr<false, float>(M, sep, block);
    if (sep) return 0;
    return tsrc ? occupancy_tr<true, double>(M, false, block) : occupancy_tr<false, double>(M, false, block);
}

}  // namespace pd

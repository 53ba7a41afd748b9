// Persistent dataflow macro-step kernel.
//
// When every "item warp" (P = 32 / M patches of one patch row, one micro column
// per lane) fits on the GPU at once, one cooperative launch runs a chunk of
// macro steps.  Each warp keeps its stencil weights and source factors in
// registers for the whole chunk and, instead of a grid-wide barrier, waits only
// for the (at most 8) neighbouring item warps whose macro nodes its 3x3 stencils
// read: after writing U at T_{n+1} every warp publishes its step counter with a
// release store, and a warp starts step n+1 once its neighbours' counters
// (acquire loads) reach n+1.  Warps therefore drift apart by up to a step, and
// the FP64 stencil work of one warp overlaps the FP32 bursts of others.
//
// Buffers: step n reads buf[n & 1] and writes buf[(n + 1) & 1].  A warp writes
// buf[n & 1] again only at step n + 1 (for U at T_{n+2}), after all its
// neighbours have published step n + 1, i.e. finished reading U at T_n.
//
// Every wait is bounded in wall time (globaltimer); on expiry the warp sets
// ERR_TIMEOUT in the grid's error word and returns, so the kernel always ends.
#include "pd_device.cuh"

#include <math.h>

namespace pd {

namespace {

constexpr int kPersistBlock = 64;   // two item warps per block: even load across SMs

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int M, bool CROSS, bool TSRC, typename real>
__global__ void __launch_bounds__(kPersistBlock, (sizeof(real) == 4 ? 8 : 2))
patch_persist_kernel(const InstDev I, const PersistArgs A, double upd_scale, double bias_scale, int n_item_warps)
{
    constexpr int P = 32 / M;
    constexpr int NC = (9 + M - 1) / M;
    constexpr int LANES = P * M;                          // lanes holding a micro column
    __shared__ double lw_s[9][9];
    __shared__ int slot_s[9][3];
    __shared__ double cw_s[9][3];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    // [warp in block][row b][lane < LANES][12]: forcing basis B_0..B_8 (+3 pad)
    real* Bs = reinterpret_cast<real*>(dyn_smem);
    real* ds_s = Bs + (size_t)(blockDim.x / 32) * M * LANES * 12;   // [n_steps][K]: s(t_k) - s(T_n)
    real* sT_s = ds_s + (TSRC ? A.n_steps * I.K : 0);                 // [n_steps]: s(T_n)
    __shared__ double tn_s[64];                                        // T_{n+1} (first 64 steps)

    const int K = I.K;
    const int stride = K + kTabExtra;
    for (int t = threadIdx.x; t < 81; t += blockDim.x) lw_s[t / 9][t % 9] = I.lw[t / 9][t % 9];
    for (int t = threadIdx.x; t < 27; t += blockDim.x) { slot_s[t / 3][t % 3] = I.c2slot[t / 3][t % 3]; cw_s[t / 3][t % 3] = I.c2w[t / 3][t % 3]; }
    for (int t = threadIdx.x; t < A.n_steps; t += blockDim.x) sT_s[t] = (real)A.tab[(size_t)(A.s0 + t) * stride + K];
    for (int t = threadIdx.x; t < A.n_steps && t < 64; t += blockDim.x) tn_s[t] = A.tab[(size_t)(A.s0 + t) * stride + K + 2];
    if (TSRC)
        for (int t = threadIdx.x; t < A.n_steps * K; t += blockDim.x)
            ds_s[t] = (real)A.tab[(size_t)(A.s0 + t / K) * stride + (t % K)];
    __syncthreads();

    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_item_warps) return;

    const int wpr = (I.ncols + P - 1) / P;
    const int jr = warp / wpr;
    const int wc = warp - jr * wpr;
    const int ic0 = wc * P;
    const int q = lane / M;
    const int a = lane - q * M;
    const int ic = ic0 + q;
    const bool active = (q < P) && (ic < I.ncols);
    const int icl = active ? ic : (I.ncols - 1);
    const int i = I.i0 + icl, j = 1 + jr;
    const int qbase = (q < P ? q : P - 1) * M;

    // neighbour item warp polled by lanes 0..8 (-1: none)
    int nbw = -1;
    if (lane < 9) {
        int r = jr + lane / 3 - 1, c = wc + lane % 3 - 1;
        if (I.periodic) c = (c + wpr) % wpr;
        if (r >= 0 && r < I.nrows && c >= 0 && c < wpr) nbw = r * wpr + c;
    }

    // weights and source factors: loaded once for the whole chunk
    const real* brec = static_cast<const real*>(I.brec);
    const long long rowstride = (long long)I.ncols * M;
    const long long base = (long long)jr * M * rowstride + (long long)icl * M + a;
    real cE[M], cW[M], cN[M], cS[M], cC[M], cX[M], Gs[M];
    real* Bw = Bs + (size_t)(threadIdx.x >> 5) * M * LANES * 12;
#pragma unroll
    for (int b = 0; b < M; ++b) {
        const real* p = brec + (base + b * rowstride) * 16;
        real e, ww, n, s, x, cc, g, B0, B1, B2, B3, B4, B5, B6, B7, B8;
        load_vec4<real>(p, e, ww, n, s);
        load_vec4<real>(p + 4, x, cc, g, B0);
        load_vec4<real>(p + 8, B1, B2, B3, B4);
        load_vec4<real>(p + 12, B5, B6, B7, B8);
        if (!active) { e = ww = n = s = x = cc = g = real(0); B0 = B1 = B2 = B3 = B4 = B5 = B6 = B7 = B8 = real(0); }
        cE[b] = e; cW[b] = ww; cN[b] = n; cS[b] = s; cX[b] = x; cC[b] = cc; Gs[b] = g;
        if (lane < LANES) {
            real* o = Bw + ((size_t)b * LANES + lane) * 12;
            o[0] = B0; o[1] = B1; o[2] = B2; o[3] = B3; o[4] = B4; o[5] = B5; o[6] = real(0); o[7] = real(0);
            o[8] = B6; o[9] = B7; o[10] = B8; o[11] = real(0);
        }
    }
    __syncwarp();
    const int bo0 = A.bnd_off[warp], bo1 = A.bnd_off[warp + 1];

    for (int ls = 0; ls < A.n_steps; ++ls) {
        const int n = A.s0 + ls;
        const double* Uc = (n & 1) ? A.U1 : A.U0;
        double* Un = (n & 1) ? A.U0 : A.U1;

        // wait until the neighbours have published U at T_n
        if (ls > 0) {
            bool late = false;
            if (nbw >= 0) {
                const int* f = A.flags + nbw;
                if (ld_acquire(f) < ls) {
                    unsigned long long t0 = global_ns();
                    unsigned polls = 0;
                    while (ld_acquire(f) < ls) {
                        if ((++polls & 127) == 0) {
                            if (global_ns() - t0 > (unsigned long long)A.wait_ns) { late = true; break; }
                            __nanosleep(16);
                        }
                    }
                }
            }
            if (__any_sync(kFull, late)) {
                if (lane == 0) atomicOr(I.err, ERR_TIMEOUT);
                return;
            }
            // the acquire loads of lanes 0..8 are ordered before the whole
            // warp's stencil loads by the warp barrier
            __syncwarp();
        }

        real cv[9];
        double c20, c02, u00;
        macro_coeffs<M, real, true>(I, Uc, i, j, a, qbase, lw_s, slot_s, cw_s, cv, c20, c02, u00);
        double bias = 0.0;
        if (I.restrict_mode == PD_RESTRICT_MACRO)
            bias = (I.dx * I.dx * c20 + I.dy * I.dy * c02) * (1.0 / 6.0);

        // forcing R = sum_k B_k c_k + s(T) Gs
        const real sT = sT_s[ls];
        real w[M], Rr[M];
#pragma unroll
        for (int b = 0; b < M; ++b) {
            const real* o = Bw + ((size_t)b * LANES + (lane < LANES ? lane : 0)) * 12;
            real B0 = o[0], B1 = o[1], B2 = o[2], B3 = o[3], B4 = o[4], B5 = o[5];
            real r = sT * Gs[b];
            r = fma(B0, cv[0], r); r = fma(B1, cv[1], r); r = fma(B2, cv[2], r);
            r = fma(B3, cv[3], r); r = fma(B4, cv[4], r); r = fma(B5, cv[5], r);
            // the edge-gap terms (c21, c12, c22) enter only at points next to a ghost
            if (b == 0 || b == M - 1 || a == 0 || a == M - 1) {
                real B6 = o[8], B7 = o[9], B8 = o[10];
                r = fma(B6, cv[6], r); r = fma(B7, cv[7], r); r = fma(B8, cv[8], r);
            }
            Rr[b] = active ? r : real(0);
            w[b] = real(0);
        }

        burst_steps<M, CROSS, TSRC, real>(w, cE, cW, cN, cS, cC, cX, Gs, Rr, ds_s + (TSRC ? ls * K : 0), K);

        // restriction, time derivative, projective step into the other buffer
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
            double inc = fma((double)col, upd_scale, bias * bias_scale);
            if (!isfinite(inc)) atomicOr(I.err, ERR_NONFINITE);
            long long node = (long long)j * I.nxp + i;
            Un[node] = u00 + inc;
        }
        // Dirichlet data at T_{n+1} on the boundary nodes this warp owns
        if (bo1 > bo0) {
            double tn = ls < 64 ? tn_s[ls] : A.tab[(size_t)n * stride + K + 2];
            for (int k = bo0 + lane; k < bo1; k += 32) {
                int idx = A.bnd_idx[k];
                int2 ij = I.bnd_ij[idx];
                double2 xy = I.bnd_xy[idx];
                Un[(long long)ij.y * I.nxp + ij.x] = exact_solution(I.sol, xy.x, xy.y, tn);
            }
        }
        // the warp barrier orders every lane's stores of U before lane 0's
        // release store (release is cumulative)
        __syncwarp();
        if (lane == 0 && warp != A.silent_warp) st_release(A.flags + warp, ls + 1);
    }
}

template <int M, typename real>
cudaError_t launch_m(const InstDev& I, const PersistArgs& A, cudaStream_t st)
{
    int n_item = persist_item_warps(I);
    int bs = kPersistBlock;
    unsigned nb = (unsigned)((n_item * 32 + bs - 1) / bs);
    size_t smem = persist_smem_bytes(I, sizeof(real), A.n_steps);
    double bias_scale = A.dtm * I.inv_tau;
    double upd_scale = bias_scale * I.inv_nn;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(bs);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    bool cross = I.has_cross != 0, tsrc = I.has_tsrc != 0;
    cudaError_t e = cudaSuccess;
    if (cross && tsrc) e = cudaFuncSetAttribute(patch_persist_kernel<M, true, true, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (cross) e = cudaFuncSetAttribute(patch_persist_kernel<M, true, false, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (tsrc) e = cudaFuncSetAttribute(patch_persist_kernel<M, false, true, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else e = cudaFuncSetAttribute(patch_persist_kernel<M, false, false, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cross && tsrc) return cudaLaunchKernelEx(&cfg, patch_persist_kernel<M, true, true, real>, I, A, upd_scale, bias_scale, n_item);
    if (cross) return cudaLaunchKernelEx(&cfg, patch_persist_kernel<M, true, false, real>, I, A, upd_scale, bias_scale, n_item);
    if (tsrc) return cudaLaunchKernelEx(&cfg, patch_persist_kernel<M, false, true, real>, I, A, upd_scale, bias_scale, n_item);
    return cudaLaunchKernelEx(&cfg, patch_persist_kernel<M, false, false, real>, I, A, upd_scale, bias_scale, n_item);
}

template <int M, typename real>
int max_blocks_per_sm(const InstDev& I, size_t smem)
{
    int nb = 0;
    bool cross = I.has_cross != 0, tsrc = I.has_tsrc != 0;
    cudaError_t e;
    if (cross && tsrc) e = cudaFuncSetAttribute(patch_persist_kernel<M, true, true, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (cross) e = cudaFuncSetAttribute(patch_persist_kernel<M, true, false, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (tsrc) e = cudaFuncSetAttribute(patch_persist_kernel<M, false, true, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else e = cudaFuncSetAttribute(patch_persist_kernel<M, false, false, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return 0;
    if (cross && tsrc) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, patch_persist_kernel<M, true, true, real>, kPersistBlock, smem);
    else if (cross) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, patch_persist_kernel<M, true, false, real>, kPersistBlock, smem);
    else if (tsrc) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, patch_persist_kernel<M, false, true, real>, kPersistBlock, smem);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, patch_persist_kernel<M, false, false, real>, kPersistBlock, smem);
    return e == cudaSuccess ? nb : 0;
}

template <typename real>
int blocks_per_sm(const InstDev& I, size_t smem)
{
    switch (I.mx) {
    case 5: return max_blocks_per_sm<5, real>(I, smem);
    case 7: return max_blocks_per_sm<7, real>(I, smem);
    case 9: return max_blocks_per_sm<9, real>(I, smem);
    case 11: return max_blocks_per_sm<11, real>(I, smem);
    default: return 0;
    }
}

}  // namespace

int persist_item_warps(const InstDev& I)
{
    int P = 32 / I.mx;
    return ((I.ncols + P - 1) / P) * I.nrows;
}

// dynamic shared memory of one 4-warp block: forcing basis + time table of the chunk
size_t persist_smem_bytes(const InstDev& I, size_t es, int n_steps)
{
    int P = 32 / I.mx;
    size_t basis = (size_t)(kPersistBlock / 32) * I.mx * (P * I.mx) * 12 * es;
    return basis + es * ((size_t)n_steps * (I.has_tsrc ? I.K : 0) + n_steps);
}

int persist_max_steps(const InstDev& I, int prec)
{
    // keep eight two-warp blocks per SM: about 27 KB of shared memory per block
    size_t es = prec == PD_FP32 ? 4 : 8;
    size_t budget = 27 * 1024;
    size_t base = persist_smem_bytes(I, es, 0);
    size_t per_step = es * ((I.has_tsrc ? I.K : 0) + 1);
    if (base + per_step > budget) budget = base + 16 * per_step;   // FP64: fewer blocks per SM anyway
    return (int)((budget - base) / per_step);
}

bool persist_fits(const InstDev& I, int prec)
{
    if (!(I.mx == I.my && (I.mx == 5 || I.mx == 7 || I.mx == 9 || I.mx == 11))) return false;
    int steps = persist_max_steps(I, prec);
    if (steps < 1) return false;
    size_t es = prec == PD_FP32 ? 4 : 8;
    size_t smem = persist_smem_bytes(I, es, steps);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = prec == PD_FP32 ? blocks_per_sm<float>(I, smem) : blocks_per_sm<double>(I, smem);
    long long blocks = ((long long)persist_item_warps(I) * 32 + kPersistBlock - 1) / kPersistBlock;
    return per_sm > 0 && blocks <= (long long)per_sm * nsm;
}

cudaError_t launch_persist(const InstDev& I, int prec, const PersistArgs& A, cudaStream_t st)
{
    if (prec == PD_FP32) {
        switch (I.mx) {
        case 5: return launch_m<5, float>(I, A, st);
        case 7: return launch_m<7, float>(I, A, st);
        case 9: return launch_m<9, float>(I, A, st);
        case 11: return launch_m<11, float>(I, A, st);
        }
    } else {
        switch (I.mx) {
        case 5: return launch_m<5, double>(I, A, st);
        case 7: return launch_m<7, double>(I, A, st);
        case 9: return launch_m<9, double>(I, A, st);
        case 11: return launch_m<11, double>(I, A, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace pd
